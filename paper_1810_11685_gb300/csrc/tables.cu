// Device construction of the time-invariant operator tables, computed in
// FP64 on the GPU and rounded once to the working precision T.
//
//  * medium diagonals (Section 3.2.2): C = c^2, rho0, dt / rho0_i at the
//    staggered points r + dr_i/2 (mean of the two neighbouring nodes,
//    periodic), tau = -2 alpha0 c^(y-1) and eta = 2 alpha0 c^y tan(pi y / 2)
//    (eq. Twelve) with alpha0 converted from dB MHz^-y cm^-1 to
//    Np (rad/s)^-y m^-1;
//  * PML diagonals A_i = exp(-alpha_i dt / 2) (eq. dis-pml) on a layer added
//    outside the interior, alpha_i = alpha_max (c_ref / dx) (xi / P)^4 with xi
//    the distance into the layer in grid units (staggered points at j + 1/2);
//  * k-space symbols (eq. grr and the fractional Laplacians): the staggered
//    shift-derivative factors i k_i exp(+-i k_i dx / 2), the correction
//    kappa = sinc(c_ref |k| dt / 2), |k|^(y-1) and |k|^(y-2) (set to 0 at
//    k = 0), the 2D ones divided by nx*ny to normalise the inverse FFT;
//  * FFT twiddles W_L^m = exp(-2 pi i m / L).
#include <math.h>

#include "qpat_internal.h"

namespace qpat {

__device__ __forceinline__ double wavenumber(int m, int n, double dx) {
  const int mm = (2 * m < n) ? m : m - n;       // even n: Nyquist bin is negative
  return 2.0 * M_PI * (double)mm / ((double)n * dx);
}

template <typename T>
__global__ void medium_kernel(TableOut<T> o, const double* c, const double* rho, const double* alpha_db,
                              int nx, int ny, double dt, double y, int lossless) {
  const long long G = (long long)nx * ny;
  for (long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x; g < G;
       g += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(g % nx), j = (int)(g / nx);
    const double cc = c[g], rr = rho[g];
    o.Cc[g] = (T)(cc * cc);
    o.rho0[g] = (T)rr;
    const double rsx = 0.5 * (rr + rho[(long long)j * nx + (i + 1) % nx]);
    const double rsy = 0.5 * (rr + rho[(long long)((j + 1) % ny) * nx + i]);
    o.dtrsx[g] = (T)(dt / rsx);
    o.dtrsy[g] = (T)(dt / rsy);
    if (!lossless) {
      const double np = alpha_db[g] * 100.0 / (20.0 / log(10.0)) / pow(2.0 * M_PI * 1e6, y);
      o.tau[g] = (T)(-2.0 * np * pow(cc, y - 1.0));
      o.eta[g] = (T)(2.0 * np * pow(cc, y) * tan(M_PI * y / 2.0));
    } else {
      o.tau[g] = (T)0;
      o.eta[g] = (T)0;
    }
  }
}

template <typename T>
__global__ void pml_kernel(T* node, T* stag, int n, int pml, double dx, double dt, double c_ref, double amax) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  for (int st = 0; st < 2; ++st) {
    const double s = (double)j + (st ? 0.5 : 0.0);
    double xi = 0.0;
    if (pml > 0) {
      const double lo = (double)pml, hi = (double)(n - pml - 1);
      if (s < lo) xi = lo - s;
      else if (s > hi) xi = s - hi;
    }
    double a = 1.0;
    if (pml > 0 && xi > 0.0) {
      const double r = xi / (double)pml;
      const double alpha = amax * (c_ref / dx) * r * r * r * r;
      a = exp(-alpha * dt / 2.0);
    }
    (st ? stag : node)[j] = (T)a;
  }
}

template <typename T>
__global__ void ktab_kernel(TableOut<T> o, int nx, int ny, int nxh, double dx, double dt, double c_ref, double y,
                            int lossless) {
  const long long tot = (long long)ny * nxh;
  const double norm = 1.0 / ((double)nx * (double)ny);
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < tot;
       t += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(t % nxh), j = (int)(t / nxh);
    const double kx = wavenumber(i, nx, dx), ky = wavenumber(j, ny, dx);
    const double k = sqrt(kx * kx + ky * ky);
    const double x = c_ref * k * dt / 2.0;
    const double kap = (x == 0.0) ? 1.0 : sin(x) / x;
    o.kap[t] = (T)(kap * norm);
    if (!lossless && k > 0.0) {
      o.kp1[t] = (T)(pow(k, y - 1.0) * norm);
      o.kp2[t] = (T)(pow(k, y - 2.0) * norm);
    } else {
      o.kp1[t] = (T)0;
      o.kp2[t] = (T)0;
    }
  }
}

template <typename C>
__global__ void shift_kernel(C* plus, C* minus, int count, int n, double dx) {
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= count) return;
  const double k = wavenumber(m, n, dx);
  double s, c;
  sincos(k * dx / 2.0, &s, &c);
  // i k e^{+i theta} = (-k sin theta, k cos theta); i k e^{-i theta} = (k sin theta, k cos theta)
  plus[m].x = -k * s;  plus[m].y = k * c;
  minus[m].x = k * s;  minus[m].y = k * c;
}

template <typename C>
__global__ void twiddle_kernel(C* tw, int L) {
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= L) return;
  double s, c;
  sincospi(2.0 * (double)m / (double)L, &s, &c);
  tw[m].x = c;
  tw[m].y = -s;
}

template <typename T>
cudaError_t build_tables(const TableOut<T>& o, const double* d_c, const double* d_rho, const double* d_alpha_db,
                         int nx, int ny, int nxh, int pml, double dx, double dt, double c_ref, double pml_alpha,
                         double y, int lossless, cudaStream_t s) {
  typedef typename V2<T>::t C;
  medium_kernel<T><<<512, 256, 0, s>>>(o, d_c, d_rho, d_alpha_db, nx, ny, dt, y, lossless);
  pml_kernel<T><<<(nx + 127) / 128, 128, 0, s>>>(o.ax, o.asx, nx, pml, dx, dt, c_ref, pml_alpha);
  pml_kernel<T><<<(ny + 127) / 128, 128, 0, s>>>(o.ay, o.asy, ny, pml, dx, dt, c_ref, pml_alpha);
  ktab_kernel<T><<<512, 256, 0, s>>>(o, nx, ny, nxh, dx, dt, c_ref, y, lossless);
  shift_kernel<C><<<(nxh + 127) / 128, 128, 0, s>>>(o.shxp, o.shxm, nxh, nx, dx);
  shift_kernel<C><<<(ny + 127) / 128, 128, 0, s>>>(o.shyp, o.shym, ny, ny, dx);
  twiddle_kernel<C><<<(nx + 127) / 128, 128, 0, s>>>(o.twx, nx);
  twiddle_kernel<C><<<(ny + 127) / 128, 128, 0, s>>>(o.twy, ny);
  return cudaGetLastError();
}

template cudaError_t build_tables<float>(const TableOut<float>&, const double*, const double*, const double*, int,
                                         int, int, int, double, double, double, double, double, int, cudaStream_t);
template cudaError_t build_tables<double>(const TableOut<double>&, const double*, const double*, const double*, int,
                                          int, int, int, double, double, double, double, double, int, cudaStream_t);

}  // namespace qpat
