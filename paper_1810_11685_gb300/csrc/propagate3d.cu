// 3D k-space PSTD passes (Section 3.2.3 and its transpose, Section 3.2.4).
//
// A spectral operator on the [nz][ny][nx] grid is applied as
//   x row pass  : inverse x-FFT of the incoming half spectra (two y-rows
//                 packed per complex transform), the pointwise update of one
//                 equation, forward x-FFT of the outgoing fields;
//   y pass      : forward y-FFT of every (z, kx) line;
//   z pass      : forward z-FFT of every (ky, kx) line, the k-space symbol
//                 (eq. grr per axis, or the fractional Laplacians), inverse
//                 z-FFT;
//   y pass      : inverse y-FFT;
// after which the next row pass takes over.  Velocity and density are split
// per axis (three components in 3D), so passes carry up to three spectral
// slots.  All FFTs are the generic mixed-radix shared-memory Stockham of
// fft_smem.cuh.
#include <math.h>

#include <initializer_list>
#include <type_traits>

#include "pass3_ops.cuh"

namespace qpat {

// ---- x row pass: rows (k, j0) and (k, j0+1) of problem blockIdx.z ----------
template <typename T, int PH>
__global__ void __launch_bounds__(k3Threads) row3_kernel(const Prop3<T> a) {
  typedef typename V2<T>::t C;
  constexpr int KIN = r3_kin(PH), KOUT = r3_kout(PH);
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int nx = a.nx;
  C* buf0 = reinterpret_cast<C*>(smem_raw);
  C* buf1 = buf0 + 3 * nx;
  T* sc = reinterpret_cast<T*>(buf1 + 3 * nx);
  const int b = blockIdx.z, k = blockIdx.y, j0 = 2 * blockIdx.x;
  const int tid = threadIdx.x, nth = blockDim.x;
  C* spec = a.spec + (long long)b * a.sstride;
  const long long row0 = ((long long)k * a.ny + j0) * a.pitch;
  const bool skip_in = (a.flags & kSkipInput) != 0;

  C* res = buf0;
  if (!skip_in) {
    for (int s = 0; s < KIN; ++s) {
      const C* r0 = spec + s * a.slot + row0;
      const C* r1 = r0 + a.pitch;
      for (int q = tid; q < nx; q += nth) {
        C P, Q;
        if (2 * q <= nx) {
          P = r0[q];
          Q = r1[q];
          if (q == 0 || 2 * q == nx) { P.y = (T)0; Q.y = (T)0; }
        } else {
          P = cconj(r0[nx - q]);
          Q = cconj(r1[nx - q]);
        }
        buf0[s * nx + q] = cmake<C>(P.x - Q.y, -(P.y + Q.x));
      }
    }
    __syncthreads();
    res = fft_batch(a.px, buf0, buf1, KIN, nx, a.twx);
  }
  C* oth = (res == buf0) ? buf1 : buf0;
  if (PH == A_R1 || PH == A_R1L) {
    for (int q = tid; q < 2 * nx; q += nth) sc[q] = (T)0;
    __syncthreads();
    const T* wn = a.io->w + ((long long)b * a.nt + a.n) * a.ns;
    for (int rr = 0; rr < 2; ++rr) {
      const int r = k * a.ny + j0 + rr;
      for (int q = a.rowptr[r] + tid; q < a.rowptr[r + 1]; q += nth) {
        T acc = (T)0;
        for (int e = a.pent[q]; e < a.pent[q + 1]; ++e) acc += a.ew[e] * wn[a.esens[e]];
        sc[rr * nx + a.pcol[q]] = acc;
      }
    }
    __syncthreads();
  }
  bool bad = false;
  for (int i = tid; i < nx; i += nth) {
#pragma unroll
    for (int rr = 0; rr < 2; ++rr) {
      T in[3] = {(T)0, (T)0, (T)0};
      if (!skip_in) {
#pragma unroll
        for (int s = 0; s < KIN; ++s) {
          const C z = res[s * nx + i];
          in[s] = rr ? -z.y : z.x;
        }
      }
      const T scv = (PH == A_R1 || PH == A_R1L) ? sc[rr * nx + i] : (T)0;
      T out[3];
      const long long g = ((long long)k * a.ny + j0 + rr) * a.nx + i;
      const R3Global<T> ld{a, g, (long long)b * a.gstride + g};
      row3_point<T>(a, PH, b, i, j0 + rr, k, in, scv, ld, out, bad);
#pragma unroll
      for (int s = 0; s < KOUT; ++s) {
        if (rr == 0) oth[s * nx + i].x = out[s];
        else oth[s * nx + i].y = out[s];
      }
    }
  }
  if (__syncthreads_or(bad) && tid == 0) atomicOr(a.err, 1);
  if (a.flags & kSkipOutput) return;
  C* res2 = fft_batch(a.px, oth, res, KOUT, nx, a.twx);
  for (int s = 0; s < KOUT; ++s) {
    C* w0 = spec + s * a.slot + row0;
    C* w1 = w0 + a.pitch;
    for (int q = tid; 2 * q <= nx; q += nth) {
      const C Z = res2[s * nx + q];
      const C Zm = cconj(res2[s * nx + (q == 0 ? 0 : nx - q)]);
      w0[q] = cscale(cadd(Z, Zm), (T)0.5);
      w1[q] = cscale(cmul_mi(csub(Z, Zm)), (T)0.5);
    }
  }
}

// ---- y pass: forward (INV = 0) or inverse (INV = 1) y-FFT of K slots -------
template <typename T, int K, int INV>
__global__ void __launch_bounds__(k3Threads) ypass3_kernel(const Prop3<T> a, const int gather) {
  typedef typename V2<T>::t C;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int cb = a.cby, ny = a.ny, S = ny + 1, nxh = a.nxh;
  C* buf0 = reinterpret_cast<C*>(smem_raw);
  C* buf1 = buf0 + 3 * cb * S;
  const int b = blockIdx.z, k = blockIdx.y, kx0 = blockIdx.x * cb;
  const int tid = threadIdx.x, nth = blockDim.x;
  if (gather) {
    const int blk = blockIdx.y * gridDim.x + blockIdx.x;
    gather3<T>(a, b, blk * nth + tid, gridDim.x * gridDim.y * nth);
  }
  C* spec = a.spec + (long long)b * a.sstride + (long long)k * ny * a.pitch;
  for (int s = 0; s < K; ++s)
    for (int idx = tid; idx < ny * cb; idx += nth) {
      const int ky = idx / cb, c = idx - ky * cb, kx = kx0 + c;
      C v = cmake<C>((T)0, (T)0);
      if (kx < nxh) v = spec[s * a.slot + (long long)ky * a.pitch + kx];
      buf0[(s * cb + c) * S + ky] = INV ? cconj(v) : v;
    }
  __syncthreads();
  C* res = fft_batch(a.py, buf0, buf1, K * cb, S, a.twy);
  for (int s = 0; s < K; ++s)
    for (int idx = tid; idx < ny * cb; idx += nth) {
      const int ky = idx / cb, c = idx - ky * cb, kx = kx0 + c;
      if (kx < nxh) {
        const C v = res[(s * cb + c) * S + ky];
        spec[s * a.slot + (long long)ky * a.pitch + kx] = INV ? cconj(v) : v;
      }
    }
}

// ---- z pass: forward z-FFT, k-space symbol, inverse z-FFT -----------------
template <typename T, int PH>
__global__ void __launch_bounds__(k3Threads) zpass3_kernel(const Prop3<T> a) {
  typedef typename V2<T>::t C;
  constexpr int KIN = z3_kin(PH), KOUT = z3_kout(PH);
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int cb = a.cbz, nz = a.nz, S = nz + 1, nxh = a.nxh;
  C* buf0 = reinterpret_cast<C*>(smem_raw);
  C* buf1 = buf0 + 3 * cb * S;
  const int b = blockIdx.z, ky = blockIdx.y, kx0 = blockIdx.x * cb;
  const int tid = threadIdx.x, nth = blockDim.x;
  const long long zs = (long long)a.ny * a.pitch;          // stride between z planes
  C* spec = a.spec + (long long)b * a.sstride + (long long)ky * a.pitch;
  for (int s = 0; s < KIN; ++s)
    for (int idx = tid; idx < nz * cb; idx += nth) {
      const int kz = idx / cb, c = idx - kz * cb, kx = kx0 + c;
      C v = cmake<C>((T)0, (T)0);
      if (kx < nxh) v = spec[s * a.slot + kz * zs + kx];
      buf0[(s * cb + c) * S + kz] = v;
    }
  __syncthreads();
  C* res = fft_batch(a.pz, buf0, buf1, KIN * cb, S, a.twz);
  C* oth = (res == buf0) ? buf1 : buf0;
  for (int idx = tid; idx < nz * cb; idx += nth) {
    const int c = idx / nz, kz = idx - c * nz, kx = kx0 + c;
    C X[3], o[3];
#pragma unroll
    for (int s = 0; s < 3; ++s) {
      X[s] = (s < KIN) ? res[(s * cb + c) * S + kz] : cmake<C>((T)0, (T)0);
      o[s] = cmake<C>((T)0, (T)0);
    }
    if (kx < nxh) z3_apply<T, C>(PH, z3_load<T, C>(a, PH, kx, ky, kz), z3_sx<T, C>(a, PH, kx),
                                 z3_sy<T, C>(a, PH, ky), X, o);
#pragma unroll
    for (int s = 0; s < KOUT; ++s) oth[(s * cb + c) * S + kz] = cconj(o[s]);
  }
  __syncthreads();
  C* res2 = fft_batch(a.pz, oth, res, KOUT * cb, S, a.twz);
  for (int s = 0; s < KOUT; ++s)
    for (int idx = tid; idx < nz * cb; idx += nth) {
      const int kz = idx / cb, c = idx - kz * cb, kx = kx0 + c;
      if (kx < nxh) spec[s * a.slot + kz * zs + kx] = cconj(res2[(s * cb + c) * S + kz]);
    }
}

template <typename T>
__global__ void gather3_kernel(const Prop3<T> a) {
  gather3<T>(a, blockIdx.y, blockIdx.x * blockDim.x + threadIdx.x, gridDim.x * blockDim.x);
}

// ---- tables ------------------------------------------------------------------
__device__ __forceinline__ double wavenumber3(int m, int n, double dx) {
  const int mm = (2 * m < n) ? m : m - n;
  return 2.0 * M_PI * (double)mm / ((double)n * dx);
}

template <typename T>
__global__ void medium3_kernel(Tables3<T> o, const double* c, const double* rho, const double* alpha_db, int nx,
                               int ny, int nz, double dt, double y, int lossless) {
  const long long G = (long long)nx * ny * nz;
  for (long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x; g < G; g += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(g % nx), j = (int)((g / nx) % ny), k = (int)(g / ((long long)nx * ny));
    const double cc = c[g], rr = rho[g];
    o.Cc[g] = (T)(cc * cc);
    o.rho0[g] = (T)rr;
    const long long gx = ((long long)k * ny + j) * nx + (i + 1) % nx;
    const long long gy = ((long long)k * ny + (j + 1) % ny) * nx + i;
    const long long gz = ((long long)((k + 1) % nz) * ny + j) * nx + i;
    o.dtrsx[g] = (T)(dt / (0.5 * (rr + rho[gx])));
    o.dtrsy[g] = (T)(dt / (0.5 * (rr + rho[gy])));
    o.dtrsz[g] = (T)(dt / (0.5 * (rr + rho[gz])));
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
__global__ void ktab3_kernel(Tables3<T> o, int nx, int ny, int nz, int nxh, double dx, double dt, double c_ref,
                             double y, int lossless) {
  const long long tot = (long long)nz * ny * nxh;
  const double norm = 1.0 / ((double)nx * ny * nz);
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < tot;
       t += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(t % nxh), j = (int)((t / nxh) % ny), k = (int)(t / ((long long)nxh * ny));
    const double kx = wavenumber3(i, nx, dx), ky = wavenumber3(j, ny, dx), kz = wavenumber3(k, nz, dx);
    const double km = sqrt(kx * kx + ky * ky + kz * kz);
    const double x = c_ref * km * dt / 2.0;
    o.kap[t] = (T)(((x == 0.0) ? 1.0 : sin(x) / x) * norm);
    if (!lossless && km > 0.0) {
      o.kp1[t] = (T)(pow(km, y - 1.0) * norm);
      o.kp2[t] = (T)(pow(km, y - 2.0) * norm);
    } else {
      o.kp1[t] = (T)0;
      o.kp2[t] = (T)0;
    }
  }
}

template <typename T>
__global__ void pml3_kernel(T* node, T* stag, int n, int pml, double dx, double dt, double c_ref, double amax) {
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
    double v = 1.0;
    if (pml > 0 && xi > 0.0) {
      const double r = xi / (double)pml;
      v = exp(-amax * (c_ref / dx) * r * r * r * r * dt / 2.0);
    }
    (st ? stag : node)[j] = (T)v;
  }
}

template <typename C>
__global__ void shift3_kernel(C* plus, C* minus, int count, int n, double dx) {
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= count) return;
  const double k = wavenumber3(m, n, dx);
  double s, c;
  sincos(k * dx / 2.0, &s, &c);
  plus[m].x = -k * s;
  plus[m].y = k * c;
  minus[m].x = k * s;
  minus[m].y = k * c;
}

template <typename C>
__global__ void twiddle3_kernel(C* tw, int L) {
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= L) return;
  double s, c;
  sincospi(2.0 * (double)m / (double)L, &s, &c);
  tw[m].x = c;
  tw[m].y = -s;
}

template <typename T>
cudaError_t build_tables3(const Tables3<T>& o, const double* d_c, const double* d_rho, const double* d_alpha_db,
                          int nx, int ny, int nz, int nxh, int pml, double dx, double dt, double c_ref,
                          double pml_alpha, double y, int lossless, cudaStream_t s) {
  typedef typename V2<T>::t C;
  medium3_kernel<T><<<1024, 256, 0, s>>>(o, d_c, d_rho, d_alpha_db, nx, ny, nz, dt, y, lossless);
  ktab3_kernel<T><<<1024, 256, 0, s>>>(o, nx, ny, nz, nxh, dx, dt, c_ref, y, lossless);
  pml3_kernel<T><<<(nx + 127) / 128, 128, 0, s>>>(o.ax, o.asx, nx, pml, dx, dt, c_ref, pml_alpha);
  pml3_kernel<T><<<(ny + 127) / 128, 128, 0, s>>>(o.ay, o.asy, ny, pml, dx, dt, c_ref, pml_alpha);
  pml3_kernel<T><<<(nz + 127) / 128, 128, 0, s>>>(o.az, o.asz, nz, pml, dx, dt, c_ref, pml_alpha);
  shift3_kernel<C><<<(nxh + 127) / 128, 128, 0, s>>>(o.shxp, o.shxm, nxh, nx, dx);
  shift3_kernel<C><<<(ny + 127) / 128, 128, 0, s>>>(o.shyp, o.shym, ny, ny, dx);
  shift3_kernel<C><<<(nz + 127) / 128, 128, 0, s>>>(o.shzp, o.shzm, nz, nz, dx);
  twiddle3_kernel<C><<<(nx + 127) / 128, 128, 0, s>>>(o.twx, nx);
  twiddle3_kernel<C><<<(ny + 127) / 128, 128, 0, s>>>(o.twy, ny);
  twiddle3_kernel<C><<<(nz + 127) / 128, 128, 0, s>>>(o.twz, nz);
  return cudaGetLastError();
}

// ---- launches -----------------------------------------------------------------
template <typename T>
size_t prop3_smem_row(int nx) {
  typedef typename V2<T>::t C;
  return 6 * (size_t)nx * sizeof(C) + 2 * (size_t)nx * sizeof(T);
}
template <typename T>
size_t prop3_smem_col(int n, int cb) {
  typedef typename V2<T>::t C;
  return 6 * (size_t)cb * (n + 1) * sizeof(C);
}

template <typename T, int PH>
void set3_row_attr() {
  cudaFuncSetAttribute(row3_kernel<T, PH>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
}
template <typename T, int PH>
void set3_z_attr() {
  cudaFuncSetAttribute(zpass3_kernel<T, PH>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
}
template <typename T, int K, int INV>
void set3_y_attr() {
  cudaFuncSetAttribute(ypass3_kernel<T, K, INV>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
}

template <typename T>
void prop3_init_attributes() {
  set3_row_attr<T, F_R1>(); set3_row_attr<T, F_R2>(); set3_row_attr<T, F_R3>(); set3_row_attr<T, F_R3L>();
  set3_row_attr<T, A_R1>(); set3_row_attr<T, A_R1L>(); set3_row_attr<T, A_R3>(); set3_row_attr<T, A_R5>();
  set3_z_attr<T, F_C1>(); set3_z_attr<T, F_C2>(); set3_z_attr<T, F_C3>();
  set3_z_attr<T, A_C2>(); set3_z_attr<T, A_C4>(); set3_z_attr<T, A_C6>();
  set3_y_attr<T, 1, 0>(); set3_y_attr<T, 2, 0>(); set3_y_attr<T, 3, 0>();
  set3_y_attr<T, 1, 1>(); set3_y_attr<T, 2, 1>(); set3_y_attr<T, 3, 1>();
}

bool fast3_supported(int L, int elt) {
  if (elt != 4) return false;
  switch (L) {
#define QPAT_SUP3_CASE(n) case n:
    QPAT_FAST3_CASES(QPAT_SUP3_CASE)
#undef QPAT_SUP3_CASE
    return true;
    default: return false;
  }
}

template <typename T>
void prop3_init_fast(const Prop3<T>& a) {
  if constexpr (std::is_same<T, float>::value) {
    for (int L : {a.fast_x ? a.nx : 0, a.fast_y ? a.ny : 0, a.fast_z ? a.nz : 0}) {
      switch (L) {
#define QPAT_PREP3_CASE(n) case n: prepare3_fast_len<T, n>(); break;
        QPAT_FAST3_CASES(QPAT_PREP3_CASE)
#undef QPAT_PREP3_CASE
        default: break;
      }
    }
  }
}

template <typename T>
void row3(const Prop3<T>& a, int ph, int batch, cudaStream_t s) {
  if constexpr (std::is_same<T, float>::value) if (a.fast_x) {
    switch (a.nx) {
#define QPAT_ROW3_CASE(n) case n: launch_row3_fast_len<T, n>(a, ph, batch, s); return;
      QPAT_FAST3_CASES(QPAT_ROW3_CASE)
#undef QPAT_ROW3_CASE
      default: break;
    }
  }
  const dim3 grid(a.ny / 2, a.nz, batch);
  const size_t sm = prop3_smem_row<T>(a.nx);
  switch (ph) {
    case F_R1: row3_kernel<T, F_R1><<<grid, k3Threads, sm, s>>>(a); break;
    case F_R2: row3_kernel<T, F_R2><<<grid, k3Threads, sm, s>>>(a); break;
    case F_R3: row3_kernel<T, F_R3><<<grid, k3Threads, sm, s>>>(a); break;
    case F_R3L: row3_kernel<T, F_R3L><<<grid, k3Threads, sm, s>>>(a); break;
    case A_R1: row3_kernel<T, A_R1><<<grid, k3Threads, sm, s>>>(a); break;
    case A_R1L: row3_kernel<T, A_R1L><<<grid, k3Threads, sm, s>>>(a); break;
    case A_R3: row3_kernel<T, A_R3><<<grid, k3Threads, sm, s>>>(a); break;
    case A_R5: row3_kernel<T, A_R5><<<grid, k3Threads, sm, s>>>(a); break;
    default: break;
  }
}

template <typename T>
void ypass3(const Prop3<T>& a, int K, int inv, int gather, int batch, cudaStream_t s) {
  if constexpr (std::is_same<T, float>::value) if (a.fast_y) {
    switch (a.ny) {
#define QPAT_Y3_CASE(n) case n: launch_y3_fast_len<T, n>(a, K, inv, gather, batch, s); return;
      QPAT_FAST3_CASES(QPAT_Y3_CASE)
#undef QPAT_Y3_CASE
      default: break;
    }
  }
  const dim3 grid((a.nxh + a.cby - 1) / a.cby, a.nz, batch);
  const size_t sm = prop3_smem_col<T>(a.ny, a.cby);
  if (!inv) {
    if (K == 1) ypass3_kernel<T, 1, 0><<<grid, k3Threads, sm, s>>>(a, gather);
    else if (K == 2) ypass3_kernel<T, 2, 0><<<grid, k3Threads, sm, s>>>(a, gather);
    else ypass3_kernel<T, 3, 0><<<grid, k3Threads, sm, s>>>(a, gather);
  } else {
    if (K == 1) ypass3_kernel<T, 1, 1><<<grid, k3Threads, sm, s>>>(a, gather);
    else if (K == 2) ypass3_kernel<T, 2, 1><<<grid, k3Threads, sm, s>>>(a, gather);
    else ypass3_kernel<T, 3, 1><<<grid, k3Threads, sm, s>>>(a, gather);
  }
}

template <typename T>
void zpass3(const Prop3<T>& a, int ph, int batch, cudaStream_t s) {
  if constexpr (std::is_same<T, float>::value) if (a.fast_z) {
    switch (a.nz) {
#define QPAT_Z3_CASE(n) case n: launch_z3_fast_len<T, n>(a, ph, batch, s); return;
      QPAT_FAST3_CASES(QPAT_Z3_CASE)
#undef QPAT_Z3_CASE
      default: break;
    }
  }
  const dim3 grid((a.nxh + a.cbz - 1) / a.cbz, a.ny, batch);
  const size_t sm = prop3_smem_col<T>(a.nz, a.cbz);
  switch (ph) {
    case F_C1: zpass3_kernel<T, F_C1><<<grid, k3Threads, sm, s>>>(a); break;
    case F_C2: zpass3_kernel<T, F_C2><<<grid, k3Threads, sm, s>>>(a); break;
    case F_C3: zpass3_kernel<T, F_C3><<<grid, k3Threads, sm, s>>>(a); break;
    case A_C2: zpass3_kernel<T, A_C2><<<grid, k3Threads, sm, s>>>(a); break;
    case A_C4: zpass3_kernel<T, A_C4><<<grid, k3Threads, sm, s>>>(a); break;
    case A_C6: zpass3_kernel<T, A_C6><<<grid, k3Threads, sm, s>>>(a); break;
    default: break;
  }
}

// One spectral operator after a row pass with `kout` outgoing slots:
// forward y, the z pass of phase zph, inverse y.
template <typename T>
long long op3(const Prop3<T>& a, int kout, int zph, int gather, int batch, cudaStream_t s) {
  ypass3<T>(a, kout, 0, gather, batch, s);
  zpass3<T>(a, zph, batch, s);
  ypass3<T>(a, z3_kout(zph), 1, 0, batch, s);
  return 3;
}

// H_a in 3D: the loop n = -1 .. Nt - 2 of Section 3.2.3.
template <typename T>
long long seq3_forward(Prop3<T> a, int batch, bool lossless, cudaStream_t s) {
  long long cnt = 0;
  const size_t bytes = (size_t)batch * a.gstride * sizeof(T);
  T* const fields[6] = {a.vx, a.vy, a.vz, a.rx, a.ry, a.rz};
  for (int f = 0; f < 6; ++f) cudaMemsetAsync(fields[f], 0, bytes, s);
  const int nt = a.nt;
  a.n = 0;
  if (!lossless) {
    a.flags = kSkipInput | kSource;
    row3<T>(a, F_R3, batch, s); ++cnt;
    a.flags = 0;
    cnt += op3<T>(a, 2, F_C3, 0, batch, s);
    for (int n = 0; n <= nt - 2; ++n) {
      a.n = n;
      a.flags = 0;
      row3<T>(a, F_R1, batch, s); ++cnt;                  // p_n
      cnt += op3<T>(a, 1, F_C1, 1, batch, s);             // sample n, d/dr^+ p_n
      row3<T>(a, F_R2, batch, s); ++cnt;                  // v
      cnt += op3<T>(a, 3, F_C2, 0, batch, s);             // d/dr^- v
      a.flags = (n == 0) ? kSource : 0;
      row3<T>(a, F_R3, batch, s); ++cnt;                  // rho
      a.flags = 0;
      cnt += op3<T>(a, 2, F_C3, 0, batch, s);             // Y_dis, Y_abs
    }
    a.n = nt - 1;
    a.flags = kSkipOutput;
    row3<T>(a, F_R1, batch, s); ++cnt;
  } else {
    a.flags = kSkipInput | kSource;
    row3<T>(a, F_R3L, batch, s); ++cnt;
    for (int n = 0; n <= nt - 2; ++n) {
      a.n = n;
      a.flags = 0;
      cnt += op3<T>(a, 1, F_C1, 1, batch, s);
      row3<T>(a, F_R2, batch, s); ++cnt;
      cnt += op3<T>(a, 3, F_C2, 0, batch, s);
      a.flags = (n == 0) ? kSource : 0;
      row3<T>(a, F_R3L, batch, s); ++cnt;
    }
    a.n = nt - 1;
  }
  gather3_kernel<T><<<dim3((a.ns + 255) / 256, batch), 256, 0, s>>>(a);
  return cnt + 1;
}

// H_a^* in 3D: transposed steps in reverse (Section 3.2.4).
template <typename T>
long long seq3_adjoint(Prop3<T> a, int batch, bool lossless, cudaStream_t s) {
  long long cnt = 0;
  const size_t bytes = (size_t)batch * a.gstride * sizeof(T);
  T* const fields[6] = {a.vx, a.vy, a.vz, a.rx, a.ry, a.rz};
  for (int f = 0; f < 6; ++f) cudaMemsetAsync(fields[f], 0, bytes, s);
  const int nt = a.nt;
  for (int n = nt - 2; n >= -1; --n) {
    a.n = n + 1;
    const int first = (n == nt - 2) ? kSkipInput : 0;
    const int acc = (n == 0) ? kAccWrite : (n == -1 ? kAccAdd : 0);
    const int last = (n == -1) ? kSkipOutput : 0;
    if (!lossless) {
      a.flags = first;
      row3<T>(a, A_R1, batch, s); ++cnt;
      a.flags = 0;
      cnt += op3<T>(a, 2, A_C2, 0, batch, s);
      a.flags = acc | last;
      row3<T>(a, A_R3, batch, s); ++cnt;
    } else {
      a.flags = first | acc | last;
      row3<T>(a, A_R1L, batch, s); ++cnt;
    }
    if (n > -1) {
      a.flags = 0;
      cnt += op3<T>(a, 3, A_C4, 0, batch, s);
      row3<T>(a, A_R5, batch, s); ++cnt;
      cnt += op3<T>(a, 3, A_C6, 0, batch, s);
    }
  }
  return cnt;
}

#define QPAT_INST3(T)                                                                                          \
  template cudaError_t build_tables3<T>(const Tables3<T>&, const double*, const double*, const double*, int,  \
                                        int, int, int, int, double, double, double, double, double, int,       \
                                        cudaStream_t);                                                         \
  template void prop3_init_attributes<T>();                                                                    \
  template void prop3_init_fast<T>(const Prop3<T>&);                                                           \
  template size_t prop3_smem_col<T>(int, int);                                                                 \
  template long long seq3_forward<T>(Prop3<T>, int, bool, cudaStream_t);                                       \
  template long long seq3_adjoint<T>(Prop3<T>, int, bool, cudaStream_t);
QPAT_INST3(float)
QPAT_INST3(double)

}  // namespace qpat
