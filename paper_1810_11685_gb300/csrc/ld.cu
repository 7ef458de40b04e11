// Inexact-Newton reconstructions of mu, or of kappa and mu together, with TV
// regularisation: lagged diffusivity with priorconditioning (Section 5.2.1,
// Algorithms 4 and 5) and the primal-dual interior-point variant (Section
// 5.2.2, Algorithm 6).
//
// Each application of H, J or J^* runs the optical half (the diffusion solve
// and the heating map, with the kappa derivatives of Lemma 1 in the joint
// form) per illumination and the acoustic half H_a or H_a^* for all
// illuminations as one batch of the propagation kernels.  The kernels below do
// the vector work on the interior grid in FP64: the log scaling
// X = X0 exp(Xbar), the residuals, the TV face weights (C = ((D Xbar)^2 +
// beta)^(-1/2), eqs. m, m1, or their primal-dual counterpart), the M_gamma
// solves (one cooperative launch each), the dual step of Algorithm 6 and the
// Krylov vector updates.  Inner products are the library's compensated FP64
// reductions; the scalars of Algorithm 4 go to the host, which runs the
// iteration control of Algorithms 4 to 6.
#include <math.h>

#include <chrono>
#include <string>
#include <vector>

#include "grid_sync.cuh"

#include "qpat.h"
#include "qpat_internal.h"

using namespace qpat;

namespace {

constexpr int kT = 256;

inline int blocks_for(long long n) {
  long long b = (n + kT - 1) / kT;
  return (int)(b < 4096 ? (b < 1 ? 1 : b) : 4096);
}

__global__ void exp_scale_kernel(long long n, const double* mu0, const double* xbar, double* mu) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    mu[i] = mu0[i] * exp(xbar[i]);
}

template <typename T>
__global__ void resid_kernel(long long n, const T* h, const T* p, T* r) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    r[i] = h[i] - p[i];
}

// y = a x + b y
__global__ void axpby_kernel(long long n, double a, const double* x, double b, double* y) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    y[i] = a * x[i] + b * y[i];
}

// out = u o v (acc = 0) or out += u o v (acc = 1)
__global__ void hadamard_kernel(long long n, const double* u, const double* v, double* out, int acc) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    out[i] = (acc ? out[i] : 0.0) + u[i] * v[i];
}

// out = u / d
__global__ void divide_kernel(long long n, const double* u, const double* d, double* out) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    out[i] = u[i] / d[i];
}

// y = a + y (a a constant), or y = a when set
__global__ void add_const_kernel(long long n, double a, double* y, int set) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    y[i] = set ? a : y[i] + a;
}

// Conjugate-gradient steps of the M_gamma solve with the Krylov scalars in
// device memory: sc[0] = r^T z, sc[1] = p^T A p, sc[2] = the new r^T z,
// sc[3] = sum of the preconditioned residual (for the mean removal).  A zero
// denominator (an exactly converged iteration) gives a zero step.
__global__ void cg_update_kernel(long long n, const double* sc, const double* pp, const double* ap, double* z,
                                 double* rr, double* zz, const double* dg) {
  const double alpha = sc[1] != 0.0 ? sc[0] / sc[1] : 0.0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    z[i] += alpha * pp[i];
    const double r = rr[i] - alpha * ap[i];
    rr[i] = r;
    zz[i] = r / dg[i];
  }
}

__global__ void cg_demean_kernel(long long n, const double* sc, double* zz) {
  const double m = sc[3] / (double)n;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    zz[i] -= m;
}

__global__ void cg_direction_kernel(long long n, const double* sc, const double* zz, double* pp) {
  const double beta = sc[0] != 0.0 ? sc[2] / sc[0] : 0.0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    pp[i] = zz[i] + beta * pp[i];
}

__global__ void cg_rotate_kernel(double* sc) {
  if (threadIdx.x == 0 && blockIdx.x == 0) sc[0] = sc[2];
}

struct TVGrid {
  int n0, n1, n2;
  double edge, beta, gamma;
  double* wx;   // faces (i, i+1): [n2][n1][n0 - 1]
  double* wy;   // faces (j, j+1): [n2][n1 - 1][n0]
  double* wz;   // faces (k, k+1): [n2 - 1][n1][n0]
};

// Face weight a^2 C_l of M = D^T C D: the row of D for face l holds +a, -a,
// so (D Xbar)_l = a (Xbar_j1 - Xbar_j2) and M couples the two cells with
// a^2 / sqrt((D Xbar)_l^2 + beta) (eq. m1).
__device__ __forceinline__ double tv_face(double a, double beta, double x1, double x2) {
  const double g = a * (x1 - x2);
  return a * a / sqrt(g * g + beta);
}

__global__ void tv_weights_kernel(TVGrid t, const double* xbar) {
  const long long N = (long long)t.n0 * t.n1 * t.n2;
  for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < N; c += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(c % t.n0);
    const int j = (int)((c / t.n0) % t.n1);
    const int k = (int)(c / ((long long)t.n0 * t.n1));
    if (i + 1 < t.n0) t.wx[((long long)k * t.n1 + j) * (t.n0 - 1) + i] = tv_face(t.edge, t.beta, xbar[c], xbar[c + 1]);
    if (j + 1 < t.n1) t.wy[((long long)k * (t.n1 - 1) + j) * t.n0 + i] = tv_face(t.edge, t.beta, xbar[c], xbar[c + t.n0]);
    if (k + 1 < t.n2)
      t.wz[((long long)k * t.n1 + j) * t.n0 + i] = tv_face(t.edge, t.beta, xbar[c], xbar[c + (long long)t.n0 * t.n1]);
  }
}

// out = M_gamma u (diag_only: out = the diagonal of M_gamma)
__global__ void tv_apply_kernel(TVGrid t, const double* u, double* out, int diag_only) {
  const long long N = (long long)t.n0 * t.n1 * t.n2;
  const long long sxy = (long long)t.n0 * t.n1;
  for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < N; c += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(c % t.n0);
    const int j = (int)((c / t.n0) % t.n1);
    const int k = (int)(c / sxy);
    const double uc = diag_only ? 1.0 : u[c];
    double acc = t.gamma * uc, w;
    if (i > 0) { w = t.wx[((long long)k * t.n1 + j) * (t.n0 - 1) + i - 1]; acc += w * (uc - (diag_only ? 0.0 : u[c - 1])); }
    if (i + 1 < t.n0) { w = t.wx[((long long)k * t.n1 + j) * (t.n0 - 1) + i]; acc += w * (uc - (diag_only ? 0.0 : u[c + 1])); }
    if (j > 0) { w = t.wy[((long long)k * (t.n1 - 1) + j - 1) * t.n0 + i]; acc += w * (uc - (diag_only ? 0.0 : u[c - t.n0])); }
    if (j + 1 < t.n1) { w = t.wy[((long long)k * (t.n1 - 1) + j) * t.n0 + i]; acc += w * (uc - (diag_only ? 0.0 : u[c + t.n0])); }
    if (k > 0) { w = t.wz[((long long)(k - 1) * t.n1 + j) * t.n0 + i]; acc += w * (uc - (diag_only ? 0.0 : u[c - sxy])); }
    if (k + 1 < t.n2) { w = t.wz[((long long)k * t.n1 + j) * t.n0 + i]; acc += w * (uc - (diag_only ? 0.0 : u[c + sxy])); }
    out[c] = acc;
  }
}

// ---- faces of the primal-dual interior-point TV (Algorithm 6) --------------------
// Faces are numbered x faces first ([n2][n1][n0 - 1]), then y ([n2][n1 - 1][n0]),
// then z ([n2 - 1][n1][n0]), the layout of TVGrid's weights.
__device__ __forceinline__ long long face_count(const TVGrid& t) {
  return (long long)t.n2 * t.n1 * (t.n0 - 1) + (long long)t.n2 * (t.n1 - 1) * t.n0 +
         (long long)(t.n2 - 1) * t.n1 * t.n0;
}
// cells (c1, c2) of face f, c2 the upper neighbour
__device__ __forceinline__ void face_cells(const TVGrid& t, long long f, long long& c1, long long& c2) {
  const long long nx = (long long)t.n2 * t.n1 * (t.n0 - 1), ny = (long long)t.n2 * (t.n1 - 1) * t.n0;
  if (f < nx) {
    const long long i = f % (t.n0 - 1), r = f / (t.n0 - 1);
    c1 = r * t.n0 + i;
    c2 = c1 + 1;
  } else if (f < nx + ny) {
    const long long g = f - nx, i = g % t.n0, j = (g / t.n0) % (t.n1 - 1), k = g / ((long long)t.n0 * (t.n1 - 1));
    c1 = (k * t.n1 + j) * t.n0 + i;
    c2 = c1 + t.n0;
  } else {
    const long long g = f - nx - ny;
    c1 = g;
    c2 = g + (long long)t.n0 * t.n1;
  }
}

// M~ = D^T C (I - C chi (D d)^T) D read face by face: face l couples its two
// cells with a^2 c_l (1 - c_l chi_l g_l), g_l = a (d_c1 - d_c2) = (D d)_l,
// c_l = (g_l^2 + beta)^(-1/2) (section PD-IPM).  The weights go to t.wx.. (one
// contiguous array in face order).
__global__ void pd_weights_kernel(TVGrid t, const double* d, const double* chi) {
  const long long nf = face_count(t);
  for (long long f = blockIdx.x * (long long)blockDim.x + threadIdx.x; f < nf; f += (long long)gridDim.x * blockDim.x) {
    long long c1, c2;
    face_cells(t, f, c1, c2);
    const double g = t.edge * (d[c1] - d[c2]);
    const double c = 1.0 / sqrt(g * g + t.beta);
    t.wx[f] = t.edge * t.edge * c * (1.0 - c * chi[f] * g);
  }
}

// eq. dw face by face: dchi = c (1 - c chi g) (D dd) - chi + c g, with c and g
// at d; per-block minimum of the largest feasible step phi (|chi + phi dchi|
// <= 1) into part[blockIdx.x] (+inf where no face limits it).
__global__ void pd_dual_kernel(TVGrid t, const double* d, const double* dd, const double* chi, double* dchi,
                               double* part) {
  __shared__ double sh[kT];
  const long long nf = face_count(t);
  double phi = INFINITY;
  for (long long f = blockIdx.x * (long long)blockDim.x + threadIdx.x; f < nf; f += (long long)gridDim.x * blockDim.x) {
    long long c1, c2;
    face_cells(t, f, c1, c2);
    const double g = t.edge * (d[c1] - d[c2]);
    const double c = 1.0 / sqrt(g * g + t.beta);
    const double x = chi[f];
    const double v = c * (1.0 - c * x * g) * t.edge * (dd[c1] - dd[c2]) - x + c * g;
    dchi[f] = v;
    if (v > 0.0) phi = fmin(phi, (1.0 - x) / v);
    else if (v < 0.0) phi = fmin(phi, (-1.0 - x) / v);
  }
  sh[threadIdx.x] = phi;
  __syncthreads();
  for (int st = blockDim.x / 2; st > 0; st >>= 1) {
    if (threadIdx.x < st) sh[threadIdx.x] = fmin(sh[threadIdx.x], sh[threadIdx.x + st]);
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = sh[0];
}

__global__ void min_final_kernel(const double* part, int n, double* out) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    double m = INFINITY;
    for (int i = 0; i < n; ++i) m = fmin(m, part[i]);
    out[0] = m;
  }
}

// chi += s dchi
__global__ void pd_chi_update_kernel(long long nf, double s, const double* dchi, double* chi) {
  for (long long f = blockIdx.x * (long long)blockDim.x + threadIdx.x; f < nf; f += (long long)gridDim.x * blockDim.x)
    chi[f] += s * dchi[f];
}

// ---- the whole M_gamma solve in one CTA (grids up to kOneCtaMax cells) -------
constexpr int kCgThreads = 1024;
constexpr long long kOneCtaMax = 1LL << 18;

// Deterministic block sum (fixed tree order) of one value per thread; every
// thread gets the result.
__device__ __forceinline__ double cta_sum(double v, double* sh) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) sh[wid] = v;
  __syncthreads();
  if (wid == 0) {
    v = lane < (int)(blockDim.x >> 5) ? sh[lane] : 0.0;
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if (lane == 0) sh[32] = v;
  }
  __syncthreads();
  return sh[32];
}

__device__ __forceinline__ double tv_row(const TVGrid& t, const double* u, long long c, int diag_only) {
  const long long sxy = (long long)t.n0 * t.n1;
  const int i = (int)(c % t.n0);
  const int j = (int)((c / t.n0) % t.n1);
  const int k = (int)(c / sxy);
  const double uc = diag_only ? 1.0 : u[c];
  double acc = t.gamma * uc, w;
  if (i > 0) { w = t.wx[((long long)k * t.n1 + j) * (t.n0 - 1) + i - 1]; acc += w * (uc - (diag_only ? 0.0 : u[c - 1])); }
  if (i + 1 < t.n0) { w = t.wx[((long long)k * t.n1 + j) * (t.n0 - 1) + i]; acc += w * (uc - (diag_only ? 0.0 : u[c + 1])); }
  if (j > 0) { w = t.wy[((long long)k * (t.n1 - 1) + j - 1) * t.n0 + i]; acc += w * (uc - (diag_only ? 0.0 : u[c - t.n0])); }
  if (j + 1 < t.n1) { w = t.wy[((long long)k * (t.n1 - 1) + j) * t.n0 + i]; acc += w * (uc - (diag_only ? 0.0 : u[c + t.n0])); }
  if (k > 0) { w = t.wz[((long long)(k - 1) * t.n1 + j) * t.n0 + i]; acc += w * (uc - (diag_only ? 0.0 : u[c - sxy])); }
  if (k + 1 < t.n2) { w = t.wz[((long long)k * t.n1 + j) * t.n0 + i]; acc += w * (uc - (diag_only ? 0.0 : u[c + sxy])); }
  return acc;
}

// z = M_gamma^-1 r: exact along constants, conjugate gradients on the
// mean-free part with the diagonal preconditioner followed by removal of the
// mean (the same iteration as the multi-kernel path), in one CTA; stats[0]
// receives the number of iterations.
__global__ void __launch_bounds__(kCgThreads) tv_cg_kernel(TVGrid t, const double* r, double* z, double* rr,
                                                            double* pp, double* ap, double* zz, double* dg,
                                                            int max_iter, double tol, int* stats) {
  __shared__ double sh[33];
  const long long N = (long long)t.n0 * t.n1 * t.n2;
  const int T = blockDim.x, tid = threadIdx.x;
  double s = 0.0;
  for (long long c = tid; c < N; c += T) s += r[c];
  const double m_r = cta_sum(s, sh) / (double)N;
  s = 0.0;
  for (long long c = tid; c < N; c += T) {
    dg[c] = tv_row(t, nullptr, c, 1);
    const double v = r[c] - m_r;
    rr[c] = v;
    zz[c] = v / dg[c];
    z[c] = 0.0;
    s += zz[c];
  }
  const double m0 = cta_sum(s, sh) / (double)N;
  s = 0.0;
  for (long long c = tid; c < N; c += T) {
    zz[c] -= m0;
    pp[c] = zz[c];
    s += rr[c] * zz[c];
  }
  const double rz0 = cta_sum(s, sh);
  double rz = rz0;
  int it = 0;
  for (; rz0 > 0.0 && it < max_iter && sqrt(fabs(rz) / rz0) > tol; ++it) {
    s = 0.0;
    for (long long c = tid; c < N; c += T) {
      const double a = tv_row(t, pp, c, 0);
      ap[c] = a;
      s += pp[c] * a;
    }
    const double pap = cta_sum(s, sh);
    const double alpha = pap != 0.0 ? rz / pap : 0.0;
    s = 0.0;
    for (long long c = tid; c < N; c += T) {
      z[c] += alpha * pp[c];
      const double v = rr[c] - alpha * ap[c];
      rr[c] = v;
      zz[c] = v / dg[c];
      s += zz[c];
    }
    const double m = cta_sum(s, sh) / (double)N;
    s = 0.0;
    for (long long c = tid; c < N; c += T) {
      zz[c] -= m;
      s += rr[c] * zz[c];
    }
    const double rzn = cta_sum(s, sh);
    const double beta = rz != 0.0 ? rzn / rz : 0.0;
    for (long long c = tid; c < N; c += T) pp[c] = zz[c] + beta * pp[c];
    rz = rzn;
    __syncthreads();
  }
  for (long long c = tid; c < N; c += T) z[c] += m_r / t.gamma;
  if (tid == 0) stats[0] = it;
}

// ---- the whole M_gamma solve in one cooperative grid --------------------------
constexpr int kCoopThreads = 256;
// a grid-barrier wait gives up after this much device time
constexpr unsigned long long kBarrierLimitNs = 2000000000ull;
constexpr int kCoopMaxBlocks = 4096;

// Deterministic sum over the grid: block sums in a fixed tree order, written
// to one of two alternating partial arrays (a block may write the next sum's
// partial only after every block has read this one, which the grid barrier of
// the next sum guarantees), then every block adds all partials in index order,
// so all threads of all blocks hold the same value.  ok turns false (in the
// whole CTA) when the grid barrier gave up; the kernel must then return.
__device__ __forceinline__ double grid_sum(double v, double* sh, double* part, int& flip, const GridBar& gb,
                                           bool& ok) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) sh[wid] = v;
  __syncthreads();
  double* pa = part + flip * kCoopMaxBlocks;
  flip ^= 1;
  if (threadIdx.x == 0) {
    double b = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) b += sh[w];
    pa[blockIdx.x] = b;
  }
  ok = grid_barrier(gb);
  if (!ok) return 0.0;
  if (wid == 0) {
    double t = 0.0;
    for (int i = lane; i < (int)gridDim.x; i += 32) t += pa[i];
    for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
    if (lane == 0) sh[32] = t;
  }
  __syncthreads();
  return sh[32];
}

// The iteration of tv_cg_kernel spread over a cooperative grid: four grid
// barriers per iteration (three sums, and the new search direction before the
// next stencil reads it).  Every barrier wait is bounded (grid_sync.cuh); a
// wait that gives up leaves QPAT_ETIMEOUT in stats[1] and the kernel returns.
__global__ void __launch_bounds__(kCoopThreads) tv_cg_coop_kernel(TVGrid t, const double* r, double* z, double* rr,
                                                                   double* pp, double* ap, double* zz, double* dg,
                                                                   double* part, int max_iter, double tol,
                                                                   int* stats, GridBar gb) {
  __shared__ double sh[33];
  bool ok = true;
  int flip = 0;
  const long long N = (long long)t.n0 * t.n1 * t.n2;
  const long long G = (long long)gridDim.x * blockDim.x;
  const long long t0 = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  double s = 0.0;
  for (long long c = t0; c < N; c += G) s += r[c];
  const double m_r = grid_sum(s, sh, part, flip, gb, ok) / (double)N;
  if (!ok) return;
  s = 0.0;
  for (long long c = t0; c < N; c += G) {
    dg[c] = tv_row(t, nullptr, c, 1);
    const double v = r[c] - m_r;
    rr[c] = v;
    zz[c] = v / dg[c];
    z[c] = 0.0;
    s += zz[c];
  }
  const double m0 = grid_sum(s, sh, part, flip, gb, ok) / (double)N;
  if (!ok) return;
  s = 0.0;
  for (long long c = t0; c < N; c += G) {
    zz[c] -= m0;
    pp[c] = zz[c];
    s += rr[c] * zz[c];
  }
  const double rz0 = grid_sum(s, sh, part, flip, gb, ok);
  if (!ok) return;
  double rz = rz0;
  int it = 0;
  for (; rz0 > 0.0 && it < max_iter && sqrt(fabs(rz) / rz0) > tol; ++it) {
    s = 0.0;
    for (long long c = t0; c < N; c += G) {
      const double a = tv_row(t, pp, c, 0);
      ap[c] = a;
      s += pp[c] * a;
    }
    const double pap = grid_sum(s, sh, part, flip, gb, ok);
    if (!ok) return;
    const double alpha = pap != 0.0 ? rz / pap : 0.0;
    s = 0.0;
    for (long long c = t0; c < N; c += G) {
      z[c] += alpha * pp[c];
      const double v = rr[c] - alpha * ap[c];
      rr[c] = v;
      zz[c] = v / dg[c];
      s += zz[c];
    }
    const double m = grid_sum(s, sh, part, flip, gb, ok) / (double)N;
    if (!ok) return;
    s = 0.0;
    for (long long c = t0; c < N; c += G) {
      zz[c] -= m;
      s += rr[c] * zz[c];
    }
    const double rzn = grid_sum(s, sh, part, flip, gb, ok);
    if (!ok) return;
    const double beta = rz != 0.0 ? rzn / rz : 0.0;
    for (long long c = t0; c < N; c += G) pp[c] = zz[c] + beta * pp[c];
    rz = rzn;
    if (!grid_barrier(gb)) return;
  }
  for (long long c = t0; c < N; c += G) z[c] += m_r / t.gamma;
  if (t0 == 0) stats[0] = it;
}

// ---- ADMM with L-BFGS (Section 5.1, Algorithms 1-3) -------------------------
// Faces of one block as in face_cells.  out_f = (D x)_f = a (x_c1 - x_c2),
// minus W_f plus Uw_f when W is given.
__global__ void admm_dx_kernel(TVGrid t, const double* x, const double* W, const double* Uw, double* out) {
  const long long nf = face_count(t);
  for (long long f = blockIdx.x * (long long)blockDim.x + threadIdx.x; f < nf; f += (long long)gridDim.x * blockDim.x) {
    long long c1, c2;
    face_cells(t, f, c1, c2);
    double v = t.edge * (x[c1] - x[c2]);
    if (W) v += Uw[f] - W[f];
    out[f] = v;
  }
}

// out_c (+)= rho (D^T v)_c: +a v_f over the faces whose lower cell is c, -a v_f
// over those whose upper cell is c (faces numbered x, then y, then z).
__global__ void admm_dt_kernel(TVGrid t, const double* v, double rho, double* out, int add) {
  const long long N = (long long)t.n0 * t.n1 * t.n2;
  const long long sxy = (long long)t.n0 * t.n1;
  const long long fy0 = (long long)t.n2 * t.n1 * (t.n0 - 1);
  const long long fz0 = fy0 + (long long)t.n2 * (t.n1 - 1) * t.n0;
  for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < N; c += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(c % t.n0);
    const int j = (int)((c / t.n0) % t.n1);
    const int k = (int)(c / sxy);
    double acc = 0.0;
    const long long fx = ((long long)k * t.n1 + j) * (t.n0 - 1) + i;
    if (i + 1 < t.n0) acc += v[fx];
    if (i > 0) acc -= v[fx - 1];
    const long long fy = fy0 + ((long long)k * (t.n1 - 1) + j) * t.n0 + i;
    if (j + 1 < t.n1) acc += v[fy];
    if (j > 0) acc -= v[fy - t.n0];
    const long long fz = fz0 + ((long long)k * t.n1 + j) * t.n0 + i;
    if (k + 1 < t.n2) acc += v[fz];
    if (k > 0) acc -= v[fz - sxy];
    const double r = rho * t.edge * acc;
    out[c] = add ? out[c] + r : r;
  }
}

// eq. thre: W = max(|v| - nu, 0) sgn(v); aw = |W|
__global__ void shrink_kernel(long long n, const double* v, double nu, double* W, double* aw) {
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x) {
    const double a = fabs(v[t]) - nu;
    const double w = a > 0.0 ? (v[t] > 0.0 ? a : -a) : 0.0;
    W[t] = w;
    aw[t] = fabs(w);
  }
}

// eq. LBFGSsearch as read: d = clamp(x + d, lo, hi) - x
__global__ void project_kernel(long long n, const double* x, double lo, double hi, double* d) {
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x) {
    double y = x[t] + d[t];
    y = y < lo ? lo : (y > hi ? hi : y);
    d[t] = y - x[t];
  }
}

// series: r = h - p + u, or u += h - p when update
template <typename T>
__global__ void admm_series_kernel(long long n, const T* h, const T* p, T* u, T* r, int update) {
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x) {
    if (update) u[t] = u[t] + (h[t] - p[t]);
    else r[t] = h[t] - p[t] + u[t];
  }
}

// Device workspace of one reconstruction, freed on every exit path.
struct Work {
  std::vector<void*> ptrs;
  cudaError_t err = cudaSuccess;
  template <typename P>
  P* get(size_t count) {
    void* v = nullptr;
    if (err == cudaSuccess) err = cudaMalloc(&v, (count ? count : 1) * sizeof(P));
    if (err != cudaSuccess) return nullptr;
    ptrs.push_back(v);
    return (P*)v;
  }
  ~Work() {
    for (void* p : ptrs) cudaFree(p);
  }
};

// Host wall time of a phase, the stream drained at both ends.
struct PhaseTimer {
  double* acc;
  cudaStream_t s;
  std::chrono::steady_clock::time_point t0;
  PhaseTimer(double* a, cudaStream_t st) : acc(a), s(st) {
    cudaStreamSynchronize(s);
    t0 = std::chrono::steady_clock::now();
  }
  ~PhaseTimer() {
    cudaStreamSynchronize(s);
    *acc += std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  }
};

struct Ld {
  qpat_ctx* c;
  double sec[3] = {0, 0, 0};    // acoustic, optical, M_gamma solves
  CtxView v;
  long long N = 0, M = 0;       // interior cells, samples per series
  size_t elt = 8;
  double* partial = nullptr;
  double* dout = nullptr;
  long long products = 0, tv_iters = 0;
  TVGrid tv{};

  qpat_status cuda(cudaError_t e, const char* where) {
    if (e == cudaSuccess) return QPAT_OK;
    return (qpat_status)ctx_fail(c, e == cudaErrorMemoryAllocation ? QPAT_ENOMEM : QPAT_ECUDA,
                                 (std::string(where) + ": " + cudaGetErrorString(e)).c_str());
  }
  // FP64 inner product of two FP64 vectors of length n (host result)
  qpat_status dot(const double* a, const double* b, long long n, double* out) {
    qpat_status st = cuda(dot_compensated<double>(1, n, a, b, partial, dout, v.stream), "dot");
    if (st != QPAT_OK) return st;
    st = cuda(cudaMemcpyAsync(out, dout, sizeof(double), cudaMemcpyDeviceToHost, v.stream), "dot copy");
    if (st != QPAT_OK) return st;
    return cuda(cudaStreamSynchronize(v.stream), "dot sync");
  }
  qpat_status dot_data(const void* a, const void* b, long long n, double* out) {
    qpat_status st;
    if (v.prec == QPAT_FP32)
      st = cuda(dot_compensated<float>(1, n, (const float*)a, (const float*)b, partial, dout, v.stream), "dot");
    else
      st = cuda(dot_compensated<double>(1, n, (const double*)a, (const double*)b, partial, dout, v.stream), "dot");
    if (st != QPAT_OK) return st;
    st = cuda(cudaMemcpyAsync(out, dout, sizeof(double), cudaMemcpyDeviceToHost, v.stream), "dot copy");
    if (st != QPAT_OK) return st;
    return cuda(cudaStreamSynchronize(v.stream), "dot sync");
  }
  void axpby(double a, const double* x, double b, double* y) {
    axpby_kernel<<<blocks_for(N), kT, 0, v.stream>>>(N, a, x, b, y);
  }

  qpat_status tv_weights(const double* xbar) {
    tv_weights_kernel<<<blocks_for(N), kT, 0, v.stream>>>(tv, xbar);
    return cuda(cudaGetLastError(), "tv_weights_kernel");
  }
  void tv_apply(const double* u, double* out) { tv_apply_kernel<<<blocks_for(N), kT, 0, v.stream>>>(tv, u, out, 0); }

  // mean of an [N] vector (ones: a vector of ones)
  qpat_status mean(const double* u, const double* ones, double* out) {
    qpat_status st = dot(u, ones, N, out);
    *out /= (double)N;
    return st;
  }

  // device Krylov scalars of the M_gamma solves and a pinned host copy
  double* sc = nullptr;
  double* hsc = nullptr;
  int* cg_stats = nullptr;
  int* hstats = nullptr;
  // cooperative grid of the M_gamma solve (0: not available)
  int coop_blocks = 0;
  double* coop_part = nullptr;

  // Size the cooperative grid: one thread per cell, at most what can be
  // resident at once on the device (and kCoopMaxBlocks).
  void setup_coop() {
    int dev = 0, sms = 0, coop = 0, per_sm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return;
    if (cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev) != cudaSuccess || !coop) return;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, tv_cg_coop_kernel, kCoopThreads, 0) != cudaSuccess)
      return;
    long long want = (N + kCoopThreads - 1) / kCoopThreads;
    long long cap = (long long)sms * per_sm;
    if (cap > kCoopMaxBlocks) cap = kCoopMaxBlocks;
    coop_blocks = (int)(want < cap ? want : cap);
  }

  // M_gamma z = r.  M annihilates constants (M 1 = 0), so M_gamma 1 = gamma 1
  // and the mean-free part is invariant: z = (mean r / gamma) 1 + y with
  // M_gamma y = r - mean(r) 1 solved by conjugate gradients on mean-free
  // vectors, preconditioned with the diagonal followed by removal of the mean
  // (symmetric positive definite on that subspace).  Without the split the
  // constant mode, of eigenvalue gamma, would dominate the conditioning.
  // rr, pp, ap, zz, dg: work vectors [N]; y accumulates in z.
  qpat_status tv_solve(const double* r, double* z, double* rr, double* pp, double* ap, double* zz, double* dg,
                       const double* ones, int max_iter, double tol) {
    if (coop_blocks > 0) {
      // the whole solve in one cooperative launch
      // cg_stats: [0] iterations, [1] barrier status, [2] arrivals, [3] generation
      const double* rp = r;
      TVGrid tvv = tv;
      GridBar gb{reinterpret_cast<unsigned*>(cg_stats + 2), reinterpret_cast<unsigned*>(cg_stats + 3),
                 cg_stats + 1, kBarrierLimitNs};
      qpat_status e = cuda(cudaMemsetAsync(cg_stats, 0, 4 * sizeof(int), v.stream), "memset");
      if (e != QPAT_OK) return e;
      void* args[] = {&tvv, &rp, &z, &rr, &pp, &ap, &zz, &dg, &coop_part, &max_iter, &tol, &cg_stats, &gb};
      e = cuda(cudaLaunchCooperativeKernel((const void*)tv_cg_coop_kernel, dim3(coop_blocks), dim3(kCoopThreads),
                                           args, 0, v.stream),
               "tv_cg_coop_kernel");
      if (e != QPAT_OK) return e;
      if ((e = cuda(cudaMemcpyAsync(hstats, cg_stats, 2 * sizeof(int), cudaMemcpyDeviceToHost, v.stream),
                    "copy")) != QPAT_OK)
        return e;
      if ((e = cuda(cudaStreamSynchronize(v.stream), "tv_solve sync")) != QPAT_OK) return e;
      if (hstats[1] != 0)
        return (qpat_status)ctx_fail(c, QPAT_ETIMEOUT, "M_gamma solve: a grid-barrier wait gave up");
      tv_iters += *hstats;
      return QPAT_OK;
    }
    if (N <= kOneCtaMax) {
      // small grids: the whole solve in one CTA, without launches per iteration
      tv_cg_kernel<<<1, kCgThreads, 0, v.stream>>>(tv, r, z, rr, pp, ap, zz, dg, max_iter, tol, cg_stats);
      qpat_status e = cuda(cudaMemcpyAsync(hstats, cg_stats, sizeof(int), cudaMemcpyDeviceToHost, v.stream), "copy");
      if (e != QPAT_OK) return e;
      if ((e = cuda(cudaStreamSynchronize(v.stream), "tv_solve sync")) != QPAT_OK) return e;
      tv_iters += *hstats;
      return QPAT_OK;
    }
    tv_apply_kernel<<<blocks_for(N), kT, 0, v.stream>>>(tv, nullptr, dg, 1);
    qpat_status st = cuda(cudaMemsetAsync(z, 0, N * sizeof(double), v.stream), "memset");
    if (st != QPAT_OK) return st;
    st = cuda(cudaMemcpyAsync(rr, r, N * sizeof(double), cudaMemcpyDeviceToDevice, v.stream), "copy");
    if (st != QPAT_OK) return st;
    double m_r, m;
    if ((st = mean(rr, ones, &m_r)) != QPAT_OK) return st;
    add_const_kernel<<<blocks_for(N), kT, 0, v.stream>>>(N, -m_r, rr, 0);
    auto precondition = [&]() -> qpat_status {
      divide_kernel<<<blocks_for(N), kT, 0, v.stream>>>(N, rr, dg, zz);
      qpat_status e = mean(zz, ones, &m);
      add_const_kernel<<<blocks_for(N), kT, 0, v.stream>>>(N, -m, zz, 0);
      return e;
    };
    if ((st = precondition()) != QPAT_OK) return st;
    st = cuda(cudaMemcpyAsync(pp, zz, N * sizeof(double), cudaMemcpyDeviceToDevice, v.stream), "copy");
    if (st != QPAT_OK) return st;
    double rz0;
    if ((st = dot(rr, zz, N, &rz0)) != QPAT_OK) return st;
    // the iterations run on the device with their scalars in sc; the host
    // reads r^T z every kChunk iterations to test convergence
    constexpr int kChunk = 16;
    if ((st = cuda(cudaMemcpyAsync(sc, &rz0, sizeof(double), cudaMemcpyHostToDevice, v.stream), "copy")) != QPAT_OK)
      return st;
    double rz = rz0;
    for (int it = 0; rz0 > 0.0 && it < max_iter && sqrt(fabs(rz) / rz0) > tol;) {
      for (int k = 0; k < kChunk && it < max_iter; ++k, ++it) {
        tv_apply(pp, ap);
        dot_compensated<double>(1, N, pp, ap, partial, sc + 1, v.stream);
        cg_update_kernel<<<blocks_for(N), kT, 0, v.stream>>>(N, sc, pp, ap, z, rr, zz, dg);
        dot_compensated<double>(1, N, zz, ones, partial, sc + 3, v.stream);
        cg_demean_kernel<<<blocks_for(N), kT, 0, v.stream>>>(N, sc, zz);
        dot_compensated<double>(1, N, rr, zz, partial, sc + 2, v.stream);
        cg_direction_kernel<<<blocks_for(N), kT, 0, v.stream>>>(N, sc, zz, pp);
        cg_rotate_kernel<<<1, 32, 0, v.stream>>>(sc);
        ++tv_iters;
      }
      if ((st = cuda(cudaMemcpyAsync(hsc, sc, sizeof(double), cudaMemcpyDeviceToHost, v.stream), "copy")) != QPAT_OK)
        return st;
      if ((st = cuda(cudaStreamSynchronize(v.stream), "tv_solve sync")) != QPAT_OK) return st;
      rz = *hsc;
    }
    // the cap bounds the work; the result is then the last iterate
    add_const_kernel<<<blocks_for(N), kT, 0, v.stream>>>(N, m_r / tv.gamma, z, 0);
    return cuda(cudaGetLastError(), "tv_solve");
  }
};

}  // namespace

extern "C" {

qpat_status qpat_tv_apply(qpat_ctx* c, const double* xbar, double edge, double beta, double gamma, const double* u,
                          double* out) {
  Ld L;
  L.c = c;
  if (!ctx_view(c, &L.v)) return QPAT_EINVAL;
  if (!xbar || !u || !out || !(edge > 0) || !(beta > 0) || gamma < 0)
    return (qpat_status)ctx_fail(c, QPAT_EINVAL, "qpat_tv_apply: bad arguments");
  L.N = L.v.N;
  Work w;
  L.tv = TVGrid{L.v.n0, L.v.n1, L.v.n2, edge, beta, gamma, nullptr, nullptr, nullptr};
  L.tv.wx = w.get<double>((size_t)L.v.n2 * L.v.n1 * (L.v.n0 - 1));
  L.tv.wy = w.get<double>((size_t)L.v.n2 * (L.v.n1 - 1) * L.v.n0);
  L.tv.wz = w.get<double>((size_t)(L.v.n2 > 1 ? L.v.n2 - 1 : 1) * L.v.n1 * L.v.n0);
  if (w.err != cudaSuccess) return L.cuda(w.err, "qpat_tv_apply workspace");
  qpat_status st = L.tv_weights(xbar);
  if (st != QPAT_OK) return st;
  L.tv_apply(u, out);
  st = L.cuda(cudaGetLastError(), "tv_apply_kernel");
  if (st != QPAT_OK) return st;
  return L.cuda(cudaStreamSynchronize(L.v.stream), "qpat_tv_apply sync");
}

// Algorithm 3 with Algorithms 1 and 2 (method 2): unknown Xbar = X / mean(X0)
// per block, [kappa-bar | mu-bar] when kappa is given.  The arithmetic and
// decisions follow oracle/admm.py step by step.
static qpat_status admm_solve(qpat_ctx* c, int nq, const unsigned* illum, const void* data, double* mu,
                              double* kappa, const qpat_ld_params& p, qpat_ld_info* info, double* eps_hist,
                              int* inner_hist) {
  Ld L;
  L.c = c;
  ctx_view(c, &L.v);
  const bool joint = kappa != nullptr;
  const int U = joint ? 2 : 1;
  const long long N = L.v.N, NU = U * N;
  L.N = N;
  L.M = (long long)L.v.nt * L.v.ns;
  L.elt = L.v.prec == QPAT_FP32 ? sizeof(float) : sizeof(double);
  const long long MS = (long long)nq * L.M;
  cudaStream_t s = L.v.stream;
  const long long nfaces = (long long)L.v.n2 * L.v.n1 * (L.v.n0 - 1) + (long long)L.v.n2 * (L.v.n1 - 1) * L.v.n0 +
                           (long long)(L.v.n2 - 1) * L.v.n1 * L.v.n0;
  const long long NF = U * nfaces;
  const int m = p.lbfgs_m;
  Work w;
  double* x = w.get<double>(NU);
  double* xt = w.get<double>(NU);      // trial point of the line search
  double* g = w.get<double>(NU);
  double* gt = w.get<double>(NU);
  double* d = w.get<double>(NU);
  double* q = w.get<double>(NU);
  double* Sv = w.get<double>((size_t)m * NU);
  double* Yv = w.get<double>((size_t)m * NU);
  double* t2 = w.get<double>(N);
  double* t3 = w.get<double>(N);
  double* ones_f = w.get<double>(NF);
  double* W = w.get<double>(NF);
  double* Uw = w.get<double>(NF);
  double* tf = w.get<double>(NF);      // D Xbar - W + Uw (or D Xbar)
  double* aw = w.get<double>(NF);      // |W|
  double* phi = w.get<double>((size_t)nq * N);
  char* Hs = w.get<char>((size_t)MS * L.elt);   // series H_q at the evaluated point
  char* Up = w.get<char>((size_t)MS * L.elt);   // multipliers U_p,q
  char* res = w.get<char>((size_t)MS * L.elt);  // H_q - P_q + U_p,q
  char* hq = w.get<char>((size_t)nq * N * L.elt);
  char* hb = w.get<char>((size_t)nq * N * L.elt);
  L.partial = w.get<double>((size_t)kPartials * 4);
  L.dout = w.get<double>(1);
  double* kap_scaled = joint ? kappa : nullptr;
  TVGrid tvg{L.v.n0, L.v.n1, L.v.n2, p.tv_edge, p.beta, p.gamma, nullptr, nullptr, nullptr};
  if (w.err != cudaSuccess) return L.cuda(w.err, "ADMM workspace");
  qpat_status st;
  // scales mean(X0) per block and the start Xbar^0 = X0 / mean(X0)
  double scale[2];
  {
    double* ones = t2;
    add_const_kernel<<<blocks_for(N), kT, 0, s>>>(N, 1.0, ones, 1);
    double sm, sk = 0.0;
    if ((st = L.dot(mu, ones, N, &sm)) != QPAT_OK) return st;
    if (joint && (st = L.dot(kappa, ones, N, &sk)) != QPAT_OK) return st;
    scale[joint ? 1 : 0] = sm / (double)N;
    if (joint) scale[0] = sk / (double)N;
  }
  double* xk = x;                         // kappa-bar block (joint)
  double* xm = x + (joint ? N : 0);       // mu-bar block
  axpby_kernel<<<blocks_for(N), kT, 0, s>>>(N, 1.0 / scale[joint ? 1 : 0], mu, 0.0, xm);
  if (joint) axpby_kernel<<<blocks_for(N), kT, 0, s>>>(N, 1.0 / scale[0], kappa, 0.0, xk);
  add_const_kernel<<<blocks_for(NF), kT, 0, s>>>(NF, 1.0, ones_f, 1);
  for (double* f : {W, Uw}) (void)cudaMemsetAsync(f, 0, NF * sizeof(double), s);
  if ((st = L.cuda(cudaMemsetAsync(Up, 0, (size_t)MS * L.elt, s), "memset")) != QPAT_OK) return st;

  auto phi_q = [&](int qq) { return phi + (size_t)qq * N; };
  auto hq_q = [&](int qq) -> void* { return hq + (size_t)qq * N * L.elt; };
  auto hb_q = [&](int qq) -> const void* { return hb + (size_t)qq * N * L.elt; };
  auto series = [&](int update) {
    if (L.v.prec == QPAT_FP32)
      admm_series_kernel<float><<<blocks_for(MS), kT, 0, s>>>(MS, (const float*)Hs, (const float*)data, (float*)Up,
                                                              (float*)res, update);
    else
      admm_series_kernel<double><<<blocks_for(MS), kT, 0, s>>>(MS, (const double*)Hs, (const double*)data,
                                                               (double*)Up, (double*)res, update);
  };
  // H_q at xv: coefficients X = scale Xbar, fluences, heatings, one batched H_a
  auto forward = [&](const double* xv) -> qpat_status {
    axpby_kernel<<<blocks_for(N), kT, 0, s>>>(N, scale[joint ? 1 : 0], xv + (joint ? N : 0), 0.0, mu);
    if (joint) {
      axpby_kernel<<<blocks_for(N), kT, 0, s>>>(N, scale[0], xv, 0.0, kap_scaled);
      qpat_status e = qpat_set_kappa(c, kap_scaled);
      if (e != QPAT_OK) return e;
    }
    {
      PhaseTimer pt(&L.sec[1], s);
      for (int qq = 0; qq < nq; ++qq) {
        qpat_status e = (qpat_status)optics_forward(c, mu, illum[qq], phi_q(qq), hq_q(qq));
        if (e != QPAT_OK) return e;
      }
    }
    PhaseTimer pt(&L.sec[0], s);
    L.products += nq;
    return qpat_acoustic_forward(c, nq, hq, Hs);
  };
  // F_A at xv (H_q current for xv) for W, Uw and Up (eq. FAm); leaves res and tf
  auto value = [&](const double* xv, const double* Wv, double* out) -> qpat_status {
    series(0);
    double data2, tv2, l1 = 0.0;
    qpat_status e = L.dot_data(res, res, MS, &data2);
    if (e != QPAT_OK) return e;
    for (int u = 0; u < U; ++u)
      admm_dx_kernel<<<blocks_for(nfaces), kT, 0, s>>>(tvg, xv + u * N, Wv ? Wv + u * nfaces : nullptr,
                                                       Uw + u * nfaces, tf + u * nfaces);
    if ((e = L.dot(tf, tf, NF, &tv2)) != QPAT_OK) return e;
    if (Wv && (e = L.dot(aw, ones_f, NF, &l1)) != QPAT_OK) return e;
    *out = p.rho * (0.5 * tv2 + p.nu * l1) + 0.5 * data2;
    return QPAT_OK;
  };
  // grad F_A into gv (res and tf as value() left them)
  auto gradient = [&](double* gv) -> qpat_status {
    qpat_status e;
    {
      PhaseTimer pt(&L.sec[0], s);
      if ((e = qpat_acoustic_adjoint(c, nq, res, hb)) != QPAT_OK) return e;
    }
    L.products += nq;
    PhaseTimer pt(&L.sec[1], s);
    for (int qq = 0; qq < nq; ++qq) {
      if ((e = (qpat_status)optics_vjp2(c, mu, phi_q(qq), hb_q(qq), illum[qq], t2, joint ? t3 : nullptr)) != QPAT_OK)
        return e;
      axpby_kernel<<<blocks_for(N), kT, 0, s>>>(N, scale[joint ? 1 : 0], t2, qq > 0 ? 1.0 : 0.0,
                                                gv + (joint ? N : 0));
      if (joint) axpby_kernel<<<blocks_for(N), kT, 0, s>>>(N, scale[0], t3, qq > 0 ? 1.0 : 0.0, gv);
    }
    for (int u = 0; u < U; ++u) admm_dt_kernel<<<blocks_for(N), kT, 0, s>>>(tvg, tf + u * nfaces, p.rho, gv + u * N, 1);
    return L.cuda(cudaGetLastError(), "ADMM gradient");
  };
  auto norm = [&](const double* v, double* out) -> qpat_status {
    qpat_status e = L.dot(v, v, NU, out);
    *out = sqrt(*out);
    return e;
  };
  auto axpy = [&](double a, const double* xv, double* yv) {
    axpby_kernel<<<blocks_for(NU), kT, 0, s>>>(NU, a, xv, 1.0, yv);
  };
  auto copy = [&](double* dst, const double* src) {
    return L.cuda(cudaMemcpyAsync(dst, src, NU * sizeof(double), cudaMemcpyDeviceToDevice, s), "copy");
  };
  auto eps_of_H = [&](double* out) -> qpat_status {   // 1/2 sum_q ||H_q - P_q||^2
    if (L.v.prec == QPAT_FP32)
      resid_kernel<float><<<blocks_for(MS), kT, 0, s>>>(MS, (const float*)Hs, (const float*)data, (float*)res);
    else
      resid_kernel<double><<<blocks_for(MS), kT, 0, s>>>(MS, (const double*)Hs, (const double*)data, (double*)res);
    double e2;
    qpat_status e = L.dot_data(res, res, MS, &e2);
    *out = 0.5 * e2;
    return e;
  };

  // start: eps^0 and ||grad F_A|| at W = 0, zero multipliers
  std::vector<double> eps;
  double e0, f, gnorm;
  if ((st = forward(x)) != QPAT_OK) return st;
  if ((st = eps_of_H(&e0)) != QPAT_OK) return st;
  eps.push_back(e0);
  if ((st = value(x, W, &f)) != QPAT_OK) return st;
  if ((st = gradient(g)) != QPAT_OK) return st;
  if ((st = norm(g, &gnorm)) != QPAT_OK) return st;
  int k = 0, inner_total = 0;
  std::vector<double> rho_pair;
  while (k < p.k_max && gnorm > p.tol_out) {
    // W^(k+1) = shrink(D Xbar^k + U_w^k, nu)
    for (int u = 0; u < U; ++u)
      admm_dx_kernel<<<blocks_for(nfaces), kT, 0, s>>>(tvg, x + u * N, nullptr, nullptr, tf + u * nfaces);
    axpby_kernel<<<blocks_for(NF), kT, 0, s>>>(NF, 1.0, Uw, 1.0, tf);
    shrink_kernel<<<blocks_for(NF), kT, 0, s>>>(NF, tf, p.nu, W, aw);
    // Xbar^(k+1): at most j_max L-BFGS iterations on F_A(., W^(k+1)) from Xbar^k
    if ((st = forward(x)) != QPAT_OK) return st;
    if ((st = value(x, W, &f)) != QPAT_OK) return st;
    if ((st = gradient(g)) != QPAT_OK) return st;
    int npair = 0, it = 0;
    rho_pair.assign(m, 0.0);
    for (;;) {
      double gn;
      if ((st = norm(g, &gn)) != QPAT_OK) return st;
      if (!(it < p.j_max && gn > p.tol_in)) break;
      // Algorithm 1 over the npair newest pairs (slot j holds pair j, oldest first)
      if ((st = copy(q, g)) != QPAT_OK) return st;
      std::vector<double> alpha(npair);
      for (int i = npair - 1; i >= 0; --i) {
        double sq;
        if ((st = L.dot(Sv + i * NU, q, NU, &sq)) != QPAT_OK) return st;
        alpha[i] = rho_pair[i] * sq;
        axpy(-alpha[i], Yv + i * NU, q);
      }
      double h0 = 1.0;
      if (npair > 0) {
        double sy, yy;
        if ((st = L.dot(Sv + (npair - 1) * NU, Yv + (npair - 1) * NU, NU, &sy)) != QPAT_OK) return st;
        if ((st = L.dot(Yv + (npair - 1) * NU, Yv + (npair - 1) * NU, NU, &yy)) != QPAT_OK) return st;
        h0 = sy / yy;
      }
      axpby_kernel<<<blocks_for(NU), kT, 0, s>>>(NU, -h0, q, 0.0, d);   // d = -r with r = h0 q
      for (int i = 0; i < npair; ++i) {
        double yr;
        if ((st = L.dot(Yv + i * NU, d, NU, &yr)) != QPAT_OK) return st;   // y^T d = -y^T r
        const double beta = rho_pair[i] * (-yr);
        axpy(-(alpha[i] - beta), Sv + i * NU, d);                          // r += s (alpha - beta)
      }
      project_kernel<<<blocks_for(NU), kT, 0, s>>>(NU, x, p.lower, p.upper, d);
      double gd;
      if ((st = L.dot(g, d, NU, &gd)) != QPAT_OK) return st;
      if (gd >= 0.0) {
        npair = 0;
        axpby_kernel<<<blocks_for(NU), kT, 0, s>>>(NU, -1.0, g, 0.0, d);
        project_kernel<<<blocks_for(NU), kT, 0, s>>>(NU, x, p.lower, p.upper, d);
        if ((st = L.dot(g, d, NU, &gd)) != QPAT_OK) return st;
        if (gd >= 0.0) break;
      }
      // Algorithm 2: alpha = 1, tau, tau^2, ... until both Wolfe conditions hold
      double a = 1.0, a_ok = -1.0, f_ok = 0.0, a_acc = -1.0, f_acc = 0.0;
      for (int tr = 0; tr < p.ls_max; ++tr) {
        if ((st = copy(xt, x)) != QPAT_OK) return st;
        axpy(a, d, xt);
        double ft;
        if ((st = forward(xt)) != QPAT_OK) return st;
        if ((st = value(xt, W, &ft)) != QPAT_OK) return st;
        if ((st = gradient(gt)) != QPAT_OK) return st;
        if (ft <= f + p.c1 * a * gd) {
          double gtd;
          if ((st = L.dot(gt, d, NU, &gtd)) != QPAT_OK) return st;
          if (gtd >= p.c2 * gd) {
            a_acc = a;
            f_acc = ft;
            break;
          }
          if (a_ok < 0.0) {
            a_ok = a;
            f_ok = ft;
            if ((st = copy(q, gt)) != QPAT_OK) return st;   // keep its gradient
          }
        }
        a *= p.tau;
      }
      if (a_acc < 0.0) {
        if (a_ok < 0.0) break;
        a_acc = a_ok;
        f_acc = f_ok;
        if ((st = copy(gt, q)) != QPAT_OK) return st;
      }
      // s = a d, y = g_new - g; keep the pair when y^T s > 0 (at most m, oldest dropped)
      if ((st = copy(xt, gt)) != QPAT_OK) return st;         // xt <- g_new
      axpy(-1.0, g, xt);                                      // xt <- y
      double ys;
      if ((st = L.dot(xt, d, NU, &ys)) != QPAT_OK) return st;
      ys *= a_acc;
      if (ys > 0.0) {
        if (npair == m) {
          for (int i = 1; i < m; ++i) {
            if ((st = copy(Sv + (i - 1) * NU, Sv + i * NU)) != QPAT_OK) return st;
            if ((st = copy(Yv + (i - 1) * NU, Yv + i * NU)) != QPAT_OK) return st;
            rho_pair[i - 1] = rho_pair[i];
          }
          --npair;
        }
        axpby_kernel<<<blocks_for(NU), kT, 0, s>>>(NU, a_acc, d, 0.0, Sv + npair * NU);
        if ((st = copy(Yv + npair * NU, xt)) != QPAT_OK) return st;
        rho_pair[npair] = 1.0 / ys;
        ++npair;
      }
      axpy(a_acc, d, x);
      if ((st = copy(g, gt)) != QPAT_OK) return st;
      f = f_acc;
      ++it;
    }
    if (inner_hist) inner_hist[k] = it;
    inner_total += it;
    // multipliers: U_w += D Xbar - W, U_p,q += H_q - P_q (H at Xbar^(k+1))
    if ((st = forward(x)) != QPAT_OK) return st;
    double ek;
    if ((st = eps_of_H(&ek)) != QPAT_OK) return st;
    eps.push_back(ek);
    for (int u = 0; u < U; ++u)
      admm_dx_kernel<<<blocks_for(nfaces), kT, 0, s>>>(tvg, x + u * N, W + u * nfaces, Uw + u * nfaces,
                                                       tf + u * nfaces);
    axpby_kernel<<<blocks_for(NF), kT, 0, s>>>(NF, 1.0, tf, 0.0, Uw);   // (D Xbar - W + Uw) = the new Uw
    series(1);
    if ((st = value(x, W, &f)) != QPAT_OK) return st;
    if ((st = gradient(g)) != QPAT_OK) return st;
    if ((st = norm(g, &gnorm)) != QPAT_OK) return st;
    ++k;
  }
  // X = scale Xbar
  axpby_kernel<<<blocks_for(N), kT, 0, s>>>(N, scale[joint ? 1 : 0], xm, 0.0, mu);
  if (joint) {
    axpby_kernel<<<blocks_for(N), kT, 0, s>>>(N, scale[0], xk, 0.0, kappa);
    if ((st = qpat_set_kappa(c, kappa)) != QPAT_OK) return st;
  }
  if ((st = L.cuda(cudaStreamSynchronize(s), "ADMM sync")) != QPAT_OK) return st;
  if (eps_hist)
    for (size_t j = 0; j < eps.size(); ++j) eps_hist[j] = eps[j];
  if (info) {
    info->outer = k;
    info->inner_total = inner_total;
    info->sub_total = 0;
    info->tv_iters = 0;
    info->products = L.products;
    info->eps_first = eps.front();
    info->eps_last = eps.back();
    for (int j = 0; j < 3; ++j) info->seconds[j] = L.sec[j];
  }
  return QPAT_OK;
}

qpat_status qpat_ld_solve(qpat_ctx* c, int nq, const unsigned* illum, const void* data, double* mu,
                          double* kappa, const qpat_ld_params* prm_in, qpat_ld_info* info, double* eps_hist,
                          int* inner_hist) {
  Ld L;
  L.c = c;
  if (!ctx_view(c, &L.v)) return QPAT_EINVAL;
  if (nq < 1 || !illum || !data || !mu) return (qpat_status)ctx_fail(c, QPAT_EINVAL, "qpat_ld_solve: bad arguments");
  if (nq > L.v.maxb)
    return (qpat_status)ctx_fail(c, QPAT_EINVAL, "qpat_ld_solve: the context's max_batch must be >= nq");
  const unsigned all = (1u << (2 * L.v.dim)) - 1;
  for (int q = 0; q < nq; ++q)
    if (illum[q] == 0 || (illum[q] & ~all))
      return (qpat_status)ctx_fail(c, QPAT_EINVAL, "qpat_ld_solve: illumination mask must select sides 0 .. 2d-1");
  qpat_ld_params p{};
  if (prm_in) p = *prm_in;
  if (p.k_max <= 0) p.k_max = 10;
  if (p.i_max <= 0) p.i_max = 30;
  if (p.i_m <= 0) p.i_m = 5;
  if (p.tol_in < 0) p.tol_in = 0;
  if (p.tol_out < 0) p.tol_out = 1e-3;
  if (p.gamma <= 0) p.gamma = 1e-6;
  if (p.beta <= 0) p.beta = 2e-5;
  if (p.tv_edge <= 0) p.tv_edge = L.v.dim == 3 ? (L.v.dx * 1e3) * (L.v.dx * 1e3) : L.v.dx * 1e3;
  if (p.tv_max_iter <= 0) p.tv_max_iter = 20000;
  if (p.tv_tol <= 0) p.tv_tol = 1e-12;
  if (p.method < 0 || p.method > 2)
    return (qpat_status)ctx_fail(c, QPAT_EINVAL,
                                 "qpat_ld_solve: method must be 0 (LD), 1 (PD-IPM) or 2 (ADMM with L-BFGS)");
  if (p.kp_max <= 0) p.kp_max = 20;
  if (p.method == 2) {
    if (prm_in && prm_in->tol_out < 0) p.tol_out = 1e-2;
    if (p.lbfgs_m <= 0) p.lbfgs_m = 5;
    if (p.j_max <= 0) p.j_max = 10;
    if (p.ls_max <= 0) p.ls_max = 20;
    if (p.c1 <= 0) p.c1 = 1e-4;
    if (p.c2 <= 0) p.c2 = 0.9;
    if (p.tau <= 0) p.tau = 0.25;
    if (p.rho <= 0) p.rho = 1.0;
    if (p.nu <= 0) p.nu = 1e-3;
    if (!(p.upper > p.lower)) {
      p.lower = 1e-3;
      p.upper = 1e3;
    }
    return admm_solve(c, nq, illum, data, mu, kappa, p, info, eps_hist, inner_hist);
  }

  // unknowns: [kappa-bar | mu-bar] (joint) or mu-bar, each block N cells
  const bool joint = kappa != nullptr;
  const int U = joint ? 2 : 1;
  const long long N = L.v.N, NU = U * N;
  L.N = N;
  L.M = (long long)L.v.nt * L.v.ns;
  L.elt = L.v.prec == QPAT_FP32 ? sizeof(float) : sizeof(double);
  cudaStream_t s = L.v.stream;
  Work w;
  double* mu0 = w.get<double>(N);
  double* kap0 = joint ? w.get<double>(N) : nullptr;
  double* xbar = w.get<double>(NU);
  double* phi = w.get<double>((size_t)nq * N);   // fluence of every illumination at the linearisation point
  double* g = w.get<double>(NU);
  double* r = w.get<double>(NU);
  double* z = w.get<double>(NU);
  double* d = w.get<double>(NU);
  double* x = w.get<double>(NU);
  double* hd = w.get<double>(NU);
  double* t1 = w.get<double>(N);
  double* t2 = w.get<double>(N);
  double* t3 = w.get<double>(N);
  double* t4 = w.get<double>(N);
  double* t5 = w.get<double>(NU);
  double* c_rr = w.get<double>(N);
  double* c_pp = w.get<double>(N);
  double* c_ap = w.get<double>(N);
  double* c_zz = w.get<double>(N);
  double* c_dg = w.get<double>(N);
  double* ones = w.get<double>(N);
  char* res = w.get<char>((size_t)nq * L.M * L.elt);   // residual series H_q - P_q
  char* jv = w.get<char>((size_t)nq * L.M * L.elt);    // J_q of the current direction
  char* hq = w.get<char>((size_t)nq * N * L.elt);      // heating (or its derivative) per q
  char* hb = w.get<char>((size_t)nq * N * L.elt);      // H_a^* of a series per q
  L.partial = w.get<double>((size_t)kPartials * 4);
  L.dout = w.get<double>(1);
  L.sc = w.get<double>(8);
  L.cg_stats = w.get<int>(4);
  L.coop_part = w.get<double>(2 * (size_t)kCoopMaxBlocks);
  const long long nfaces = (long long)L.v.n2 * L.v.n1 * (L.v.n0 - 1) + (long long)L.v.n2 * (L.v.n1 - 1) * L.v.n0 +
                           (long long)(L.v.n2 - 1) * L.v.n1 * L.v.n0;
  TVGrid tvb[2];                                       // TV operator of each unknown block
  for (int u = 0; u < U; ++u) {
    tvb[u] = TVGrid{L.v.n0, L.v.n1, L.v.n2, p.tv_edge, p.beta, p.gamma, nullptr, nullptr, nullptr};
    // the three face sets of a block back to back (face order of face_cells)
    double* wall = w.get<double>((size_t)nfaces + 1);
    tvb[u].wx = wall;
    tvb[u].wy = wall + (size_t)L.v.n2 * L.v.n1 * (L.v.n0 - 1);
    tvb[u].wz = tvb[u].wy + (size_t)L.v.n2 * (L.v.n1 - 1) * L.v.n0;
  }
  // primal-dual state (Algorithm 6): the update d, and chi, dchi per face of each block
  const bool pd = p.method == 1;
  double* dvec = pd ? w.get<double>(NU) : nullptr;
  double* chi = pd ? w.get<double>((size_t)U * nfaces + 1) : nullptr;
  double* dchi = pd ? w.get<double>((size_t)U * nfaces + 1) : nullptr;
  double* phipart = pd ? w.get<double>(1024) : nullptr;
  double* phimin = pd ? w.get<double>(1) : nullptr;
  if (w.err != cudaSuccess) return L.cuda(w.err, "qpat_ld_solve workspace");
  struct PinnedScalars {
    double* p = nullptr;
    ~PinnedScalars() {
      if (p) cudaFreeHost(p);
    }
  } pinned;
  qpat_status st;
  if ((st = L.cuda(cudaMallocHost(&pinned.p, 8 * sizeof(double)), "pinned scalars")) != QPAT_OK) return st;
  L.hsc = pinned.p;
  L.hstats = reinterpret_cast<int*>(pinned.p + 4);
  L.setup_coop();
  if ((st = L.cuda(cudaMemcpyAsync(mu0, mu, N * sizeof(double), cudaMemcpyDeviceToDevice, s), "copy")) != QPAT_OK)
    return st;
  if (joint &&
      (st = L.cuda(cudaMemcpyAsync(kap0, kappa, N * sizeof(double), cudaMemcpyDeviceToDevice, s), "copy")) != QPAT_OK)
    return st;
  if ((st = L.cuda(cudaMemsetAsync(xbar, 0, NU * sizeof(double), s), "memset")) != QPAT_OK) return st;
  add_const_kernel<<<blocks_for(N), kT, 0, s>>>(N, 1.0, ones, 1);

  auto phi_q = [&](int q) { return phi + (size_t)q * N; };
  auto hq_q = [&](int q) -> void* { return hq + (size_t)q * N * L.elt; };
  auto hb_q = [&](int q) -> const void* { return hb + (size_t)q * N * L.elt; };
  auto blk_mu = [&](double* v) { return v + (joint ? N : 0); };   // mu-bar block
  auto blk_k = [&](double* v) { return v; };                        // kappa-bar block (joint)

  // out = sum_q dX/dXbar o J_o,q^*(hbar_q), block by block (eq. gr / apj);
  // the acoustic halves of all illuminations have run as one batch
  auto optical_adjoint_sum = [&](double* out) -> qpat_status {
    PhaseTimer pt(&L.sec[1], s);
    for (int q = 0; q < nq; ++q) {
      qpat_status e = (qpat_status)optics_vjp2(c, mu, phi_q(q), hb_q(q), illum[q], t2, joint ? t3 : nullptr);
      if (e != QPAT_OK) return e;
      hadamard_kernel<<<blocks_for(N), kT, 0, s>>>(N, mu, t2, blk_mu(out), q > 0);
      if (joint) hadamard_kernel<<<blocks_for(N), kT, 0, s>>>(N, kappa, t3, blk_k(out), q > 0);
    }
    return L.cuda(cudaGetLastError(), "optical adjoint");
  };

  // H d = sum_q S J_q^* J_q S d into hd (eq. apj), S = dX/dXbar
  auto gn_product = [&](double* dd) -> qpat_status {
    hadamard_kernel<<<blocks_for(N), kT, 0, s>>>(N, mu, blk_mu(dd), t1, 0);
    if (joint) hadamard_kernel<<<blocks_for(N), kT, 0, s>>>(N, kappa, blk_k(dd), t4, 0);
    {
      PhaseTimer pt(&L.sec[1], s);
      for (int q = 0; q < nq; ++q) {
        qpat_status e = (qpat_status)optics_jvp2(c, mu, phi_q(q), t1, joint ? t4 : nullptr, illum[q], hq_q(q));
        if (e != QPAT_OK) return e;
      }
    }
    qpat_status e;
    {
      PhaseTimer pt(&L.sec[0], s);
      if ((e = qpat_acoustic_forward(c, nq, hq, jv)) != QPAT_OK) return e;
      if ((e = qpat_acoustic_adjoint(c, nq, jv, hb)) != QPAT_OK) return e;
    }
    L.products += 2 * nq;
    return optical_adjoint_sum(hd);
  };

  // z = M_gamma^-1 r, block by block (D is block diagonal, eq. dd)
  auto precond = [&](double* rv, double* zv) -> qpat_status {
    PhaseTimer pt(&L.sec[2], s);
    for (int u = 0; u < U; ++u) {
      L.tv = tvb[u];
      qpat_status e = L.tv_solve(rv + u * N, zv + u * N, c_rr, c_pp, c_ap, c_zz, c_dg, ones, p.tv_max_iter, p.tv_tol);
      if (e != QPAT_OK) return e;
    }
    return QPAT_OK;
  };
  auto axpby_u = [&](double a, const double* xv, double b, double* yv) {
    axpby_kernel<<<blocks_for(NU), kT, 0, s>>>(NU, a, xv, b, yv);
  };

  // Algorithm 4: PCG on H x = -gv with the preconditioner of tvb (weights set
  // by the caller), from x = 0; iterations and the last r^T z to the caller
  auto run_pcg = [&](const double* gv, int* iters, double* rz_last) -> qpat_status {
    qpat_status e;
    if ((e = L.cuda(cudaMemsetAsync(x, 0, NU * sizeof(double), s), "memset")) != QPAT_OK) return e;
    if ((e = L.cuda(cudaMemsetAsync(r, 0, NU * sizeof(double), s), "memset")) != QPAT_OK) return e;
    axpby_u(-1.0, gv, 1.0, r);
    if ((e = precond(r, z)) != QPAT_OK) return e;
    if ((e = L.cuda(cudaMemcpyAsync(d, z, NU * sizeof(double), cudaMemcpyDeviceToDevice, s), "copy")) != QPAT_OK)
      return e;
    std::vector<double> rz(1);
    if ((e = L.dot(r, z, NU, &rz[0])) != QPAT_OK) return e;
    int i = 0;
    while (i < p.i_max && rz[i] != 0.0 && (i < p.i_m || 1.0 - rz[i] / rz[i - p.i_m] > p.tol_in)) {
      if ((e = gn_product(d)) != QPAT_OK) return e;
      double dhd;
      if ((e = L.dot(d, hd, NU, &dhd)) != QPAT_OK) return e;
      const double alpha = rz[i] / dhd;
      axpby_u(alpha, d, 1.0, x);
      axpby_u(-alpha, hd, 1.0, r);
      if ((e = precond(r, z)) != QPAT_OK) return e;
      double rzn;
      if ((e = L.dot(r, z, NU, &rzn)) != QPAT_OK) return e;
      rz.push_back(rzn);
      axpby_u(1.0, z, rz[i + 1] / rz[i], d);
      ++i;
    }
    *iters = i;
    *rz_last = rz.back();
    return QPAT_OK;
  };

  std::vector<double> eps;
  int inner_total = 0, sub_total = 0;
  int k = 0;
  for (;;) {
    // linearisation point X^k = X0 exp(Xbar^k): coefficients, residuals, eps^k, fluences
    exp_scale_kernel<<<blocks_for(N), kT, 0, s>>>(N, mu0, blk_mu(xbar), mu);
    if (joint) {
      exp_scale_kernel<<<blocks_for(N), kT, 0, s>>>(N, kap0, blk_k(xbar), kappa);
      if ((st = qpat_set_kappa(c, kappa)) != QPAT_OK) return st;
    }
    {
      PhaseTimer pt(&L.sec[1], s);
      for (int q = 0; q < nq; ++q)
        if ((st = (qpat_status)optics_forward(c, mu, illum[q], phi_q(q), hq_q(q))) != QPAT_OK) return st;
    }
    {
      PhaseTimer pt(&L.sec[0], s);
      if ((st = qpat_acoustic_forward(c, nq, hq, res)) != QPAT_OK) return st;
    }
    L.products += nq;
    const long long MS = (long long)nq * L.M;
    if (L.v.prec == QPAT_FP32)
      resid_kernel<float><<<blocks_for(MS), kT, 0, s>>>(MS, (const float*)res, (const float*)data, (float*)res);
    else
      resid_kernel<double><<<blocks_for(MS), kT, 0, s>>>(MS, (const double*)res, (const double*)data, (double*)res);
    double e2;
    if ((st = L.dot_data(res, res, MS, &e2)) != QPAT_OK) return st;
    eps.push_back(0.5 * e2);
    if (k > 0 && !(1.0 - eps[k] / eps[k - 1] > p.tol_out)) break;
    if (k >= p.k_max) break;

    // gradient (eq. gr)
    {
      PhaseTimer pt(&L.sec[0], s);
      if ((st = qpat_acoustic_adjoint(c, nq, res, hb)) != QPAT_OK) return st;
    }
    L.products += nq;
    if ((st = optical_adjoint_sum(g)) != QPAT_OK) return st;
    if (!pd) {
      // M_gamma^k frozen at Xbar^k (lagged diffusivity), one per block
      for (int u = 0; u < U; ++u) {
        L.tv = tvb[u];
        if ((st = L.tv_weights(xbar + u * N)) != QPAT_OK) return st;
      }
      int i;
      double rz_last;
      if ((st = run_pcg(g, &i, &rz_last)) != QPAT_OK) return st;   // H x = -g
      if (inner_hist) inner_hist[k] = i;
      inner_total += i;
      axpby_u(1.0, x, 1.0, xbar);   // Xbar^{k+1} = Xbar^k + d^k (alpha^k = 1)
    } else {
      // Algorithm 6: sub-subproblems k' on the update d with the dual chi
      if ((st = L.cuda(cudaMemsetAsync(dvec, 0, NU * sizeof(double), s), "memset")) != QPAT_OK) return st;
      if ((st = L.cuda(cudaMemsetAsync(chi, 0, (size_t)U * nfaces * sizeof(double), s), "memset")) != QPAT_OK)
        return st;
      int its = 0;
      double r_prev = 0.0;
      for (int kp = 0; kp < p.kp_max; ++kp) {
        for (int u = 0; u < U; ++u) {
          pd_weights_kernel<<<blocks_for(nfaces), kT, 0, s>>>(tvb[u], dvec + u * N, chi + u * nfaces);
          if ((st = L.cuda(cudaGetLastError(), "pd_weights_kernel")) != QPAT_OK) return st;
        }
        // grad eps~_k' = grad eps + H d_k' (eq. du with lambda = 0); H d = 0 at d = 0
        if (kp == 0) {
          if ((st = L.cuda(cudaMemcpyAsync(t5, g, NU * sizeof(double), cudaMemcpyDeviceToDevice, s), "copy")) !=
              QPAT_OK)
            return st;
        } else {
          if ((st = gn_product(dvec)) != QPAT_OK) return st;
          if ((st = L.cuda(cudaMemcpyAsync(t5, g, NU * sizeof(double), cudaMemcpyDeviceToDevice, s), "copy")) !=
              QPAT_OK)
            return st;
          axpby_u(1.0, hd, 1.0, t5);
        }
        int i;
        double r_star;
        if ((st = run_pcg(t5, &i, &r_star)) != QPAT_OK) return st;   // eq. pre1: H dd = -grad eps~
        its += i;
        // dual step (eq. dw) with the step length rule, then d += dd (alpha_k' = 1)
        for (int u = 0; u < U; ++u) {
          const int nb = 1024;
          pd_dual_kernel<<<nb, kT, 0, s>>>(tvb[u], dvec + u * N, x + u * N, chi + u * nfaces, dchi + u * nfaces,
                                           phipart);
          min_final_kernel<<<1, 32, 0, s>>>(phipart, nb, phimin);
          double phi;
          if ((st = L.cuda(cudaMemcpyAsync(L.hsc + 2, phimin, sizeof(double), cudaMemcpyDeviceToHost, s), "copy")) !=
              QPAT_OK)
            return st;
          if ((st = L.cuda(cudaStreamSynchronize(s), "dual step sync")) != QPAT_OK) return st;
          phi = L.hsc[2];
          pd_chi_update_kernel<<<blocks_for(nfaces), kT, 0, s>>>(nfaces, phi < 1.0 ? phi : 1.0, dchi + u * nfaces,
                                                                 chi + u * nfaces);
        }
        axpby_u(1.0, x, 1.0, dvec);
        ++sub_total;
        if (kp > 0 && !(1.0 - r_star / r_prev > p.tol_med)) break;
        r_prev = r_star;
      }
      if (inner_hist) inner_hist[k] = its;
      inner_total += its;
      axpby_u(1.0, dvec, 1.0, xbar);   // Xbar^{k+1} = Xbar_0^k + d (alpha^k = 1)
    }
    ++k;
  }
  if ((st = L.cuda(cudaStreamSynchronize(s), "qpat_ld_solve sync")) != QPAT_OK) return st;
  if (eps_hist)
    for (size_t j = 0; j < eps.size(); ++j) eps_hist[j] = eps[j];
  if (info) {
    info->outer = k;
    info->inner_total = inner_total;
    info->sub_total = sub_total;
    info->tv_iters = L.tv_iters;
    info->products = L.products;
    info->eps_first = eps.front();
    info->eps_last = eps.back();
    for (int j = 0; j < 3; ++j) info->seconds[j] = L.sec[j];
  }
  return QPAT_OK;
}

}  // extern "C"
