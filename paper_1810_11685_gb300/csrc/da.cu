// Diffusion-approximation optical solve (Section 2.1, eq. DA) in FP64.
//
// Cell-centred finite volumes on the interior grid (the optical grid is the
// acoustic interior): an interior face between cells a, b carries
// kappa_f (phi_a - phi_b) with the harmonic mean kappa_f (2D, the face
// length h cancels the 1/h of the gradient); the Robin condition
// phi + kappa/(2 gamma) dphi/dn = I/gamma, eliminated through the half-cell
// gradient, adds 2 gamma kappa h / (gamma h + kappa) to the diagonal and
// 2 kappa I h / (gamma h + kappa) to the right-hand side per boundary face;
// absorption adds mu h^2.  The matrix is symmetric positive definite and is
// solved by Jacobi-preconditioned conjugate gradients with FP64 dot products
// (deterministic two-level reductions), batched over problems.
#include <algorithm>

#include "qpat_internal.h"

namespace qpat {

constexpr int kThreads = 256;

__device__ __forceinline__ double harmonic(double a, double b) { return 2.0 * a * b / (a + b); }

// Face, Robin and source coefficients of the finite-volume system for a
// grid of n0 x n1 x n2 cells (n2 = 1 in 2D): an interior face carries
// kappa_f h^(d-2), a boundary face adds 2 gamma kappa h^(d-1)/(gamma h + kappa)
// to the diagonal and 2 kappa I h^(d-1)/(gamma h + kappa) to the right-hand side.
__global__ void da_setup_kernel(int n0, int n1, int n2, int dim, double h, double gam, const double* kappa,
                                double* diag0, double* cxf, double* cyf, double* czf, double* bside) {
  const long long N = (long long)n0 * n1 * n2;
  const double hf = (dim == 3) ? h : 1.0;           // h^(d-2)
  const double hb = (dim == 3) ? h * h : h;         // h^(d-1)
  const long long sy = n0, sz = (long long)n0 * n1;
  for (long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x; g < N; g += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(g % n0), j = (int)((g / n0) % n1), k = (int)(g / sz);
    const double kc = kappa[g];
    double d = 0.0;
    if (i > 0) d += harmonic(kc, kappa[g - 1]) * hf;
    if (i < n0 - 1) d += harmonic(kc, kappa[g + 1]) * hf;
    if (j > 0) d += harmonic(kc, kappa[g - sy]) * hf;
    if (j < n1 - 1) d += harmonic(kc, kappa[g + sy]) * hf;
    if (dim == 3) {
      if (k > 0) d += harmonic(kc, kappa[g - sz]) * hf;
      if (k < n2 - 1) d += harmonic(kc, kappa[g + sz]) * hf;
    }
    const double robin = 2.0 * gam * kc * hb / (gam * h + kc);
    const double src = 2.0 * kc * hb / (gam * h + kc);
    const bool on[6] = {i == 0, i == n0 - 1, j == 0, j == n1 - 1, dim == 3 && k == 0, dim == 3 && k == n2 - 1};
    for (int s = 0; s < 2 * dim; ++s) {
      if (on[s]) d += robin;
      bside[(long long)s * N + g] = on[s] ? src : 0.0;
    }
    diag0[g] = d;
    cxf[g] = (i < n0 - 1) ? harmonic(kc, kappa[g + 1]) * hf : 0.0;
    cyf[g] = (j < n1 - 1) ? harmonic(kc, kappa[g + sy]) * hf : 0.0;
    if (dim == 3) czf[g] = (k < n2 - 1) ? harmonic(kc, kappa[g + sz]) * hf : 0.0;
  }
}

cudaError_t da_setup(DAArgs& a, double* d_diag0, double* d_cxf, double* d_cyf, double* d_czf, double* d_bside,
                     const double* d_kappa, cudaStream_t s) {
  da_setup_kernel<<<256, kThreads, 0, s>>>(a.n0, a.n1, a.n2, a.dim, a.h, a.gamma, d_kappa, d_diag0, d_cxf, d_cyf,
                                           d_czf, d_bside);
  a.diag0 = d_diag0;
  a.cxf = d_cxf;
  a.cyf = d_cyf;
  a.czf = d_czf;
  a.bside = d_bside;
  return cudaGetLastError();
}

__global__ void rhs_sides_kernel(DAArgs a, unsigned mask, double* rhs) {
  const int b = blockIdx.y;
  for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < a.N; g += gridDim.x * blockDim.x) {
    double v = 0.0;
    for (int s = 0; s < 2 * a.dim; ++s)
      if ((mask >> s) & 1u) v += a.bside[(long long)s * a.N + g];
    rhs[(long long)b * a.N + g] = v;
  }
}

cudaError_t da_rhs_from_sides(const DAArgs& a, unsigned mask, int batch, double* rhs, cudaStream_t s) {
  rhs_sides_kernel<<<dim3(64, batch), kThreads, 0, s>>>(a, mask, rhs);
  return cudaGetLastError();
}

__device__ __forceinline__ double apply_A(const DAArgs& a, const double* mu, const double* x, int g, double hd) {
  const int sy = a.n0, sz = a.n0 * a.n1;
  const int i = g % a.n0, j = (g / a.n0) % a.n1, k = g / sz;
  double y = (a.diag0[g] + mu[g] * hd) * x[g];
  if (i > 0) y -= a.cxf[g - 1] * x[g - 1];
  if (i < a.n0 - 1) y -= a.cxf[g] * x[g + 1];
  if (j > 0) y -= a.cyf[g - sy] * x[g - sy];
  if (j < a.n1 - 1) y -= a.cyf[g] * x[g + sy];
  if (a.dim == 3) {
    if (k > 0) y -= a.czf[g - sz] * x[g - sz];
    if (k < a.n2 - 1) y -= a.czf[g] * x[g + sz];
  }
  return y;
}

// Block-wide sum of up to 3 values, deterministic tree order; thread 0 writes.
__device__ __forceinline__ void block_sum3(double v0, double v1, double v2, double* out) {
  __shared__ double sh[3][kThreads];
  sh[0][threadIdx.x] = v0;
  sh[1][threadIdx.x] = v1;
  sh[2][threadIdx.x] = v2;
  __syncthreads();
  for (int st = kThreads / 2; st > 0; st >>= 1) {
    if (threadIdx.x < st) {
      sh[0][threadIdx.x] += sh[0][threadIdx.x + st];
      sh[1][threadIdx.x] += sh[1][threadIdx.x + st];
      sh[2][threadIdx.x] += sh[2][threadIdx.x + st];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    out[0] = sh[0][0];
    out[1] = sh[1][0];
    out[2] = sh[2][0];
  }
}

// scal layout per problem: [0] rz (even its), [1] rz (odd its), [2] pq, [3] rr, [4] bb, [5] done
__global__ void pcg_init_kernel(DAArgs a, const double* mu, const double* rhs, PCGWork w) {
  const int b = blockIdx.y;
  const long long o = (long long)b * a.N;
  const double h2 = a.hd;
  double rz = 0, rr = 0, bb = 0;
  for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < a.N; g += gridDim.x * blockDim.x) {
    const double di = 1.0 / (a.diag0[g] + mu[o + g] * h2);
    const double r = rhs[o + g];
    w.dinv[o + g] = di;
    w.x[o + g] = 0.0;
    w.r[o + g] = r;
    w.z[o + g] = di * r;
    w.p[o + g] = di * r;
    rz += r * di * r;
    rr += r * r;
    bb += r * r;
  }
  block_sum3(rz, rr, bb, w.partial + ((long long)b * kPCGBlocks + blockIdx.x) * 4);
}

// Sum the partials of problem blockIdx.x into scal slots.
__global__ void pcg_reduce_kernel(PCGWork w, int s0, int s1, int s2) {
  const int b = blockIdx.x;
  const double* p = w.partial + (long long)b * kPCGBlocks * 4;
  double v0 = 0, v1 = 0, v2 = 0;
  for (int t = threadIdx.x; t < kPCGBlocks; t += blockDim.x) {
    v0 += p[4 * t];
    v1 += p[4 * t + 1];
    v2 += p[4 * t + 2];
  }
  __shared__ double res[3];
  block_sum3(v0, v1, v2, res);
  if (threadIdx.x == 0) {
    double* sc = w.scal + 8 * b;
    if (s0 >= 0) sc[s0] = res[0];
    if (s1 >= 0) sc[s1] = res[1];
    if (s2 >= 0) sc[s2] = res[2];
  }
}

__global__ void pcg_spmv_kernel(DAArgs a, const double* mu, PCGWork w) {
  const int b = blockIdx.y;
  const long long o = (long long)b * a.N;
  const double h2 = a.hd;
  double pq = 0;
  for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < a.N; g += gridDim.x * blockDim.x) {
    const double q = apply_A(a, mu + o, w.p + o, g, h2);
    w.q[o + g] = q;
    pq += w.p[o + g] * q;
  }
  block_sum3(pq, 0.0, 0.0, w.partial + ((long long)b * kPCGBlocks + blockIdx.x) * 4);
}

__global__ void pcg_update_kernel(DAArgs a, PCGWork w, int parity) {
  const int b = blockIdx.y;
  const long long o = (long long)b * a.N;
  const double* sc = w.scal + 8 * b;
  const bool done = sc[5] != 0.0;
  const double rz = sc[parity], pq = sc[2];
  const double alpha = (done || pq == 0.0) ? 0.0 : rz / pq;
  double rz1 = 0, rr = 0;
  for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < a.N; g += gridDim.x * blockDim.x) {
    const double x = w.x[o + g] + alpha * w.p[o + g];
    const double r = w.r[o + g] - alpha * w.q[o + g];
    const double z = w.dinv[o + g] * r;
    w.x[o + g] = x;
    w.r[o + g] = r;
    w.z[o + g] = z;
    rz1 += r * z;
    rr += r * r;
  }
  block_sum3(rz1, rr, 0.0, w.partial + ((long long)b * kPCGBlocks + blockIdx.x) * 4);
}

__global__ void pcg_pupdate_kernel(DAArgs a, PCGWork w, int parity) {
  const int b = blockIdx.y;
  const long long o = (long long)b * a.N;
  const double* sc = w.scal + 8 * b;
  const bool done = sc[5] != 0.0;
  const double rz_old = sc[parity], rz_new = sc[parity ^ 1];
  const double beta = (done || rz_old == 0.0) ? 0.0 : rz_new / rz_old;
  for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < a.N; g += gridDim.x * blockDim.x)
    w.p[o + g] = w.z[o + g] + beta * w.p[o + g];
}

__global__ void pcg_mark_done_kernel(PCGWork w, int batch, double tol2) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= batch) return;
  double* sc = w.scal + 8 * b;
  if (sc[3] <= tol2 * sc[4]) sc[5] = 1.0;
}

__global__ void copy_kernel(long long n, const double* in, double* out) {
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x)
    out[t] = in[t];
}

// ---- multigrid preconditioner ------------------------------------------------
// Cell-centred geometric multigrid on the same finite-volume discretisation:
// level l + 1 halves every axis of level l (while all are even and >= 4), its
// operator is rediscretised at spacing 2h from the children's mean kappa and
// mean mu, restriction sums the four (eight) children's residuals (R = P^T for
// the piecewise-constant prolongation P), smoothing is damped Jacobi with the
// same sweeps before and after the coarse correction, and the coarsest level
// gets a fixed number of Jacobi sweeps from zero.  Every step is linear and
// the V-cycle is symmetric, so it is a valid conjugate-gradient preconditioner.

__global__ void coarsen_mean_kernel(const double* f, double* c, int fn0, int fn1, int fn2, int dim, long long fstride,
                                    long long cstride) {
  const int b = blockIdx.y;
  const int cn0 = fn0 / 2, cn1 = fn1 / 2, cn2 = dim == 3 ? fn2 / 2 : 1;
  const long long Nc = (long long)cn0 * cn1 * cn2;
  const double inv = dim == 3 ? 0.125 : 0.25;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < Nc; t += (long long)gridDim.x * blockDim.x) {
    const int I = (int)(t % cn0), J = (int)((t / cn0) % cn1), K = (int)(t / ((long long)cn0 * cn1));
    double acc = 0.0;
    for (int dz = 0; dz < (dim == 3 ? 2 : 1); ++dz)
      for (int dy = 0; dy < 2; ++dy)
        for (int dx = 0; dx < 2; ++dx)
          acc += f[(long long)b * fstride + ((long long)(dim == 3 ? 2 * K + dz : 0) * fn1 + 2 * J + dy) * fn0 + 2 * I + dx];
    c[(long long)b * cstride + t] = acc * inv;
  }
}

cudaError_t mg_setup(MGHierarchy& h, const DAArgs& fine, const double* d_kappa, int max_batch, DevAlloc alloc,
                     void* owner, cudaStream_t s) {
  h.nlev = 1;
  h.lev[0].A = fine;
  h.lev[0].kappa = const_cast<double*>(d_kappa);
  const double* kap = d_kappa;
  while (h.nlev < kMaxLevels) {
    const DAArgs& f = h.lev[h.nlev - 1].A;
    const bool ok = f.n0 % 2 == 0 && f.n1 % 2 == 0 && f.n0 >= 4 && f.n1 >= 4 &&
                    (f.dim == 2 || (f.n2 % 2 == 0 && f.n2 >= 4));
    if (!ok) break;
    DAArgs c = f;
    c.n0 = f.n0 / 2;
    c.n1 = f.n1 / 2;
    c.n2 = f.dim == 3 ? f.n2 / 2 : 1;
    c.N = c.n0 * c.n1 * c.n2;
    c.h = 2.0 * f.h;
    c.hd = f.dim == 3 ? c.h * c.h * c.h : c.h * c.h;
    double *ck, *d0, *cx, *cy, *cz, *bs;
    cudaError_t e;
    if ((e = alloc(owner, (void**)&ck, c.N * sizeof(double))) != cudaSuccess) return e;
    coarsen_mean_kernel<<<dim3(128, 1), kThreads, 0, s>>>(kap, ck, f.n0, f.n1, f.n2, f.dim, 0, 0);
    for (double** p : {&d0, &cx, &cy, &cz})
      if ((e = alloc(owner, (void**)p, c.N * sizeof(double))) != cudaSuccess) return e;
    if ((e = alloc(owner, (void**)&bs, (size_t)2 * c.dim * c.N * sizeof(double))) != cudaSuccess) return e;
    if ((e = da_setup(c, d0, cx, cy, cz, bs, ck, s)) != cudaSuccess) return e;
    h.lev[h.nlev].A = c;
    h.lev[h.nlev].kappa = ck;
    kap = ck;
    ++h.nlev;
  }
  for (int l = 0; l < h.nlev; ++l) {
    MGLevel& L = h.lev[l];
    const size_t bytes = (size_t)max_batch * L.A.N * sizeof(double);
    cudaError_t e;
    if (l > 0 && (e = alloc(owner, (void**)&L.mu, bytes)) != cudaSuccess) return e;
    if ((e = alloc(owner, (void**)&L.x2, bytes)) != cudaSuccess) return e;
    if (l > 0 && (e = alloc(owner, (void**)&L.x, bytes)) != cudaSuccess) return e;
    if (l > 0 && (e = alloc(owner, (void**)&L.b, bytes)) != cudaSuccess) return e;
  }
  return cudaGetLastError();
}

cudaError_t mg_rekappa(MGHierarchy& h, cudaStream_t s) {
  for (int l = 1; l < h.nlev; ++l) {
    const DAArgs& f = h.lev[l - 1].A;
    DAArgs& c = h.lev[l].A;
    coarsen_mean_kernel<<<dim3(128, 1), kThreads, 0, s>>>(h.lev[l - 1].kappa, h.lev[l].kappa, f.n0, f.n1, f.n2, f.dim,
                                                          0, 0);
    cudaError_t e = da_setup(c, const_cast<double*>(c.diag0), const_cast<double*>(c.cxf),
                             const_cast<double*>(c.cyf), const_cast<double*>(c.czf), const_cast<double*>(c.bside),
                             h.lev[l].kappa, s);
    if (e != cudaSuccess) return e;
  }
  return cudaGetLastError();
}

// x_out = x_in + omega D^-1 (b - A x_in); x_in = 0 when first
__global__ void mg_jacobi_kernel(DAArgs a, const double* mu, const double* xin, const double* b, double* xout,
                                 double omega, int first) {
  const long long o = (long long)blockIdx.y * a.N;
  for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < a.N; g += gridDim.x * blockDim.x) {
    const double d = a.diag0[g] + mu[o + g] * a.hd;
    if (first) {
      xout[o + g] = omega * b[o + g] / d;
    } else {
      const double ax = apply_A(a, mu + o, xin + o, g, a.hd);
      xout[o + g] = xin[o + g] + omega * (b[o + g] - ax) / d;
    }
  }
}

// b_c[I] = sum over the children i of I of (b_f - A_f x_f)[i]
__global__ void mg_restrict_kernel(DAArgs f, const double* mu, const double* x, const double* bf, double* bc,
                                   int cn0, int cn1, int cn2) {
  const long long Nc = (long long)cn0 * cn1 * cn2;
  const long long of = (long long)blockIdx.y * f.N, oc = (long long)blockIdx.y * Nc;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < Nc; t += (long long)gridDim.x * blockDim.x) {
    const int I = (int)(t % cn0), J = (int)((t / cn0) % cn1), K = (int)(t / ((long long)cn0 * cn1));
    double acc = 0.0;
    for (int dz = 0; dz < (f.dim == 3 ? 2 : 1); ++dz)
      for (int dy = 0; dy < 2; ++dy)
        for (int dx = 0; dx < 2; ++dx) {
          const int g = ((f.dim == 3 ? 2 * K + dz : 0) * f.n1 + 2 * J + dy) * f.n0 + 2 * I + dx;
          acc += bf[of + g] - apply_A(f, mu + of, x + of, g, f.hd);
        }
    bc[oc + t] = acc;
  }
}

// x_f[i] += x_c[parent(i)]
__global__ void mg_prolong_kernel(DAArgs f, const double* xc, double* xf, int cn0, int cn1, int cn2) {
  const long long Nc = (long long)cn0 * cn1 * cn2;
  const long long of = (long long)blockIdx.y * f.N, oc = (long long)blockIdx.y * Nc;
  for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < f.N; g += gridDim.x * blockDim.x) {
    const int i = g % f.n0, j = (g / f.n0) % f.n1, k = g / (f.n0 * f.n1);
    const long long pc = ((long long)(f.dim == 3 ? k / 2 : 0) * cn1 + j / 2) * cn0 + i / 2;
    xf[of + g] += xc[oc + pc];
  }
}

// All sweeps of the coarsest level in one CTA per problem (the level has at
// most kCoarseCells cells): x = 0, then `sweeps` damped-Jacobi sweeps, the
// result left in x.
constexpr int kCoarseCells = 4096;
__global__ void mg_coarse_kernel(DAArgs a, const double* mu, const double* b, double* x, double* x2, double omega,
                                 int sweeps) {
  const long long o = (long long)blockIdx.x * a.N;
  double* cur = x + o;
  double* nxt = x2 + o;
  for (int g = threadIdx.x; g < a.N; g += blockDim.x)
    cur[g] = omega * b[o + g] / (a.diag0[g] + mu[o + g] * a.hd);
  for (int it = 1; it < sweeps; ++it) {
    __syncthreads();
    for (int g = threadIdx.x; g < a.N; g += blockDim.x) {
      const double d = a.diag0[g] + mu[o + g] * a.hd;
      nxt[g] = cur[g] + omega * (b[o + g] - apply_A(a, mu + o, cur, g, a.hd)) / d;
    }
    double* t = cur;
    cur = nxt;
    nxt = t;
  }
  __syncthreads();
  if (cur != x + o)
    for (int g = threadIdx.x; g < a.N; g += blockDim.x) x[o + g] = cur[g];
}

static dim3 mg_grid(int N, int batch) {
  return dim3((unsigned)std::min(kPCGBlocks, (N + kThreads - 1) / kThreads), batch);
}

// z = V-cycle(r) for level l; x/x2/b of level 0 are bound by the caller.
static void mg_vcycle(MGHierarchy& h, int l, int batch, cudaStream_t s) {
  MGLevel& L = h.lev[l];
  const dim3 g = mg_grid(L.A.N, batch);
  if (l == h.nlev - 1 && L.A.N <= kCoarseCells) {
    mg_coarse_kernel<<<batch, 1024, 0, s>>>(L.A, L.mu, L.b, L.x, L.x2, h.omega, h.coarse_sweeps);
    return;
  }
  if (l == h.nlev - 1) {
    mg_jacobi_kernel<<<g, kThreads, 0, s>>>(L.A, L.mu, L.x, L.b, L.x, h.omega, 1);
    for (int it = 1; it < h.coarse_sweeps; ++it) {
      mg_jacobi_kernel<<<g, kThreads, 0, s>>>(L.A, L.mu, L.x, L.b, L.x2, h.omega, 0);
      mg_jacobi_kernel<<<g, kThreads, 0, s>>>(L.A, L.mu, L.x2, L.b, L.x, h.omega, 0);
      ++it;
    }
    return;
  }
  MGLevel& Cl = h.lev[l + 1];
  // pre-smoothing: nu sweeps from zero, result in x
  mg_jacobi_kernel<<<g, kThreads, 0, s>>>(L.A, L.mu, L.x, L.b, L.x2, h.omega, 1);
  mg_jacobi_kernel<<<g, kThreads, 0, s>>>(L.A, L.mu, L.x2, L.b, L.x, h.omega, 0);
  mg_restrict_kernel<<<mg_grid(Cl.A.N, batch), kThreads, 0, s>>>(L.A, L.mu, L.x, L.b, Cl.b, Cl.A.n0, Cl.A.n1, Cl.A.n2);
  mg_vcycle(h, l + 1, batch, s);
  mg_prolong_kernel<<<g, kThreads, 0, s>>>(L.A, Cl.x, L.x, Cl.A.n0, Cl.A.n1, Cl.A.n2);
  // post-smoothing: the same nu sweeps, result in x
  mg_jacobi_kernel<<<g, kThreads, 0, s>>>(L.A, L.mu, L.x, L.b, L.x2, h.omega, 0);
  mg_jacobi_kernel<<<g, kThreads, 0, s>>>(L.A, L.mu, L.x2, L.b, L.x, h.omega, 0);
}

__global__ void pcg_init_mg_kernel(DAArgs a, const double* rhs, PCGWork w) {
  const int b = blockIdx.y;
  const long long o = (long long)b * a.N;
  double rr = 0;
  for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < a.N; g += gridDim.x * blockDim.x) {
    const double r = rhs[o + g];
    w.x[o + g] = 0.0;
    w.r[o + g] = r;
    rr += r * r;
  }
  block_sum3(0.0, rr, rr, w.partial + ((long long)b * kPCGBlocks + blockIdx.x) * 4);
}

// x += alpha p, r -= alpha q, partial r.r  (the preconditioner runs after)
__global__ void pcg_update_mg_kernel(DAArgs a, PCGWork w, int parity) {
  const int b = blockIdx.y;
  const long long o = (long long)b * a.N;
  const double* sc = w.scal + 8 * b;
  const bool done = sc[5] != 0.0;
  const double rz = sc[parity], pq = sc[2];
  const double alpha = (done || pq == 0.0) ? 0.0 : rz / pq;
  double rr = 0;
  for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < a.N; g += gridDim.x * blockDim.x) {
    w.x[o + g] += alpha * w.p[o + g];
    const double r = w.r[o + g] - alpha * w.q[o + g];
    w.r[o + g] = r;
    rr += r * r;
  }
  block_sum3(0.0, rr, 0.0, w.partial + ((long long)b * kPCGBlocks + blockIdx.x) * 4);
}

__global__ void pcg_dot_rz_kernel(DAArgs a, PCGWork w, int set_p) {
  const int b = blockIdx.y;
  const long long o = (long long)b * a.N;
  double rz = 0;
  for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < a.N; g += gridDim.x * blockDim.x) {
    rz += w.r[o + g] * w.z[o + g];
    if (set_p) w.p[o + g] = w.z[o + g];
  }
  block_sum3(rz, 0.0, 0.0, w.partial + ((long long)b * kPCGBlocks + blockIdx.x) * 4);
}

// One conjugate-gradient iteration of every problem in the batch (parity =
// iteration number mod 2 selects the slot holding the current r.z).
static void pcg_iteration(const DAArgs& a, const double* mu, int batch, PCGWork& w, int parity, cudaStream_t s) {
  const dim3 grid(kPCGBlocks, batch);
  MGHierarchy* mg = w.mg;
  pcg_spmv_kernel<<<grid, kThreads, 0, s>>>(a, mu, w);
  pcg_reduce_kernel<<<batch, kThreads, 0, s>>>(w, 2, -1, -1);
  if (mg && mg->nlev > 0) {
    pcg_update_mg_kernel<<<grid, kThreads, 0, s>>>(a, w, parity);
    pcg_reduce_kernel<<<batch, kThreads, 0, s>>>(w, -1, 3, -1);
    mg_vcycle(*mg, 0, batch, s);
    pcg_dot_rz_kernel<<<grid, kThreads, 0, s>>>(a, w, 0);
    pcg_reduce_kernel<<<batch, kThreads, 0, s>>>(w, parity ^ 1, -1, -1);
  } else {
    pcg_update_kernel<<<grid, kThreads, 0, s>>>(a, w, parity);
    pcg_reduce_kernel<<<batch, kThreads, 0, s>>>(w, parity ^ 1, 3, -1);
  }
  pcg_pupdate_kernel<<<grid, kThreads, 0, s>>>(a, w, parity);
}

int pcg_solve(const DAArgs& a, const double* mu_in, int batch, const double* rhs, double* x, PCGWork& w,
              int max_iter, double tol, cudaStream_t s, cudaError_t* err) {
  const dim3 grid(kPCGBlocks, batch);
  const double tol2 = tol * tol;
  MGHierarchy* mg = w.mg;
  const bool multigrid = mg && mg->nlev > 0;
  // the iterations read mu from a buffer of their own, so that a captured
  // chunk of them stays valid for every call
  copy_kernel<<<256, kThreads, 0, s>>>((long long)batch * a.N, mu_in, w.mu);
  const double* mu = w.mu;
  cudaMemsetAsync(w.scal, 0, sizeof(double) * 8 * batch, s);
  if (multigrid) {
    // level 0 of the hierarchy works on the PCG vectors: the V-cycle maps r to z
    MGLevel& L0 = mg->lev[0];
    L0.A = a;
    L0.mu = w.mu;
    L0.b = w.r;
    L0.x = w.z;
    for (int l = 1; l < mg->nlev; ++l) {
      const DAArgs& f = mg->lev[l - 1].A;
      coarsen_mean_kernel<<<dim3(128, batch), kThreads, 0, s>>>(mg->lev[l - 1].mu, mg->lev[l].mu, f.n0, f.n1, f.n2,
                                                                 f.dim, f.N, mg->lev[l].A.N);
    }
    pcg_init_mg_kernel<<<grid, kThreads, 0, s>>>(a, rhs, w);
    pcg_reduce_kernel<<<batch, kThreads, 0, s>>>(w, -1, 3, 4);
    mg_vcycle(*mg, 0, batch, s);
    pcg_dot_rz_kernel<<<grid, kThreads, 0, s>>>(a, w, 1);
    pcg_reduce_kernel<<<batch, kThreads, 0, s>>>(w, 0, -1, -1);
  } else {
    pcg_init_kernel<<<grid, kThreads, 0, s>>>(a, mu, rhs, w);
    pcg_reduce_kernel<<<batch, kThreads, 0, s>>>(w, 0, 3, 4);
  }
  *err = cudaGetLastError();
  if (*err != cudaSuccess) return -1;
  // the host looks at the convergence flags after every chunk of iterations
  // (an even number, so that every chunk starts at parity 0)
  const int chunk = multigrid ? kPCGChunk : 4 * kPCGChunk;
  if (w.use_graphs && w.chunk_batch != batch) {
    if (w.chunk) cudaGraphExecDestroy(w.chunk);
    w.chunk = nullptr;
    w.chunk_batch = 0;
    if (!w.cap && (*err = cudaStreamCreateWithFlags(&w.cap, cudaStreamNonBlocking)) != cudaSuccess) return -1;
    if ((*err = cudaStreamBeginCapture(w.cap, cudaStreamCaptureModeThreadLocal)) != cudaSuccess) return -1;
    for (int k = 0; k < chunk; ++k) {
      pcg_iteration(a, mu, batch, w, k & 1, w.cap);
      pcg_mark_done_kernel<<<(batch + 127) / 128, 128, 0, w.cap>>>(w, batch, tol2);
    }
    cudaGraph_t g = nullptr;
    *err = cudaStreamEndCapture(w.cap, &g);
    if (*err != cudaSuccess) return -1;
    *err = cudaGraphInstantiate(&w.chunk, g, 0);
    cudaGraphDestroy(g);
    if (*err != cudaSuccess) { w.chunk = nullptr; return -1; }
    w.chunk_batch = batch;
  }
  int it = 0;
  int used = -1;
  while (it < max_iter) {
    const int len = std::min(chunk, max_iter - it);
    if (w.use_graphs && len == chunk) {
      if ((*err = cudaGraphLaunch(w.chunk, s)) != cudaSuccess) return -1;
    } else {
      for (int k = 0; k < len; ++k) {
        pcg_iteration(a, mu, batch, w, k & 1, s);
        pcg_mark_done_kernel<<<(batch + 127) / 128, 128, 0, s>>>(w, batch, tol2);
      }
    }
    it += len;
    cudaMemcpyAsync(w.hostscal, w.scal, sizeof(double) * 8 * batch, cudaMemcpyDeviceToHost, s);
    cudaError_t e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) { *err = e; return -1; }
    bool all = true;
    for (int b = 0; b < batch; ++b) all = all && (w.hostscal[8 * b + 5] != 0.0);
    if (all) { used = it; break; }
  }
  copy_kernel<<<256, kThreads, 0, s>>>((long long)batch * a.N, w.x, x);
  *err = cudaGetLastError();
  return used;
}

__global__ void hadamard_kernel(long long n, double alpha, const double* u, const double* v, double* out) {
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x)
    out[t] = alpha * u[t] * v[t];
}

cudaError_t da_hadamard(int batch, int N, double alpha, const double* u, const double* v, double* out,
                        cudaStream_t s) {
  hadamard_kernel<<<512, kThreads, 0, s>>>((long long)batch * N, alpha, u, v, out);
  return cudaGetLastError();
}

template <typename T>
__global__ void heating_kernel(long long n, const double* a1, const double* b1, const double* a2, const double* b2,
                               T* out) {
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x) {
    double v = a1[t] * b1[t];
    if (a2) v += a2[t] * b2[t];
    out[t] = (T)v;
  }
}

template <typename T>
cudaError_t da_heating_T(int batch, int N, const double* a1, const double* b1, const double* a2, const double* b2,
                         T* out, cudaStream_t s) {
  heating_kernel<T><<<512, kThreads, 0, s>>>((long long)batch * N, a1, b1, a2, b2, out);
  return cudaGetLastError();
}

template <typename T>
__global__ void adjoint_out_kernel(long long n, const double* phi, const T* hbar, const double* ht, double* g) {
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x)
    g[t] = phi[t] * ((double)hbar[t] + ht[t]);
}

template <typename T>
cudaError_t da_adjoint_out(int batch, int N, const double* phi, const T* hbar, const double* ht, double* g,
                           cudaStream_t s) {
  adjoint_out_kernel<T><<<512, kThreads, 0, s>>>((long long)batch * N, phi, hbar, ht, g);
  return cudaGetLastError();
}

template <typename T>
__global__ void to_double_kernel(long long n, const T* in, double* out) {
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x)
    out[t] = (double)in[t];
}

template <typename T>
cudaError_t T_to_double(long long n, const T* in, double* out, cudaStream_t s) {
  to_double_kernel<T><<<512, kThreads, 0, s>>>(n, in, out);
  return cudaGetLastError();
}

template <typename T>
__global__ void adjoint_rhs_kernel(long long n, double scale, const double* mu, const T* hbar, double* out) {
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x)
    out[t] = scale * mu[t] * (double)hbar[t];
}

template <typename T>
cudaError_t da_adjoint_rhs(int batch, int N, double scale, const double* mu, const T* hbar, double* out,
                           cudaStream_t s) {
  adjoint_rhs_kernel<T><<<512, kThreads, 0, s>>>((long long)batch * N, scale, mu, hbar, out);
  return cudaGetLastError();
}

// ---- derivatives in kappa --------------------------------------------------
// d/da of the harmonic mean 2ab/(a+b)
__device__ __forceinline__ double dharmonic(double a, double b) { return 2.0 * b * b / ((a + b) * (a + b)); }

// Per cell c: the faces to its neighbours (axis, direction) and its boundary
// sides.  mode 0: out = delta-b - delta-A phi for dkappa (gather form: the
// face (c, nb) changes its coefficient by hf (dh(k_c, k_nb) dk_c +
// dh(k_nb, k_c) dk_nb) and contributes -delta-t (phi_c - phi_nb); a boundary
// side s adds 2 q dk_c (I_s - gamma phi_c) with q = d/dk of k h^(d-1)/(gamma h
// + k)).  mode 1: out = the kappa gradient sum over faces of
// -dh(k_c, k_nb) hf (phi_c - phi_nb)(psi_c - psi_nb) plus 2 q (I_s - gamma
// phi_c) psi_c per boundary side.
__global__ void kappa_deriv_kernel(DAArgs a, const double* kappa, const double* phi, const double* v, unsigned mask,
                                   double* out, int mode, double scale) {
  const long long o = (long long)blockIdx.y * a.N;
  const double hf = (a.dim == 3) ? a.h : 1.0;
  const double hb = (a.dim == 3) ? a.h * a.h : a.h;
  const int sy = a.n0, sz = a.n0 * a.n1;
  for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < a.N; g += gridDim.x * blockDim.x) {
    const int i = g % a.n0, j = (g / a.n0) % a.n1, k = g / sz;
    const double kc = kappa[g], pc = phi[o + g], vc = v[o + g];
    double acc = 0.0;
    const int nbs[6] = {i > 0 ? g - 1 : -1, i < a.n0 - 1 ? g + 1 : -1, j > 0 ? g - sy : -1,
                        j < a.n1 - 1 ? g + sy : -1, (a.dim == 3 && k > 0) ? g - sz : -1,
                        (a.dim == 3 && k < a.n2 - 1) ? g + sz : -1};
    for (int f = 0; f < 6; ++f) {
      const int nb = nbs[f];
      if (nb < 0) continue;
      const double kn = kappa[nb];
      if (mode == 0) {
        const double dt = hf * (dharmonic(kc, kn) * vc + dharmonic(kn, kc) * v[o + nb]);
        acc -= dt * (pc - phi[o + nb]);
      } else {
        acc -= dharmonic(kc, kn) * hf * (pc - phi[o + nb]) * (vc - v[o + nb]);
      }
    }
    const double gh = a.gamma * a.h;
    const double q = gh * hb / ((gh + kc) * (gh + kc));
    const bool on[6] = {i == 0, i == a.n0 - 1, j == 0, j == a.n1 - 1, a.dim == 3 && k == 0,
                        a.dim == 3 && k == a.n2 - 1};
    for (int s = 0; s < 2 * a.dim; ++s) {
      if (!on[s]) continue;
      const double I = ((mask >> s) & 1u) ? 1.0 : 0.0;
      acc += 2.0 * q * (I - a.gamma * pc) * vc;
    }
    out[o + g] = scale * acc;
  }
}

cudaError_t da_kappa_source(const DAArgs& a, const double* kappa, int batch, const double* phi, const double* dkappa,
                            unsigned mask, double* out, cudaStream_t s) {
  kappa_deriv_kernel<<<dim3(128, batch), kThreads, 0, s>>>(a, kappa, phi, dkappa, mask, out, 0, 1.0);
  return cudaGetLastError();
}

cudaError_t da_kappa_grad(const DAArgs& a, const double* kappa, int batch, const double* phi, const double* psi,
                          unsigned mask, double scale, double* out, cudaStream_t s) {
  kappa_deriv_kernel<<<dim3(128, batch), kThreads, 0, s>>>(a, kappa, phi, psi, mask, out, 1, scale);
  return cudaGetLastError();
}

__global__ void axpy_kernel(long long n, double alpha, const double* x, double* y) {
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x)
    y[t] += alpha * x[t];
}

cudaError_t da_axpy(long long n, double alpha, const double* x, double* y, cudaStream_t s) {
  axpy_kernel<<<512, kThreads, 0, s>>>(n, alpha, x, y);
  return cudaGetLastError();
}

// Inner products in FP64: per thread a Neumaier-compensated running sum of
// the FP64 products, a fixed-order tree over the block, and a compensated
// sequential sum of the block partials.
__device__ __forceinline__ void neumaier(double& s, double& c, double v) {
  const double t = s + v;
  if (fabs(s) >= fabs(v)) c += (s - t) + v;
  else c += (v - t) + s;
  s = t;
}

template <typename T>
__global__ void dot_partial_kernel(long long len, const T* a, const T* b, double* partial) {
  const int bb = blockIdx.y;
  const T* x = a + (long long)bb * len;
  const T* y = b + (long long)bb * len;
  double s = 0, c = 0;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < len; t += (long long)gridDim.x * blockDim.x)
    neumaier(s, c, (double)x[t] * (double)y[t]);
  block_sum3(s, c, 0.0, partial + ((long long)bb * kPartials + blockIdx.x) * 4);
}

__global__ void dot_final_kernel(const double* partial, double* out, int batch) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= batch) return;
  double s = 0, c = 0;
  for (int t = 0; t < kPartials; ++t) {
    neumaier(s, c, partial[((long long)b * kPartials + t) * 4]);
    neumaier(s, c, partial[((long long)b * kPartials + t) * 4 + 1]);
  }
  out[b] = s + c;
}

template <typename T>
cudaError_t dot_compensated(int batch, long long len, const T* a, const T* b, double* d_partial, double* d_out,
                            cudaStream_t s) {
  dot_partial_kernel<T><<<dim3(kPartials, batch), kThreads, 0, s>>>(len, a, b, d_partial);
  dot_final_kernel<<<(batch + 127) / 128, 128, 0, s>>>(d_partial, d_out, batch);
  return cudaGetLastError();
}

#define QPAT_DA_INST(T)                                                                                  \
  template cudaError_t da_heating_T<T>(int, int, const double*, const double*, const double*,           \
                                       const double*, T*, cudaStream_t);                                 \
  template cudaError_t da_adjoint_out<T>(int, int, const double*, const T*, const double*, double*,      \
                                         cudaStream_t);                                                  \
  template cudaError_t T_to_double<T>(long long, const T*, double*, cudaStream_t);                      \
  template cudaError_t da_adjoint_rhs<T>(int, int, double, const double*, const T*, double*, cudaStream_t); \
  template cudaError_t dot_compensated<T>(int, long long, const T*, const T*, double*, double*, cudaStream_t);
QPAT_DA_INST(float)
QPAT_DA_INST(double)

}  // namespace qpat
