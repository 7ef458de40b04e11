// Derivatives of H_a in the sound speed and the density on the GPU: the C
// entry points qpat_jvp_medium and qpat_vjp_medium over the loops of
// medium_ops.cuh (tangent loop; forward loop followed by its exact transpose,
// with the forward fields kept for every step or recomputed segment by
// segment from forward-state checkpoints), run on a 2D context's own tables
// in its precision (FP64 or FP32; directions, weights, outputs and gradient
// sums FP64).  Every per-element functor is launched as a grid-stride kernel on
// the context's stream; 2D FFTs run as one shared-memory line-FFT launch per
// axis.
#include <math.h>

#include <map>
#include <vector>

#include "fast_kernels.cuh"
#include "medium_ops.cuh"
#include "qpat.h"
#include "qpat_internal.h"

namespace qpat {
// Defined in api.cu: the FP64 (FP32) 2D tables of a context (NULL for a
// context of the other precision or a 3D context), the absorption exponent,
// the lossless flag and the stream.
const PropArgs<double>* ctx_tables64(const ::qpat_ctx* c, double* y, int* lossless, cudaStream_t* stream);
const PropArgs<float>* ctx_tables32(const ::qpat_ctx* c, double* y, int* lossless, cudaStream_t* stream);
void ctx_add_launches(::qpat_ctx* c, long long n);
// Checkpoint interval of the medium gradient set on the context (0: automatic).
int ctx_medium_k(const ::qpat_ctx* c);
}  // namespace qpat

namespace {

using namespace qpat;
using namespace qpat::med;

constexpr int kThreads = 256;
// Largest whole-history tape of the medium gradient (beyond it: checkpoints).
constexpr double kFullTapeBytes = 2.0 * 1024 * 1024 * 1024;
constexpr long long kMaxBlocks = 152 * 16;

template <class F>
__global__ void __launch_bounds__(kThreads) for_each_kernel(const F f, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    f(i);
}

// x transforms of nb real fields of G points: Z[b] = F_x (f_b + 0 i), field
// b = blockIdx.y.  A CTA loads M consecutive rows into shared memory (row
// stride S = L + 1), runs the mixed-radix Stockham stages of fft_batch there
// and stores the complex rows.
constexpr int kLineThreads = 256;
template <typename R>
__global__ void __launch_bounds__(kLineThreads) rows_fwd_kernel(const FieldPtrs<const R*> f, Cplx<R>* Z, long long G,
                                                                 int nx, int ny, const FFTPlan plan,
                                                                 const Cplx<R>* tw, int M) {
  typedef Cplx<R> C;
  extern __shared__ __align__(16) unsigned char sm_raw[];
  const int L = plan.L, S = L + 1;
  C* buf0 = reinterpret_cast<C*>(sm_raw);
  C* buf1 = buf0 + M * S;
  const int line0 = blockIdx.x * M;
  const int mloc = min(M, ny - line0);
  const R* fb = f.p[blockIdx.y];
  for (int t = threadIdx.x; t < M * L; t += blockDim.x) {
    const int m = t / L, i = t - m * L;
    C v;
    v.x = m < mloc ? fb[(long long)(line0 + m) * nx + i] : (R)0;
    v.y = 0;
    buf0[m * S + i] = v;
  }
  __syncthreads();
  const C* res = fft_batch(plan, buf0, buf1, M, S, tw);
  C* Zb = Z + (long long)blockIdx.y * G;
  for (int t = threadIdx.x; t < M * L; t += blockDim.x) {
    const int m = t / L, i = t - m * L;
    if (m < mloc) Zb[(long long)(line0 + m) * nx + i] = res[m * S + i];
  }
}

// Per group of M adjacent columns (x index col0 + m): the y transforms of the
// nin x-transformed inputs, the combined products of the tm.no outputs and
// their inverse y transforms (as conj(FFT(conj .))), Zc[o] on the same
// layout.  Shared memory: two buffers of W = max(nin, no) lines per column,
// line (b M + m) of each holding column m of field b; the loads and stores
// run with m fastest, so a warp moves M adjacent values of each row.
constexpr int kColThreads = 512;
template <typename R>
__global__ void __launch_bounds__(kColThreads) cols_kernel(const Cplx<R>* Zi, int nin, Cplx<R>* Zc, const Terms tm,
                                                            const Tables<R> t, long long G, const FFTPlan plan, int M,
                                                            int W) {
  typedef Cplx<R> C;
  extern __shared__ __align__(16) unsigned char sm_raw[];
  const int L = plan.L, S = L + 1, nx = t.nx;
  C* A = reinterpret_cast<C*>(sm_raw);
  C* B = A + (long long)W * M * S;
  const int col0 = blockIdx.x * M;
  const int mloc = min(M, nx - col0);
  for (int u = threadIdx.x; u < nin * M * L; u += blockDim.x) {
    const int b = u / (M * L), r = u - b * M * L, i = r / M, m = r - i * M;
    C v;
    v.x = 0;
    v.y = 0;
    if (m < mloc) v = Zi[b * G + (long long)i * nx + col0 + m];
    A[(b * M + m) * S + i] = v;
  }
  __syncthreads();
  C* res = fft_batch(plan, A, B, nin * M, S, t.twy);
  C* oth = res == A ? B : A;
  for (int u = threadIdx.x; u < tm.no * M * L; u += blockDim.x) {
    const int o = u / (M * L), r = u - o * M * L, j = r / M, m = r - j * M;
    C acc = z<R>((R)0, (R)0);
    if (m < mloc) {
      for (int q = 0; q < tm.nterm[o]; ++q) {
        C s = symbol(t, tm.sym[o][q], j, col0 + m);
        if (tm.conj) s = zconj(s);
        acc = zadd(acc, zmul(s, res[(tm.in[o][q] * M + m) * S + j]));
      }
    }
    oth[(o * M + m) * S + j] = zconj(acc);
  }
  __syncthreads();
  const C* res2 = fft_batch(plan, oth, res, tm.no * M, S, t.twy);
  for (int u = threadIdx.x; u < tm.no * M * L; u += blockDim.x) {
    const int o = u / (M * L), r = u - o * M * L, j = r / M, m = r - j * M;
    if (m < mloc) Zc[o * G + (long long)j * nx + col0 + m] = zconj(res2[(o * M + m) * S + j]);
  }
}

// Inverse x transforms of no spectra (as conj(FFT(conj .))), keeping
// out[o] = alpha Re(.), output o = blockIdx.y; M rows per CTA.
template <typename R>
__global__ void __launch_bounds__(kLineThreads) rows_inv_kernel(const Cplx<R>* Z, const FieldPtrs<R*> out, R alpha,
                                                                 long long G, int nx, int ny, const FFTPlan plan,
                                                                 const Cplx<R>* tw, int M) {
  typedef Cplx<R> C;
  extern __shared__ __align__(16) unsigned char sm_raw[];
  const int L = plan.L, S = L + 1;
  C* buf0 = reinterpret_cast<C*>(sm_raw);
  C* buf1 = buf0 + M * S;
  const int line0 = blockIdx.x * M;
  const int mloc = min(M, ny - line0);
  const C* Zb = Z + (long long)blockIdx.y * G;
  for (int t = threadIdx.x; t < M * L; t += blockDim.x) {
    const int m = t / L, i = t - m * L;
    C v;
    v.x = 0;
    v.y = 0;
    if (m < mloc) v = zconj(Zb[(long long)(line0 + m) * nx + i]);
    buf0[m * S + i] = v;
  }
  __syncthreads();
  const C* res = fft_batch(plan, buf0, buf1, M, S, tw);
  R* ob = out.p[blockIdx.y];
  for (int t = threadIdx.x; t < M * L; t += blockDim.x) {
    const int m = t / L, i = t - m * L;
    if (m < mloc) ob[(long long)(line0 + m) * nx + i] = alpha * res[m * S + i].x;
  }
}

// FP32 x transforms (forward: real fields in, spectra out; inverse: spectra
// in as conj(FFT(conj .)), alpha times the real part out) on the
// compile-time Stockham FFT of the propagation passes, for the extents that
// have one: TPT threads per row, several rows per CTA, the twiddles read
// through L1.  Field blockIdx.y.
template <int L>
constexpr int med_rows_per_cta() { return (256 / SGeom<L>::TPT) > 0 ? 256 / SGeom<L>::TPT : 1; }
template <int L, bool INV>
__global__ void __launch_bounds__(med_rows_per_cta<L>() * SGeom<L>::TPT)
rows_fast_kernel(const FieldPtrs<const float*> fin, const float2* Zin, float2* Zout, const FieldPtrs<float*> fout,
                 float alpha, long long G, int nx, int ny, const float2* tw) {
  typedef SGeom<L> Gm;
  constexpr int TPT = Gm::TPT, SL = Gm::SL, Q1 = Gm::Q1, QL = Gm::QL, RPC = med_rows_per_cta<L>();
  extern __shared__ __align__(16) unsigned char sm_raw[];
  const int m = threadIdx.x / TPT, j = threadIdx.x - m * TPT;
  float2* bufA = reinterpret_cast<float2*>(sm_raw) + m * 2 * SL;
  float2* bufB = bufA + SL;
  const int row = blockIdx.x * RPC + m;
  const bool valid = row < ny;
  const long long o = (long long)(valid ? row : 0) * nx;
  const long long of = (long long)blockIdx.y * G + o;
  float2 v[1][Q1];
  if (j < L / Q1) {
#pragma unroll
    for (int r = 0; r < Q1; ++r) {
      const int i = j + r * (L / Q1);
      float2 x = make_float2(0.f, 0.f);
      if (valid) {
        if (INV) x = zconj(Zin[of + i]);
        else x.x = fin.p[blockIdx.y][o + i];
      }
      v[0][r] = x;
    }
  }
  float2 X[1][QL];
  fft_stockham<L, Gm::Q1, Gm::Q2, Gm::Q3, 1, false, false>(v, X, bufA, bufB, SL, j, tw);
  if (valid && j < L / QL) {
#pragma unroll
    for (int r = 0; r < QL; ++r) {
      const int k = j + r * (L / QL);
      if (INV) fout.p[blockIdx.y][o + k] = alpha * X[0][r].x;
      else Zout[of + k] = X[0][r];
    }
  }
}

// FP32 y transforms, products and inverse y transforms of M adjacent columns
// on the compile-time Stockham FFT (extents with one): the columns are
// staged as in cols_kernel, then NG thread groups of TPT threads transform
// one staged line each per wave, reading it into registers and writing the
// transform back in natural order (in place); the products and the stores
// follow as in cols_kernel.  Every thread runs every wave (the transforms
// synchronise the CTA).
template <int L>
constexpr int med_col_groups() { return L >= 512 ? 8 : 16; }
template <int L>
__global__ void __launch_bounds__(med_col_groups<L>() * SGeom<L>::TPT)
cols_fast_kernel(const float2* Zi, int nin, float2* Zc, const Terms tm, const Tables<float> t, long long G, int M) {
  typedef SGeom<L> Gm;
  typedef float2 C;
  constexpr int TPT = Gm::TPT, SL = Gm::SL, Q1 = Gm::Q1, QL = Gm::QL, NG = med_col_groups<L>(), S = L + 1;
  extern __shared__ __align__(16) unsigned char sm_raw[];
  C* A = reinterpret_cast<C*>(sm_raw);                           // [nin M][S] inputs, then their transforms
  C* B = A + (long long)nin * M * S;                             // [no M][S] products, then their transforms
  C* scr = B + (long long)tm.no * M * S;                         // [NG][SL] Stockham buffer per group
  const int g = threadIdx.x / TPT, j = threadIdx.x - g * TPT;
  C* buf = scr + g * SL;
  const int nx = t.nx, col0 = blockIdx.x * M, mloc = min(M, nx - col0);
  for (int u = threadIdx.x; u < nin * M * L; u += blockDim.x) {
    const int b = u / (M * L), r = u - b * M * L, i = r / M, m = r - i * M;
    C v = make_float2(0.f, 0.f);
    if (m < mloc) v = Zi[b * G + (long long)i * nx + col0 + m];
    A[(b * M + m) * S + i] = v;
  }
  __syncthreads();
  // lines [0, n) of X in place: forward transforms (the inverse ones are
  // fed conjugated and stored conjugated by the caller's loops)
  auto transform = [&](C* X, int n) {
    for (int w0 = 0; w0 < n; w0 += NG) {
      const int line = w0 + g;
      const bool lv = line < n;
      C v[1][Q1];
      if (j < L / Q1) {
#pragma unroll
        for (int r = 0; r < Q1; ++r) v[0][r] = lv ? X[line * S + j + r * (L / Q1)] : make_float2(0.f, 0.f);
      }
      C Y[1][QL];
      fft_stockham<L, Gm::Q1, Gm::Q2, Gm::Q3, 1, true, false>(v, Y, buf, buf, SL, j, t.twy);
      if (lv && j < L / QL) {
#pragma unroll
        for (int r = 0; r < QL; ++r) X[line * S + j + r * (L / QL)] = Y[0][r];
      }
      __syncthreads();
    }
  };
  transform(A, nin * M);
  for (int u = threadIdx.x; u < tm.no * M * L; u += blockDim.x) {
    const int o = u / (M * L), r = u - o * M * L, jj = r / M, m = r - jj * M;
    C acc = make_float2(0.f, 0.f);
    if (m < mloc) {
      for (int q = 0; q < tm.nterm[o]; ++q) {
        C sy = symbol(t, tm.sym[o][q], jj, col0 + m);
        if (tm.conj) sy = zconj(sy);
        acc = zadd(acc, zmul(sy, A[(tm.in[o][q] * M + m) * S + jj]));
      }
    }
    B[(o * M + m) * S + jj] = zconj(acc);
  }
  __syncthreads();
  transform(B, tm.no * M);
  for (int u = threadIdx.x; u < tm.no * M * L; u += blockDim.x) {
    const int o = u / (M * L), r = u - o * M * L, jj = r / M, m = r - jj * M;
    if (m < mloc) Zc[o * G + (long long)jj * nx + col0 + m] = zconj(B[(o * M + m) * S + jj]);
  }
}

// Lines per CTA of the row launches: about 48 KB of shared memory per
// buffer, 1 to 16 lines.
int lines_per_cta(int L, int csize) {
  const int m = 49152 / ((L + 1) * csize);
  return m < 1 ? 1 : m > 16 ? 16 : m;
}
// Columns per CTA of the column launch: two buffers of W lines per column
// within the shared-memory budget, a power of two from 1 to 8 (so that a
// warp's accesses to a row cover whole 32-byte sectors where possible).
// Budget 110 KB in FP32 (two CTAs per SM) and 220 KB in FP64 (measured at
// 576^2, 2000 steps, gradient / tangent: FP32 1.95 / 0.79 s against 2.51 /
// 0.85 s with 220 KB and 1.89 / 0.89 s with 56 KB; FP64 4.73 / 2.90 s with
// 220 KB against 4.93 / 3.06 s with 110 KB).
int cols_per_cta(int L, int W, int csize) {
  const int budget = csize >= 16 ? 225280 : 112640;
  const int m = budget / (2 * W * (L + 1) * csize);
  int p = 1;
  while (2 * p <= m && 2 * p <= 8) p *= 2;
  return p;
}

FFTPlan to_fft_plan(const Plan& p) {
  FFTPlan f{};
  f.L = p.L;
  f.nstages = p.nstages;
  for (int s = 0; s < p.nstages && s < qpat::kMaxStages; ++s) f.radix[s] = p.radix[s];
  return f;
}

struct GpuEx {
  cudaStream_t s;
  std::map<const void*, size_t> smem_set;
  long long launches = 0;
  cudaError_t err = cudaSuccess;
  // shared-memory limit of a launch, then the launch bookkeeping
  template <class K>
  bool smem_limit(K* kernel, size_t smem) {
    if (err != cudaSuccess) return false;
    size_t& set = smem_set[reinterpret_cast<const void*>(kernel)];   // limit already set during this call
    if (smem <= set) return true;
    const cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) err = e;
    else set = smem;
    return e == cudaSuccess;
  }
  void launched() {
    ++launches;
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess && err == cudaSuccess) err = e;
  }
  // the compile-time x transforms (FP32, extents 24, 168, 576); false when
  // the extent has none
  template <int L, bool INV>
  bool rows_fast_len(const FieldPtrs<const float*>& fin, const float2* Zin, float2* Zout,
                     const FieldPtrs<float*>& fout, float alpha, int nf, const Tables<float>& t, long long G) {
    constexpr int RPC = med_rows_per_cta<L>();
    const size_t smem = (size_t)RPC * 2 * SGeom<L>::SL * sizeof(float2);
    if (!smem_limit(rows_fast_kernel<L, INV>, smem)) return true;
    rows_fast_kernel<L, INV><<<dim3((t.ny + RPC - 1) / RPC, nf), RPC * SGeom<L>::TPT, smem, s>>>(
        fin, Zin, Zout, fout, alpha, G, t.nx, t.ny, t.twx);
    launched();
    return true;
  }
  template <bool INV>
  bool rows_fast(const FieldPtrs<const float*>& fin, const float2* Zin, float2* Zout, const FieldPtrs<float*>& fout,
                 float alpha, int nf, const Tables<float>& t, long long G) {
    if (t.px.L != t.nx) return false;
    switch (t.nx) {
      case 24: return rows_fast_len<24, INV>(fin, Zin, Zout, fout, alpha, nf, t, G);
      case 168: return rows_fast_len<168, INV>(fin, Zin, Zout, fout, alpha, nf, t, G);
      case 576: return rows_fast_len<576, INV>(fin, Zin, Zout, fout, alpha, nf, t, G);
      default: return false;
    }
  }
  // Z[b] = F_x f_b for b < nb
  template <typename R>
  void rows_forward(const FieldPtrs<const R*>& f, int nb, Cplx<R>* Z, const Tables<R>& t, long long G) {
    if constexpr (std::is_same<R, float>::value) {
      if (nb > 0 && err == cudaSuccess && rows_fast<false>(f, nullptr, Z, FieldPtrs<float*>{}, 1.f, nb, t, G)) return;
    }
    const FFTPlan plan = to_fft_plan(t.px);
    const int M = lines_per_cta(plan.L, (int)sizeof(Cplx<R>));
    const size_t smem = 2 * (size_t)M * (plan.L + 1) * sizeof(Cplx<R>);
    if (nb <= 0 || !smem_limit(rows_fwd_kernel<R>, smem)) return;
    rows_fwd_kernel<R><<<dim3((t.ny + M - 1) / M, nb), kLineThreads, smem, s>>>(f, Z, G, t.nx, t.ny, plan, t.twx, M);
    launched();
  }
  // the compile-time column launch (FP32, extents 24, 168, 576)
  template <int L>
  bool cols_fast_len(const float2* Zi, int nin, float2* Zc, const Terms& tm, const Tables<float>& t, long long G) {
    constexpr int NG = med_col_groups<L>();
    const int W = nin > tm.no ? nin : tm.no;
    int M = 1;
    while (2 * M * W <= NG && 2 * M <= 8) M *= 2;                // a wave transforms M W lines
    const size_t smem = ((size_t)(nin + tm.no) * M * (L + 1) + (size_t)NG * SGeom<L>::SL) * sizeof(float2);
    if (!smem_limit(cols_fast_kernel<L>, smem)) return true;
    cols_fast_kernel<L><<<(t.nx + M - 1) / M, NG * SGeom<L>::TPT, smem, s>>>(Zi, nin, Zc, tm, t, G, M);
    launched();
    return true;
  }
  // per column: y transforms of Zi[0..nin), the products tm, inverse y transforms into Zc
  template <typename R>
  void cols_combine(const Cplx<R>* Zi, int nin, Cplx<R>* Zc, const Terms& tm, const Tables<R>& t, long long G) {
    if constexpr (std::is_same<R, float>::value) {
      if (nin > 0 && err == cudaSuccess && t.py.L == t.ny) {
        switch (t.ny) {
          case 24: cols_fast_len<24>(Zi, nin, Zc, tm, t, G); return;
          case 168: cols_fast_len<168>(Zi, nin, Zc, tm, t, G); return;
          case 576: cols_fast_len<576>(Zi, nin, Zc, tm, t, G); return;
          default: break;
        }
      }
    }
    const FFTPlan plan = to_fft_plan(t.py);
    const int W = nin > tm.no ? nin : tm.no;
    const int M = cols_per_cta(plan.L, W, (int)sizeof(Cplx<R>));
    const size_t smem = 2 * (size_t)W * M * (plan.L + 1) * sizeof(Cplx<R>);
    if (nin <= 0 || !smem_limit(cols_kernel<R>, smem)) return;
    cols_kernel<R><<<(t.nx + M - 1) / M, kColThreads, smem, s>>>(Zi, nin, Zc, tm, t, G, plan, M, W);
    launched();
  }
  // out[o] = alpha Re F_x^-1 Z[o] for o < no
  template <typename R>
  void rows_inverse(const Cplx<R>* Z, const FieldPtrs<R*>& out, int no, R alpha, const Tables<R>& t, long long G) {
    if constexpr (std::is_same<R, float>::value) {
      if (no > 0 && err == cudaSuccess && rows_fast<true>(FieldPtrs<const float*>{}, Z, nullptr, out, alpha, no, t, G))
        return;
    }
    const FFTPlan plan = to_fft_plan(t.px);
    const int M = lines_per_cta(plan.L, (int)sizeof(Cplx<R>));
    const size_t smem = 2 * (size_t)M * (plan.L + 1) * sizeof(Cplx<R>);
    if (no <= 0 || !smem_limit(rows_inv_kernel<R>, smem)) return;
    rows_inv_kernel<R><<<dim3((t.ny + M - 1) / M, no), kLineThreads, smem, s>>>(Z, out, alpha, G, t.nx, t.ny, plan,
                                                                                t.twx, M);
    launched();
  }
  template <class F>
  void run(long long n, const F& f) {
    if (n <= 0 || err != cudaSuccess) return;
    long long blocks = (n + kThreads - 1) / kThreads;
    if (blocks > kMaxBlocks) blocks = kMaxBlocks;
    for_each_kernel<F><<<(unsigned)blocks, kThreads, 0, s>>>(f, n);
    ++launches;
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) err = e;
  }
  // record a host-side failure; later run() calls launch nothing
  void fail(cudaError_t e) {
    if (err == cudaSuccess) err = e;
  }
};

// Device workspace of one call, zero-filled, freed on every exit path.
struct Arena {
  std::vector<void*> ptrs;
  cudaError_t err = cudaSuccess;
  cudaStream_t s;
  template <typename P>
  P* get(long long count) {
    void* v = nullptr;
    if (err == cudaSuccess) err = cudaMalloc(&v, (size_t)(count > 0 ? count : 1) * sizeof(P));
    if (err != cudaSuccess) return nullptr;
    ptrs.push_back(v);
    err = cudaMemsetAsync(v, 0, (size_t)(count > 0 ? count : 1) * sizeof(P), s);
    return (P*)v;
  }
  ~Arena() {
    cudaStreamSynchronize(s);
    for (void* p : ptrs) cudaFree(p);
  }
};

void copy_plan(const FFTPlan& in, Plan& out) {
  out.L = in.L;
  out.nstages = in.nstages;
  for (int s = 0; s < in.nstages && s < med::kMaxStages; ++s) out.radix[s] = in.radix[s];
}

// Tables of a 2D context of precision R; QPAT_EINVAL when the context is of
// the other precision or 3D.
template <typename R>
int tables_of(qpat_ctx* c, Tables<R>& t, cudaStream_t* s) {
  double y = 0.0;
  int lossless = 0;
  const PropArgs<R>* a;
  if constexpr (sizeof(R) == sizeof(double)) a = ctx_tables64(c, &y, &lossless, s);
  else a = ctx_tables32(c, &y, &lossless, s);
  if (!a) return ctx_fail(c, QPAT_EINVAL, "medium derivatives need a 2D context");
  t.nx = a->nx; t.ny = a->ny; t.nxh = a->nxh; t.pml = a->pml; t.n0 = a->n0; t.n1 = a->n1; t.ns = a->ns;
  t.nt = a->nt; t.lossless = lossless; t.dt = a->dt; t.y = y;
  t.Cc = a->Cc; t.rho0 = a->rho0; t.dtrsx = a->dtrsx; t.dtrsy = a->dtrsy; t.tau = a->tau; t.eta = a->eta;
  t.ax = a->ax; t.asx = a->asx; t.ay = a->ay; t.asy = a->asy;
  t.kap = a->kap; t.kp1 = a->kp1; t.kp2 = a->kp2;
  t.shxp = a->shxp; t.shxm = a->shxm; t.shyp = a->shyp; t.shym = a->shym; t.twx = a->twx; t.twy = a->twy;
  t.sidx = a->sidx; t.sw = a->sw; t.rowptr = a->rowptr; t.pcol = a->pcol; t.pent = a->pent; t.esens = a->esens;
  t.ew = a->ew;
  copy_plan(a->px, t.px);
  copy_plan(a->py, t.py);
  if (a->px.nstages > med::kMaxStages || a->py.nstages > med::kMaxStages)
    return ctx_fail(c, QPAT_EINVAL, "FFT plan has too many stages");
  return QPAT_OK;
}

int finish(qpat_ctx* c, GpuEx& ex, Arena& w) {
  ctx_add_launches(c, ex.launches);
  cudaError_t e = ex.err != cudaSuccess ? ex.err : w.err;
  if (e == cudaSuccess) e = cudaStreamSynchronize(ex.s);
  if (e == cudaSuccess) return QPAT_OK;
  return ctx_fail(c, e == cudaErrorMemoryAllocation ? QPAT_ENOMEM : QPAT_ECUDA, cudaGetErrorString(e));
}

template <typename R>
qpat_status jvp_medium(qpat_ctx* ctx, const double* p0, const double* dc, const double* drho, double* dP) {
  Tables<R> t{};
  cudaStream_t s = nullptr;
  int st = tables_of(ctx, t, &s);
  if (st != QPAT_OK) return (qpat_status)st;
  const long long G = (long long)t.nx * t.ny;
  Arena w;
  w.s = s;
  GpuEx ex;
  ex.s = s;
  Fields<R> f{};
  for (R** q : {&f.P0, &f.p, &f.vx, &f.vy, &f.rx, &f.ry, &f.r, &f.u, &f.gx, &f.gy, &f.dx, &f.dy, &f.Yr, &f.Yu,
                &f.dp, &f.dvx, &f.dvy, &f.drx, &f.dry, &f.dr, &f.du, &f.dgx, &f.dgy, &f.ddx, &f.ddy, &f.YdR, &f.Ydu})
    *q = w.get<R>(G);
  double* zero = w.get<double>(G);
  Cplx<R>* Z[2];
  for (Cplx<R>*& z : Z) z = w.get<Cplx<R>>(kMaxBatch * G);
  if (w.err != cudaSuccess) return (qpat_status)finish(ctx, ex, w);
  Spectral<GpuEx, R> S{ex, t, G, Z[0], Z[1]};
  ex.run(G, Embed<R>{t, p0, f.P0});
  jvp_loop(ex, t, S, f, dc ? dc : zero, drho ? drho : zero, dP);
  return (qpat_status)finish(ctx, ex, w);
}

template <typename R>
qpat_status vjp_medium(qpat_ctx* ctx, const double* p0, const double* wts, double* g_c, double* g_rho) {
  Tables<R> t{};
  cudaStream_t s = nullptr;
  int st = tables_of(ctx, t, &s);
  if (st != QPAT_OK) return (qpat_status)st;
  const long long G = (long long)t.nx * t.ny;
  Arena w;
  w.s = s;
  GpuEx ex;
  ex.s = s;
  Fields<R> f{};
  for (R** q : {&f.P0, &f.p, &f.vx, &f.vy, &f.rx, &f.ry, &f.r, &f.u}) *q = w.get<R>(G);
  // Tape length: every step while the whole history stays within
  // kFullTapeBytes, else checkpoints every K steps with K near
  // sqrt(5 nt / fields), which minimises checkpoints (5 fields each) plus
  // tape (fields per step); a K set with qpat_set_medium_checkpoints wins.
  const int nf = t.lossless ? 5 : 7;
  int K = ctx_medium_k(ctx);
  if (K <= 0) {
    K = (double)t.nt * nf * G * sizeof(R) <= kFullTapeBytes ? t.nt : (int)ceil(sqrt(5.0 * t.nt / nf));
  }
  if (K > t.nt) K = t.nt;
  Tape<R> tp{};
  for (R** q : {&tp.gx, &tp.gy, &tp.dx, &tp.dy, &tp.X}) *q = w.get<R>(G * K);
  if (!t.lossless) {
    tp.Yr = w.get<R>(G * K);
    tp.Yu = w.get<R>(G * K);
  }
  R* ck = K < t.nt ? w.get<R>(5 * G * ((t.nt + K - 1) / K)) : nullptr;
  RevFields<R> b{};
  for (R** q : {&b.pb, &b.Cp, &b.e1, &b.e2, &b.t1, &b.ub, &b.rbx, &b.rby, &b.dbx, &b.dby, &b.vbx, &b.vby, &b.fx,
                &b.fy, &b.ex, &b.ey})
    *q = w.get<R>(G);
  for (double** q : {&b.qb, &b.gC, &b.gtau, &b.geta, &b.grho, &b.grsx, &b.grsy}) *q = w.get<double>(G);
  double* gc = g_c ? g_c : w.get<double>(G);
  double* gr = g_rho ? g_rho : w.get<double>(G);
  Cplx<R>* Z[2];
  for (Cplx<R>*& z : Z) z = w.get<Cplx<R>>(kMaxBatch * G);
  if (w.err != cudaSuccess) return (qpat_status)finish(ctx, ex, w);
  Spectral<GpuEx, R> S{ex, t, G, Z[0], Z[1]};
  ex.run(G, Embed<R>{t, p0, f.P0});
  vjp_loop(ex, t, S, f, tp, b, K, ck, wts, gc, gr);
  return (qpat_status)finish(ctx, ex, w);
}

// Sweep precision of a context: its own (FP64 or FP32), -1 for 3D.
int sweep_precision(qpat_ctx* c) {
  double y;
  int lossless;
  cudaStream_t s;
  if (ctx_tables64(c, &y, &lossless, &s)) return QPAT_FP64;
  if (ctx_tables32(c, &y, &lossless, &s)) return QPAT_FP32;
  return -1;
}

}  // namespace

extern "C" qpat_status qpat_jvp_medium(qpat_ctx* ctx, const double* p0, const double* dc, const double* drho,
                                       double* dP) {
  if (!ctx) return QPAT_EINVAL;
  if (!p0 || !dP) return (qpat_status)ctx_fail(ctx, QPAT_EINVAL, "qpat_jvp_medium: p0 and dP are required");
  return sweep_precision(ctx) == QPAT_FP32 ? jvp_medium<float>(ctx, p0, dc, drho, dP)
                                           : jvp_medium<double>(ctx, p0, dc, drho, dP);
}

extern "C" qpat_status qpat_vjp_medium(qpat_ctx* ctx, const double* p0, const double* wts, double* g_c,
                                       double* g_rho) {
  if (!ctx) return QPAT_EINVAL;
  if (!p0 || !wts) return (qpat_status)ctx_fail(ctx, QPAT_EINVAL, "qpat_vjp_medium: p0 and w are required");
  return sweep_precision(ctx) == QPAT_FP32 ? vjp_medium<float>(ctx, p0, wts, g_c, g_rho)
                                           : vjp_medium<double>(ctx, p0, wts, g_c, g_rho);
}
