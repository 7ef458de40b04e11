// Length-specialised propagation passes on the register-resident FFT.
//
// Row pass (one thread group per pair of grid rows j0, j0+1):
//   load the incoming half spectra, Hermitian-extend them and pack the two
//   rows into one complex sequence (stride-B layout) -> inverse x-FFT via
//   conj(FFT(conj .)) -> every thread now owns grid points l + A k2 of both
//   rows in registers -> pointwise update (row_point) -> forward x-FFT of the
//   packed outgoing fields (its stride-A input layout is exactly what the
//   thread holds) -> split into two half spectra through shared memory.
// Column pass (one thread group per half-spectrum column, CBW adjacent
//   columns per CTA so that global accesses are contiguous):
//   load a column (stride-B layout) -> forward y-FFT -> spectral symbol
//   (col_point) on the registers -> inverse y-FFT (stride-A input layout) ->
//   store in the original layout.
// Each transform touches shared memory once (one exchange), against one
// round trip per radix stage in the generic kernels.
#pragma once
#include "fft_reg.cuh"
#include "pass_ops.cuh"

namespace qpat {

template <int A, int B>
struct FastGeom {
  static constexpr int L = A * B;
  static constexpr int TPT = A > B ? A : B;
  static constexpr int XAB = XLayout<A, B>::XS;
  static constexpr int XBA = XLayout<B, A>::XS;
  static constexpr int XS = XAB > XBA ? XAB : XBA;        // per-slot exchange size (>= L)
  static constexpr int RP = (128 / TPT) > 0 ? (128 / TPT) : 1;                       // row pairs per CTA
  static constexpr int CBW = (128 / TPT) >= 8 ? 8 : 4;                               // columns per CTA
};

template <typename T, int A, int B, int KIN, int KOUT>
__global__ void __launch_bounds__(FastGeom<A, B>::RP * FastGeom<A, B>::TPT)
row_fast(const PropArgs<T> a, const int ph) {
  typedef typename V2<T>::t C;
  typedef FastGeom<A, B> G;
  constexpr int L = G::L, TPT = G::TPT, XS = G::XS, RP = G::RP;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int m = threadIdx.x / TPT;
  const int l = threadIdx.x - m * TPT;
  C* ex = reinterpret_cast<C*>(smem_raw) + m * 2 * XS;
  T* sc = reinterpret_cast<T*>(reinterpret_cast<C*>(smem_raw) + RP * 2 * XS) + m * 2 * L;
  const int b = blockIdx.y;
  const int jp = blockIdx.x * RP + m;
  const bool valid = jp < (a.ny >> 1);
  const int j0 = valid ? 2 * jp : 0;
  C* spec = a.spec + (long long)b * a.sstride;
  const long long slot = (long long)a.ny * a.pitch;
  const bool skip_in = (a.flags & kSkipInput) != 0;

  // 1. inverse x-transform of the incoming half spectra
  C y[KIN][B];
  if (!skip_in) {
    C v[KIN][A];
    if (l < B) {
#pragma unroll
      for (int s = 0; s < KIN; ++s) {
        const C* r0 = spec + s * slot + (long long)j0 * a.pitch;
        const C* r1 = r0 + a.pitch;
#pragma unroll
        for (int n1 = 0; n1 < A; ++n1) {
          const int n = B * n1 + l;
          C P, Q;
          if (2 * n <= L) {
            P = r0[n];
            Q = r1[n];
            if (n == 0 || 2 * n == L) { P.y = (T)0; Q.y = (T)0; }
          } else {
            P = cconj(r0[L - n]);
            Q = cconj(r1[L - n]);
          }
          v[s][n1] = cmake<C>(P.x - Q.y, -(P.y + Q.x));   // conj(P + i Q)
        }
      }
    }
    fft_group<A, B, KIN>(v, y, ex, XS, a.fx_ab, l);
  } else {
#pragma unroll
    for (int s = 0; s < KIN; ++s)
#pragma unroll
      for (int k = 0; k < B; ++k) y[s][k] = cmake<C>((T)0, (T)0);
  }

  // adjoint sensor source M^T w_n on the two rows (A_R1, A_R1L)
  if (KIN == 1) {
    for (int i = l; i < 2 * L; i += TPT) sc[i] = (T)0;
    __syncthreads();
    if (valid) sensor_scatter_rows<T>(a, b, j0, sc, l, TPT);
    __syncthreads();
  }

  // 2. pointwise update on the grid points this thread owns: i = l + A k2
  C o[KOUT][B];
  bool bad = false;
#pragma unroll
  for (int k2 = 0; k2 < B; ++k2) {
    T r0v[2] = {(T)0, (T)0}, r1v[2] = {(T)0, (T)0};
    if (l < A && valid) {
      const int i = l + A * k2;
#pragma unroll
      for (int rr = 0; rr < 2; ++rr) {
        const T in0 = rr ? -y[0][k2].y : y[0][k2].x;
        const T in1 = (KIN > 1) ? (rr ? -y[KIN - 1][k2].y : y[KIN - 1][k2].x) : (T)0;
        const T scv = (KIN == 1) ? sc[rr * L + i] : (T)0;
        T out0, out1;
        row_point<T>(a, ph, b, i, j0 + rr, in0, in1, scv, out0, out1, bad);
        r0v[rr] = out0;
        r1v[rr] = out1;
      }
    }
    o[0][k2] = cmake<C>(r0v[0], r0v[1]);
    if (KOUT > 1) o[KOUT - 1][k2] = cmake<C>(r1v[0], r1v[1]);
  }
  if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr(a.err, 1);
  if (a.flags & kSkipOutput) return;

  // 3. forward x-transform of the packed outgoing rows (stride-A layout)
  C X[KOUT][A];
  fft_group<B, A, KOUT>(o, X, ex, XS, a.fx_ba, l);
  // thread l < B holds Z[l + B k] for k < A; split Z into the two rows'
  // half spectra A(k) = (Z(k) + conj Z(-k))/2, B(k) = -i (Z(k) - conj Z(-k))/2
  if (l < B) {
#pragma unroll
    for (int s = 0; s < KOUT; ++s)
#pragma unroll
      for (int k = 0; k < A; ++k) ex[s * XS + l + B * k] = X[s][k];
  }
  __syncthreads();
  if (valid) {
#pragma unroll
    for (int s = 0; s < KOUT; ++s) {
      C* w0 = spec + s * slot + (long long)j0 * a.pitch;
      C* w1 = w0 + a.pitch;
      for (int k = l; 2 * k <= L; k += TPT) {
        const C Z = ex[s * XS + k];
        const C Zm = cconj(ex[s * XS + (k == 0 ? 0 : L - k)]);
        w0[k] = cscale(cadd(Z, Zm), (T)0.5);
        w1[k] = cscale(cmul_mi(csub(Z, Zm)), (T)0.5);
      }
    }
  }
}

template <typename T, int A, int B, int KIN, int KOUT>
__global__ void __launch_bounds__(FastGeom<A, B>::CBW * FastGeom<A, B>::TPT)
col_fast(const PropArgs<T> a, const int ph) {
  typedef typename V2<T>::t C;
  typedef FastGeom<A, B> G;
  constexpr int XS = G::XS, CBW = G::CBW;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int c = threadIdx.x % CBW;
  const int l = threadIdx.x / CBW;
  C* ex = reinterpret_cast<C*>(smem_raw) + c * 2 * XS;
  const int b = blockIdx.y;
  const int kx = blockIdx.x * CBW + c;
  const bool valid = kx < a.nxh;
  const int kxs = valid ? kx : 0;
  C* spec = a.spec + (long long)b * a.sstride;
  const long long slot = (long long)a.ny * a.pitch;

  if (ph == F_C1) sensor_gather<T>(a, b, blockIdx.x * blockDim.x + threadIdx.x, gridDim.x * blockDim.x);

  C v[KIN][A];
  if (l < B) {
#pragma unroll
    for (int s = 0; s < KIN; ++s)
#pragma unroll
      for (int n1 = 0; n1 < A; ++n1) v[s][n1] = spec[s * slot + (long long)(B * n1 + l) * a.pitch + kxs];
  }
  C X[KIN][B];
  fft_group<A, B, KIN>(v, X, ex, XS, a.fy_ab, l);
  // thread l < A holds X[ky = l + A k2]
  C o[KOUT][B];
#pragma unroll
  for (int k2 = 0; k2 < B; ++k2) {
    C o0 = cmake<C>((T)0, (T)0), o1 = o0;
    if (l < A && valid) col_point<T, C>(a, ph, kx, l + A * k2, X[0][k2], X[KIN - 1][k2], o0, o1);
    o[0][k2] = cconj(o0);
    if (KOUT > 1) o[KOUT - 1][k2] = cconj(o1);
  }
  C Y[KOUT][A];
  fft_group<B, A, KOUT>(o, Y, ex, XS, a.fy_ba, l);
  // thread l < B holds the inverse at rows l + B k
  if (l < B && valid) {
#pragma unroll
    for (int s = 0; s < KOUT; ++s)
#pragma unroll
      for (int k = 0; k < A; ++k) spec[s * slot + (long long)(l + B * k) * a.pitch + kx] = cconj(Y[s][k]);
  }
}

template <typename T, int A, int B, int KIN, int KOUT>
void run_row_fast(const PropArgs<T>& a, int ph, int batch, cudaStream_t s) {
  typedef FastGeom<A, B> G;
  typedef typename V2<T>::t C;
  const size_t sm = G::RP * 2 * G::XS * sizeof(C) + (KIN == 1 ? G::RP * 2 * G::L * sizeof(T) : 0);
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(row_fast<T, A, B, KIN, KOUT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    attr = true;
  }
  dim3 grid((a.ny / 2 + G::RP - 1) / G::RP, batch);
  row_fast<T, A, B, KIN, KOUT><<<grid, G::RP * G::TPT, sm, s>>>(a, ph);
}

template <typename T, int A, int B, int KIN, int KOUT>
void run_col_fast(const PropArgs<T>& a, int ph, int batch, cudaStream_t s) {
  typedef FastGeom<A, B> G;
  typedef typename V2<T>::t C;
  const size_t sm = G::CBW * 2 * G::XS * sizeof(C);
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(col_fast<T, A, B, KIN, KOUT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    attr = true;
  }
  dim3 grid((a.nxh + G::CBW - 1) / G::CBW, batch);
  col_fast<T, A, B, KIN, KOUT><<<grid, G::CBW * G::TPT, sm, s>>>(a, ph);
}

// Entry points of one specialised length L (one translation unit each).
template <typename T, int L>
void launch_row_fast_len(const PropArgs<T>& a, int ph, int batch, cudaStream_t s) {
  constexpr int A = fast_split_a(L), B = L / (A > 0 ? A : 1);
  const int kin = row_kin(ph), kout = row_kout(ph);
  if (kin == 2 && kout == 2) run_row_fast<T, A, B, 2, 2>(a, ph, batch, s);
  else if (kin == 2) run_row_fast<T, A, B, 2, 1>(a, ph, batch, s);
  else run_row_fast<T, A, B, 1, 2>(a, ph, batch, s);
}

template <typename T, int L>
void launch_col_fast_len(const PropArgs<T>& a, int ph, int batch, cudaStream_t s) {
  constexpr int A = fast_split_a(L), B = L / (A > 0 ? A : 1);
  const int kin = col_kin(ph), kout = col_kout(ph);
  if (kin == 2 && kout == 2) run_col_fast<T, A, B, 2, 2>(a, ph, batch, s);
  else if (kin == 1) run_col_fast<T, A, B, 1, 2>(a, ph, batch, s);
  else run_col_fast<T, A, B, 2, 1>(a, ph, batch, s);
}

#define QPAT_FAST_LENGTH(L)                                                                              \
  template void launch_row_fast_len<float, L>(const PropArgs<float>&, int, int, cudaStream_t);         \
  template void launch_row_fast_len<double, L>(const PropArgs<double>&, int, int, cudaStream_t);       \
  template void launch_col_fast_len<float, L>(const PropArgs<float>&, int, int, cudaStream_t);         \
  template void launch_col_fast_len<double, L>(const PropArgs<double>&, int, int, cudaStream_t);

}  // namespace qpat
