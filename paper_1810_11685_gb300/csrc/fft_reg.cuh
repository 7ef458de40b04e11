// Compile-time Stockham FFTs with register end points (sm_103a).
//
// A length-L transform with L = Q1 * Q2 [* Q3] runs on a group of
// TPT = L / min(Q) threads.  In stage s of radix R (stride Ns = product of the
// earlier radices) thread j < L/R holds the R values x[j + r L/R] in
// registers, multiplies them by W_L^{(j mod Ns) r L/(Ns R)}, performs an
// R-point DFT, and the results go to position (j/Ns) Ns R + (j mod Ns) + r Ns
// (Stockham self-sorting order).  Between stages the values pass through
// shared memory; the first stage starts from registers (loaded straight from
// global memory) and the last stage leaves them in registers, thread j
// holding X[j + r L/Q_last].  The R-point DFTs are fully unrolled mixed-radix
// Cooley-Tukey recursions whose twiddles are compile-time constants
// (constexpr Taylor series in double precision); the stage twiddles come
// from a W_L^m table built in FP64 on the device.
#pragma once
#include <type_traits>

#include "fft_smem.cuh"

namespace qpat {

// ---- compile-time trigonometry ---------------------------------------------
constexpr double kPi = 3.141592653589793238462643383279502884;

// sin and cos of 2 pi p / q by Taylor series after reducing the angle to
// [-pi, pi] (40 terms: the remainder is far below double rounding there).
constexpr double taylor_sin(double x) {
  double term = x, sum = x;
  for (int n = 1; n < 40; ++n) {
    term *= -x * x / ((2.0 * n) * (2.0 * n + 1.0));
    sum += term;
  }
  return sum;
}
constexpr double taylor_cos(double x) {
  double term = 1.0, sum = 1.0;
  for (int n = 1; n < 40; ++n) {
    term *= -x * x / ((2.0 * n - 1.0) * (2.0 * n));
    sum += term;
  }
  return sum;
}
constexpr double angle_2pi(long p, long q) {
  long r = ((p % q) + q) % q;           // 0 <= r < q
  if (2 * r > q) r -= q;                // -q/2 < r <= q/2
  return 2.0 * kPi * (double)r / (double)q;
}
constexpr double cos2pi(long p, long q) { return taylor_cos(angle_2pi(p, q)); }
constexpr double sin2pi(long p, long q) { return taylor_sin(angle_2pi(p, q)); }

template <int Begin, int End, typename F>
__device__ __forceinline__ void static_for(F&& f) {
  if constexpr (Begin < End) {
    f(std::integral_constant<int, Begin>{});
    static_for<Begin + 1, End>(f);
  }
}

constexpr int first_factor(int N) {
  return (N % 8 == 0 && N != 8) ? 8
       : (N % 4 == 0 && N != 4) ? 4
       : (N % 2 == 0 && N != 2) ? 2
       : (N % 3 == 0 && N != 3) ? 3
       : (N % 5 == 0 && N != 5) ? 5
       : (N % 7 == 0 && N != 7) ? 7 : N;
}

// In-place forward DFT of a[0..N-1] held in registers, natural order in and out.
template <int N, typename C>
__device__ __forceinline__ void dft(C (&a)[N]) {
  typedef decltype(C().x) R;
  if constexpr (N == 1) {
  } else if constexpr (N == 2) { dft2(a);
  } else if constexpr (N == 3) { dft3(a);
  } else if constexpr (N == 4) { dft4(a);
  } else if constexpr (N == 5) { dft5(a);
  } else if constexpr (N == 7) { dft7(a);
  } else if constexpr (N == 8) { dft8(a);
  } else {
    constexpr int P = first_factor(N);
    constexpr int M = N / P;
    static_assert(P > 1 && P < N, "DFT length must factor into 2, 3, 5, 7");
    C y[M][P];
    // P-point DFTs over n1 of x[M n1 + n2]
#pragma unroll
    for (int n2 = 0; n2 < M; ++n2) {
      C t[P];
#pragma unroll
      for (int n1 = 0; n1 < P; ++n1) t[n1] = a[M * n1 + n2];
      dft<P>(t);
#pragma unroll
      for (int k1 = 0; k1 < P; ++k1) y[n2][k1] = t[k1];
    }
    // twiddles W_N^(n2 k1), compile-time constants
    static_for<1, M>([&](auto n2c) {
      constexpr int n2 = decltype(n2c)::value;
      static_for<1, P>([&](auto k1c) {
        constexpr int k1 = decltype(k1c)::value;
        constexpr double c = cos2pi(n2 * k1, N);
        constexpr double s = sin2pi(n2 * k1, N);
        y[n2][k1] = cmul(y[n2][k1], cmake<C>((R)c, (R)(-s)));
      });
    });
    // M-point DFTs over n2; output index k1 + P k2
#pragma unroll
    for (int k1 = 0; k1 < P; ++k1) {
      C u[M];
#pragma unroll
      for (int n2 = 0; n2 < M; ++n2) u[n2] = y[n2][k1];
      dft<M>(u);
#pragma unroll
      for (int k2 = 0; k2 < M; ++k2) a[k1 + P * k2] = u[k2];
    }
  }
}

// Shared-memory index with one complex of padding per 16, so that the
// strided Stockham stores of a half warp spread over the banks.
__device__ __forceinline__ int spad(int n) { return n + (n >> 4); }
__host__ __device__ constexpr int spad_size(int L) { return L + (L >> 4) + 1; }

// Twiddle and DFT of one radix-R butterfly of a stage with stride Ns, for NS
// sequences at once.  a[s][r] = x_s[j + r L/R] on entry, the butterfly's
// outputs (for positions (j/Ns) Ns R + (j mod Ns) + r Ns) on exit.
template <int L, int R, int Ns, int NS, typename C>
__device__ __forceinline__ void butterfly(C (&a)[NS][R], int j, const C* __restrict__ tw) {
  if constexpr (Ns > 1) {
    constexpr int step = L / (Ns * R);
    const int k = j % Ns;
#pragma unroll
    for (int r = 1; r < R; ++r) {
      const C w = tw[k * r * step];          // exponent < L, no reduction needed
#pragma unroll
      for (int s = 0; s < NS; ++s) a[s][r] = cmul(a[s][r], w);
    }
  }
#pragma unroll
  for (int s = 0; s < NS; ++s) dft<R>(a[s]);
}

template <int R, int Ns>
__device__ __forceinline__ int stockham_pos(int j, int r) {
  return (j / Ns) * Ns * R + (j % Ns) + r * Ns;
}

// Forward FFT of NS sequences of length L = Q1 Q2 Q3 (Q3 = 1: two stages) by
// the thread group; j is the thread's index in the group.
// in:  a1[s][r] = x_s[j + r L/Q1] for j < L/Q1 (others ignored)
// out: a3[s][r] = X_s[j + r L/Qlast] for j < L/Qlast
// bufA, bufB: NS * spad_size(L) complex each, sequences `sl` apart.
// Every thread of the CTA must call it (it synchronises the CTA).
// ONEBUF: bufB may alias bufA; the middle stage of a three-stage plan then
// waits for every thread's reads before its writes (one more barrier, half
// the shared memory).
template <int L, int Q1, int Q2, int Q3, int NS, bool ONEBUF = false, typename C>
__device__ __forceinline__ void fft_stockham(C (&a1)[NS][Q1], C (&a3)[NS][(Q3 > 1 ? Q3 : Q2)], C* bufA, C* bufB,
                                             int sl, int j, const C* __restrict__ tw) {
  static_assert(Q1 * Q2 * Q3 == L, "radices must multiply to L");
  if (j < L / Q1) {
    butterfly<L, Q1, 1, NS>(a1, j, tw);
#pragma unroll
    for (int s = 0; s < NS; ++s)
#pragma unroll
      for (int r = 0; r < Q1; ++r) bufA[s * sl + spad(stockham_pos<Q1, 1>(j, r))] = a1[s][r];
  }
  __syncthreads();
  if constexpr (Q3 == 1) {
    if (j < L / Q2) {
#pragma unroll
      for (int s = 0; s < NS; ++s)
#pragma unroll
        for (int r = 0; r < Q2; ++r) a3[s][r] = bufA[s * sl + spad(j + r * (L / Q2))];
      butterfly<L, Q2, Q1, NS>(a3, j, tw);
    }
  } else if constexpr (ONEBUF) {
    C a2[NS][Q2];
    if (j < L / Q2) {
#pragma unroll
      for (int s = 0; s < NS; ++s)
#pragma unroll
        for (int r = 0; r < Q2; ++r) a2[s][r] = bufA[s * sl + spad(j + r * (L / Q2))];
      butterfly<L, Q2, Q1, NS>(a2, j, tw);
    }
    __syncthreads();
    if (j < L / Q2) {
#pragma unroll
      for (int s = 0; s < NS; ++s)
#pragma unroll
        for (int r = 0; r < Q2; ++r) bufB[s * sl + spad(stockham_pos<Q2, Q1>(j, r))] = a2[s][r];
    }
    __syncthreads();
    if (j < L / Q3) {
#pragma unroll
      for (int s = 0; s < NS; ++s)
#pragma unroll
        for (int r = 0; r < Q3; ++r) a3[s][r] = bufB[s * sl + spad(j + r * (L / Q3))];
      butterfly<L, Q3, Q1 * Q2, NS>(a3, j, tw);
    }
  } else {
    if (j < L / Q2) {
      C a2[NS][Q2];
#pragma unroll
      for (int s = 0; s < NS; ++s)
#pragma unroll
        for (int r = 0; r < Q2; ++r) a2[s][r] = bufA[s * sl + spad(j + r * (L / Q2))];
      butterfly<L, Q2, Q1, NS>(a2, j, tw);
#pragma unroll
      for (int s = 0; s < NS; ++s)
#pragma unroll
        for (int r = 0; r < Q2; ++r) bufB[s * sl + spad(stockham_pos<Q2, Q1>(j, r))] = a2[s][r];
    }
    __syncthreads();
    if (j < L / Q3) {
#pragma unroll
      for (int s = 0; s < NS; ++s)
#pragma unroll
        for (int r = 0; r < Q3; ++r) a3[s][r] = bufB[s * sl + spad(j + r * (L / Q3))];
      butterfly<L, Q3, Q1 * Q2, NS>(a3, j, tw);
    }
  }
  __syncthreads();
}

}  // namespace qpat
