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
// Index of a pair of complex values (16 bytes) with one pair of padding per 8.
__device__ __forceinline__ int spad2(int n) { return n + (n >> 3); }
// Complex values per sequence in the Stockham buffers: room for either layout
// (a sequence pair takes two sequences' room), rounded up to an even count so
// that every pair starts on a 16-byte boundary.
__host__ __device__ constexpr int spad_size(int L) { return (L + (L >> 3) + 2) & ~1; }

// ---- packed FP32 pairs (sm_100 family FADD2 / FMUL2 / FFMA2) -----------------
// F2 holds one FP32 value of each of two independent sequences; P2 holds a
// complex value of each (real parts in x, imaginary parts in y), so that the
// butterflies of two sequences run as one stream of packed instructions.
// Products are kept lazy (F2Mul) so that a product added to or subtracted from
// a value becomes one fused multiply-add, rounded once, like the scalar
// contraction the compiler applies to the float2 code.
struct F2 {
  float2 v;
  F2() = default;
  __device__ __forceinline__ explicit F2(float2 w) : v(w) {}
  __device__ __forceinline__ F2(float s) : v(make_float2(s, s)) {}
  __device__ __forceinline__ F2(float a, float b) : v(make_float2(a, b)) {}
};
struct F2Mul {
  F2 a, b;
  __device__ __forceinline__ operator F2() const { return F2(__fmul2_rn(a.v, b.v)); }
};
__device__ __forceinline__ F2 operator-(F2 a) { return F2(make_float2(-a.v.x, -a.v.y)); }
__device__ __forceinline__ F2 operator+(F2 a, F2 b) { return F2(__fadd2_rn(a.v, b.v)); }
__device__ __forceinline__ F2 operator-(F2 a, F2 b) { return F2(__fadd2_rn(a.v, (-b).v)); }
__device__ __forceinline__ F2Mul operator*(F2 a, F2 b) { return F2Mul{a, b}; }
__device__ __forceinline__ F2Mul operator-(F2Mul p) { return F2Mul{-p.a, p.b}; }
__device__ __forceinline__ F2 operator+(F2 c, F2Mul p) { return F2(__ffma2_rn(p.a.v, p.b.v, c.v)); }
__device__ __forceinline__ F2 operator+(F2Mul p, F2 c) { return F2(__ffma2_rn(p.a.v, p.b.v, c.v)); }
__device__ __forceinline__ F2 operator-(F2 c, F2Mul p) { return F2(__ffma2_rn((-p.a).v, p.b.v, c.v)); }
__device__ __forceinline__ F2 operator-(F2Mul p, F2 c) { return F2(__ffma2_rn(p.a.v, p.b.v, (-c).v)); }
__device__ __forceinline__ F2 operator+(F2Mul p, F2Mul q) { return p + F2(q); }
__device__ __forceinline__ F2 operator-(F2Mul p, F2Mul q) { return F2(p) - q; }
__device__ __forceinline__ F2& operator+=(F2& c, F2Mul p) { return c = c + p; }
__device__ __forceinline__ F2& operator+=(F2& c, F2 p) { return c = c + p; }

struct P2 {
  F2 x, y;
};
__device__ __forceinline__ P2 pack2(float2 a, float2 b) { return P2{F2(a.x, b.x), F2(a.y, b.y)}; }
__device__ __forceinline__ float2 lane0(P2 p) { return make_float2(p.x.v.x, p.y.v.x); }
__device__ __forceinline__ float2 lane1(P2 p) { return make_float2(p.x.v.y, p.y.v.y); }
// p times the complex scalar w (the same twiddle for both sequences)
__device__ __forceinline__ P2 cmul(P2 p, float2 w) {
  const F2 wx(w.x), wy(w.y);
  return P2{p.x * wx - p.y * wy, p.x * wy + p.y * wx};
}
__device__ __forceinline__ float4 p2_bits(P2 p) { return make_float4(p.x.v.x, p.x.v.y, p.y.v.x, p.y.v.y); }
__device__ __forceinline__ P2 p2_from(float4 f) { return P2{F2(f.x, f.y), F2(f.z, f.w)}; }

#ifndef QPAT_FFT_PAIRS
#define QPAT_FFT_PAIRS 1
#endif

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

// butterfly() for NP sequence pairs.
template <int L, int R, int Ns, int NP>
__device__ __forceinline__ void butterfly2(P2 (&a)[NP][R], int j, const float2* __restrict__ tw) {
  if constexpr (Ns > 1) {
    constexpr int step = L / (Ns * R);
    const int k = j % Ns;
#pragma unroll
    for (int r = 1; r < R; ++r) {
      const float2 w = tw[k * r * step];
#pragma unroll
      for (int q = 0; q < NP; ++q) a[q][r] = cmul(a[q][r], w);
    }
  }
#pragma unroll
  for (int q = 0; q < NP; ++q) dft<R>(a[q]);
}

// Stage I/O of the paired transform: sequence pairs q as 16-byte entries at
// buf + 2 q sl (index spad2), an odd last sequence as complex values at
// buf + (NS - 1) sl (index spad).
template <int NS, int R, int NP>
__device__ __forceinline__ void st_store(float2* buf, int sl, const P2 (&p)[NP][R], const float2 (&o)[1][R],
                                         int pos0, int dpos) {
#pragma unroll
  for (int q = 0; q < NP; ++q) {
    float4* B = reinterpret_cast<float4*>(buf + 2 * q * sl);
#pragma unroll
    for (int r = 0; r < R; ++r) B[spad2(pos0 + r * dpos)] = p2_bits(p[q][r]);
  }
  if constexpr (NS % 2 == 1) {
#pragma unroll
    for (int r = 0; r < R; ++r) buf[(NS - 1) * sl + spad(pos0 + r * dpos)] = o[0][r];
  }
}
template <int NS, int R, int NP>
__device__ __forceinline__ void st_load(const float2* buf, int sl, P2 (&p)[NP][R], float2 (&o)[1][R], int pos0,
                                        int dpos) {
#pragma unroll
  for (int q = 0; q < NP; ++q) {
    const float4* B = reinterpret_cast<const float4*>(buf + 2 * q * sl);
#pragma unroll
    for (int r = 0; r < R; ++r) p[q][r] = p2_from(B[spad2(pos0 + r * dpos)]);
  }
  if constexpr (NS % 2 == 1) {
#pragma unroll
    for (int r = 0; r < R; ++r) o[0][r] = buf[(NS - 1) * sl + spad(pos0 + r * dpos)];
  }
}

// fft_stockham for NS >= 2 FP32 sequences: pairs of sequences run as packed
// FP32x2 arithmetic, an odd last sequence as complex float2 values.
template <int L, int Q1, int Q2, int Q3, int NS, bool ONEBUF>
__device__ __forceinline__ void fft_stockham_pairs(float2 (&a1)[NS][Q1], float2 (&a3)[NS][(Q3 > 1 ? Q3 : Q2)],
                                                   float2* bufA, float2* bufB, int sl, int j,
                                                   const float2* __restrict__ tw) {
  constexpr int NP = NS / 2, QL = (Q3 > 1 ? Q3 : Q2);
  constexpr bool ODD = NS % 2 == 1;
  P2 p1[NP][Q1];
  float2 o1[1][Q1];
  if (j < L / Q1) {
#pragma unroll
    for (int q = 0; q < NP; ++q)
#pragma unroll
      for (int r = 0; r < Q1; ++r) p1[q][r] = pack2(a1[2 * q][r], a1[2 * q + 1][r]);
    butterfly2<L, Q1, 1, NP>(p1, j, tw);
    if constexpr (ODD) {
#pragma unroll
      for (int r = 0; r < Q1; ++r) o1[0][r] = a1[NS - 1][r];
      butterfly<L, Q1, 1, 1>(o1, j, tw);
    }
    st_store<NS, Q1, NP>(bufA, sl, p1, o1, stockham_pos<Q1, 1>(j, 0), 1);
  }
  __syncthreads();
  P2 p3[NP][QL];
  float2 o3[1][QL];
  if constexpr (Q3 == 1) {
    if (j < L / Q2) {
      st_load<NS, Q2, NP>(bufA, sl, p3, o3, j, L / Q2);
      butterfly2<L, Q2, Q1, NP>(p3, j, tw);
      if constexpr (ODD) butterfly<L, Q2, Q1, 1>(o3, j, tw);
    }
  } else {
    P2 p2[NP][Q2];
    float2 o2[1][Q2];
    if (j < L / Q2) {
      st_load<NS, Q2, NP>(bufA, sl, p2, o2, j, L / Q2);
      butterfly2<L, Q2, Q1, NP>(p2, j, tw);
      if constexpr (ODD) butterfly<L, Q2, Q1, 1>(o2, j, tw);
    }
    if constexpr (ONEBUF) __syncthreads();
    if (j < L / Q2) st_store<NS, Q2, NP>(bufB, sl, p2, o2, stockham_pos<Q2, Q1>(j, 0), Q1);
    __syncthreads();
    if (j < L / Q3) {
      st_load<NS, Q3, NP>(bufB, sl, p3, o3, j, L / Q3);
      butterfly2<L, Q3, Q1 * Q2, NP>(p3, j, tw);
      if constexpr (ODD) butterfly<L, Q3, Q1 * Q2, 1>(o3, j, tw);
    }
  }
  if (j < L / QL) {
#pragma unroll
    for (int q = 0; q < NP; ++q)
#pragma unroll
      for (int r = 0; r < QL; ++r) {
        a3[2 * q][r] = lane0(p3[q][r]);
        a3[2 * q + 1][r] = lane1(p3[q][r]);
      }
    if constexpr (ODD) {
#pragma unroll
      for (int r = 0; r < QL; ++r) a3[NS - 1][r] = o3[0][r];
    }
  }
  __syncthreads();
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
template <int L, int Q1, int Q2, int Q3, int NS, bool ONEBUF = false, bool PAIRS = true, typename C>
__device__ __forceinline__ void fft_stockham(C (&a1)[NS][Q1], C (&a3)[NS][(Q3 > 1 ? Q3 : Q2)], C* bufA, C* bufB,
                                             int sl, int j, const C* __restrict__ tw) {
  static_assert(Q1 * Q2 * Q3 == L, "radices must multiply to L");
  if constexpr (PAIRS && QPAT_FFT_PAIRS && NS >= 2 && std::is_same<C, float2>::value) {
    fft_stockham_pairs<L, Q1, Q2, Q3, NS, ONEBUF>(a1, a3, bufA, bufB, sl, j, tw);
    return;
  }
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
