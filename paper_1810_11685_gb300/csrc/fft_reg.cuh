// Register-resident FFTs of compile-time length (sm_103a).
//
// A length-L transform with L = A * B is split Cooley-Tukey style over a
// group of max(A, B) threads:
//
//   X[k1 + A k2] = sum_n2 W_L^(n2 k1) W_B^(n2 k2) sum_n1 x[B n1 + n2] W_A^(n1 k1)
//
// Thread l < B holds x[B n1 + l] (n1 < A) in registers and does the A-point
// DFT there; after the twiddle W_L^(l k1) the values are exchanged once
// through shared memory, and thread l' < A does the B-point DFT over n2 and
// ends holding X[l' + A k2] (k2 < B).  The A- and B-point DFTs themselves
// are fully unrolled mixed-radix (2, 3, 4, 5, 7, 8) Cooley-Tukey recursions
// whose twiddles are compile-time constants, computed by constexpr Taylor
// series in double precision.  The inter-thread twiddles W_L^(l k1) come from
// a device table built in FP64 (see tables.cu).
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

// Shared-memory strides of the exchange: an odd row stride, and a per-
// sequence size congruent to 2 mod 8 complex values, keep the 8-byte
// accesses of a half warp on distinct banks for the thread layouts used.
template <int A, int B>
struct XLayout {
  static constexpr int SB = B + ((B % 2 == 0) ? 1 : 0);    // row stride of the [A][SB] tile
  static constexpr int raw = A * SB;
  static constexpr int XS = raw + ((2 - raw % 8) + 8) % 8;  // per-sequence size, == 2 mod 8
};

// Cooperative length-A*B forward FFT of NS sequences by one thread group.
// In:  thread l < B holds in[s][n1] = x_s[B n1 + l], n1 < A.
// Out: thread l < A holds out[s][k2] = X_s[l + A k2], k2 < B.
// ex:  the group's exchange area, NS * XLayout<A,B>::XS complex values (the
//      stride between sequences is `xs`); tw: W_L^(l k1) at tw[k1 * B + l].
// All threads of the CTA must call it (it contains __syncthreads).
template <int A, int B, int NS, typename C>
__device__ __forceinline__ void fft_group(C (&in)[NS][A], C (&out)[NS][B], C* ex, int xs, const C* __restrict__ tw,
                                          int l) {
  constexpr int SB = XLayout<A, B>::SB;
  if (l < B) {
#pragma unroll
    for (int s = 0; s < NS; ++s) dft<A>(in[s]);
#pragma unroll
    for (int k1 = 1; k1 < A; ++k1) {
      const C w = tw[k1 * B + l];
#pragma unroll
      for (int s = 0; s < NS; ++s) in[s][k1] = cmul(in[s][k1], w);
    }
#pragma unroll
    for (int s = 0; s < NS; ++s)
#pragma unroll
      for (int k1 = 0; k1 < A; ++k1) ex[s * xs + k1 * SB + l] = in[s][k1];
  }
  __syncthreads();
  if (l < A) {
#pragma unroll
    for (int s = 0; s < NS; ++s) {
#pragma unroll
      for (int n2 = 0; n2 < B; ++n2) out[s][n2] = ex[s * xs + l * SB + n2];
      dft<B>(out[s]);
    }
  }
  __syncthreads();
}

}  // namespace qpat
