// Batched mixed-radix Stockham FFT in shared memory (sm_103a).
//
// A CTA transforms M sequences of length L held contiguously in shared
// memory (sequence m at offset m*L).  Each stage with radix R reads R points
// at stride L/R, applies the twiddles W_{Ns R}^(k r) and an R-point DFT, and
// writes them self-sorted (Stockham autosort), so the result comes out in
// natural order after ping-ponging between two buffers.  Radices 2, 3, 4, 5,
// 7 and 8 are written out by hand.  The transform is the forward DFT
// X_k = sum_n x_n exp(-2 pi i n k / L), unnormalised; inverse transforms use
// conj(FFT(conj(.))).  Twiddles come from a table W_L^m, m = 0..L-1,
// computed in FP64 on the device and rounded to the working precision.
#pragma once
#include <cuda_runtime.h>

namespace qpat {

template <typename T> struct V2;
template <> struct V2<float> { typedef float2 t; };
template <> struct V2<double> { typedef double2 t; };

template <typename C> __device__ __forceinline__ C cmake(decltype(C().x) a, decltype(C().x) b) {
  C r; r.x = a; r.y = b; return r;
}
template <typename C> __device__ __forceinline__ C cadd(C a, C b) { return cmake<C>(a.x + b.x, a.y + b.y); }
template <typename C> __device__ __forceinline__ C csub(C a, C b) { return cmake<C>(a.x - b.x, a.y - b.y); }
template <typename C> __device__ __forceinline__ C cmul(C a, C b) {
  return cmake<C>(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
template <typename C> __device__ __forceinline__ C cconj(C a) { return cmake<C>(a.x, -a.y); }
template <typename C> __device__ __forceinline__ C cscale(C a, decltype(C().x) s) { return cmake<C>(a.x * s, a.y * s); }
// multiply by -i
template <typename C> __device__ __forceinline__ C cmul_mi(C a) { return cmake<C>(a.y, -a.x); }
// multiply by +i
template <typename C> __device__ __forceinline__ C cmul_pi(C a) { return cmake<C>(-a.y, a.x); }

constexpr int kMaxStages = 12;

struct FFTPlan {
  int L;                   // length
  int nstages;
  int radix[kMaxStages];   // radix of each stage, product = L
};

// ---- small DFT kernels (forward sign) --------------------------------------

template <typename C> __device__ __forceinline__ void dft2(C* a) {
  C t = a[0];
  a[0] = cadd(t, a[1]);
  a[1] = csub(t, a[1]);
}

template <typename C> __device__ __forceinline__ void dft3(C* a) {
  typedef decltype(C().x) R;
  const R h = (R)0.8660254037844386467637231707529362;   // sqrt(3)/2
  C t1 = cadd(a[1], a[2]);
  C t2 = csub(a[1], a[2]);
  C m = cmake<C>(a[0].x - (R)0.5 * t1.x, a[0].y - (R)0.5 * t1.y);
  C s = cmul_mi(cscale(t2, h));
  a[0] = cadd(a[0], t1);
  a[1] = cadd(m, s);
  a[2] = csub(m, s);
}

template <typename C> __device__ __forceinline__ void dft4(C* a) {
  C t0 = cadd(a[0], a[2]), t1 = csub(a[0], a[2]);
  C t2 = cadd(a[1], a[3]), t3 = csub(a[1], a[3]);
  a[0] = cadd(t0, t2);
  a[2] = csub(t0, t2);
  a[1] = cadd(t1, cmul_mi(t3));
  a[3] = csub(t1, cmul_mi(t3));
}

template <typename C> __device__ __forceinline__ void dft5(C* a) {
  typedef decltype(C().x) R;
  const R c1 = (R)0.3090169943749474241022934171828191;   // cos(2 pi / 5)
  const R c2 = (R)-0.8090169943749474241022934171828191;  // cos(4 pi / 5)
  const R s1 = (R)0.9510565162951535721164393333793821;   // sin(2 pi / 5)
  const R s2 = (R)0.5877852522924731291687059546390728;   // sin(4 pi / 5)
  C b1 = cadd(a[1], a[4]), b2 = cadd(a[2], a[3]);
  C d1 = csub(a[1], a[4]), d2 = csub(a[2], a[3]);
  C m1 = cmake<C>(a[0].x + c1 * b1.x + c2 * b2.x, a[0].y + c1 * b1.y + c2 * b2.y);
  C m2 = cmake<C>(a[0].x + c2 * b1.x + c1 * b2.x, a[0].y + c2 * b1.y + c1 * b2.y);
  C n1 = cmul_mi(cmake<C>(s1 * d1.x + s2 * d2.x, s1 * d1.y + s2 * d2.y));
  C n2 = cmul_mi(cmake<C>(s2 * d1.x - s1 * d2.x, s2 * d1.y - s1 * d2.y));
  a[0] = cadd(a[0], cadd(b1, b2));
  a[1] = cadd(m1, n1);
  a[4] = csub(m1, n1);
  a[2] = cadd(m2, n2);
  a[3] = csub(m2, n2);
}

template <typename C> __device__ __forceinline__ void dft7(C* a) {
  typedef decltype(C().x) R;
  // cos(2 pi j / 7), sin(2 pi j / 7), j = 1, 2, 3
  const R c[3] = {(R)0.6234898018587335305250048840042398, (R)-0.2225209339563144042889025644967948,
                  (R)-0.9009688679024191262361023195074451};
  const R s[3] = {(R)0.7818314824680298087084445266740578, (R)0.9749279121818236070181316829939312,
                  (R)0.4338837391175581204757683328483587};
  C b[3], d[3];
#pragma unroll
  for (int j = 0; j < 3; ++j) { b[j] = cadd(a[1 + j], a[6 - j]); d[j] = csub(a[1 + j], a[6 - j]); }
  C y[7];
  y[0] = cadd(a[0], cadd(b[0], cadd(b[1], b[2])));
#pragma unroll
  for (int k = 1; k <= 3; ++k) {
    C m = a[0], n = cmake<C>((R)0, (R)0);
#pragma unroll
    for (int j = 1; j <= 3; ++j) {
      int idx = (j * k) % 7;            // angle index of 2 pi j k / 7
      R cj, sj;
      if (idx <= 3) { cj = c[idx - 1]; sj = s[idx - 1]; }
      else { cj = c[7 - idx - 1]; sj = -s[7 - idx - 1]; }
      m.x += cj * b[j - 1].x; m.y += cj * b[j - 1].y;
      n.x += sj * d[j - 1].x; n.y += sj * d[j - 1].y;
    }
    C t = cmul_mi(n);
    y[k] = cadd(m, t);
    y[7 - k] = csub(m, t);
  }
#pragma unroll
  for (int k = 0; k < 7; ++k) a[k] = y[k];
}

template <typename C> __device__ __forceinline__ void dft8(C* a) {
  typedef decltype(C().x) R;
  const R r = (R)0.7071067811865475244008443621048490;   // 1/sqrt(2)
  C e[4] = {a[0], a[2], a[4], a[6]};
  C o[4] = {a[1], a[3], a[5], a[7]};
  dft4(e);
  dft4(o);
  // W8^k for k = 0..3: 1, (1-i)/sqrt2, -i, (-1-i)/sqrt2
  C o1 = cmake<C>(r * (o[1].x + o[1].y), r * (o[1].y - o[1].x));
  C o2 = cmul_mi(o[2]);
  C o3 = cmake<C>(r * (o[3].y - o[3].x), -r * (o[3].x + o[3].y));
  a[0] = cadd(e[0], o[0]); a[4] = csub(e[0], o[0]);
  a[1] = cadd(e[1], o1);   a[5] = csub(e[1], o1);
  a[2] = cadd(e[2], o2);   a[6] = csub(e[2], o2);
  a[3] = cadd(e[3], o3);   a[7] = csub(e[3], o3);
}

// One Stockham stage of radix R over M sequences.
template <int R, typename C>
__device__ __forceinline__ void stockham_stage(const C* __restrict__ in, C* __restrict__ out, int L, int M,
                                               int S, int Ns, const C* __restrict__ tw) {
  const int nb = L / R;                  // butterflies per sequence
  const int total = nb * M;
  const int twstep = L / (Ns * R);       // W_{Ns R}^k = W_L^(k * twstep)
  for (int t = threadIdx.x; t < total; t += blockDim.x) {
    const int m = t / nb;
    const int j = t - m * nb;
    const C* src = in + m * S;
    C a[R];
#pragma unroll
    for (int r = 0; r < R; ++r) a[r] = src[j + r * nb];
    const int k = j % Ns;
    if (Ns > 1) {
      const int base = k * twstep;
#pragma unroll
      for (int r = 1; r < R; ++r) a[r] = cmul(a[r], tw[(base * r) % L]);
    }
    if (R == 2) dft2(a);
    else if (R == 3) dft3(a);
    else if (R == 4) dft4(a);
    else if (R == 5) dft5(a);
    else if (R == 7) dft7(a);
    else if (R == 8) dft8(a);
    C* dst = out + m * S + (j / Ns) * Ns * R + k;
#pragma unroll
    for (int r = 0; r < R; ++r) dst[r * Ns] = a[r];
  }
}

// Forward FFT of M sequences of length plan.L, sequence m at buf0 + m*S
// (S >= L; S > L pads shared-memory rows against bank conflicts); buf1 is
// scratch of the same size.  Returns the buffer that holds the result.
// Must be called by all threads of the CTA; ends with __syncthreads().
template <typename C>
__device__ C* fft_batch(const FFTPlan& plan, C* buf0, C* buf1, int M, int S, const C* __restrict__ tw) {
  C* in = buf0;
  C* out = buf1;
  int Ns = 1;
  for (int s = 0; s < plan.nstages; ++s) {
    const int R = plan.radix[s];
    switch (R) {
      case 2: stockham_stage<2>(in, out, plan.L, M, S, Ns, tw); break;
      case 3: stockham_stage<3>(in, out, plan.L, M, S, Ns, tw); break;
      case 4: stockham_stage<4>(in, out, plan.L, M, S, Ns, tw); break;
      case 5: stockham_stage<5>(in, out, plan.L, M, S, Ns, tw); break;
      case 7: stockham_stage<7>(in, out, plan.L, M, S, Ns, tw); break;
      case 8: stockham_stage<8>(in, out, plan.L, M, S, Ns, tw); break;
      default: break;
    }
    __syncthreads();
    Ns *= R;
    C* t = in; in = out; out = t;
  }
  return in;
}

}  // namespace qpat
