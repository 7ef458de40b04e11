// Length-specialised 3D propagation passes on the compile-time Stockham FFTs
// of fft_reg.cuh (the 3D counterpart of fast_kernels.cuh).
//
// x row pass (one thread group per pair of y-rows (k, j0), (k, j0 + 1)):
//   start bulk copies of the two rows of up to three incoming half spectra
//   and of every state and medium field the update reads into shared memory
//   (one thread for all row pairs of the CTA); take
//   the spectra into registers, Hermitian-extend and pack the two
//   rows into one complex sequence -> inverse x-FFT via conj(FFT(conj .))
//   with the reversed plan -> wait for the copies -> pointwise update of one
//   equation (row3_point) on the registers -> forward x-FFT -> split into the
//   two rows' half spectra through shared memory -> store.
// y pass (one thread group per (z, kx) line, CBW adjacent kx per CTA so that a
//   warp's accesses are contiguous): forward y-FFT of K slots, or the inverse
//   as conj(FFT(conj .)).
// z pass (one thread group per (ky, kx) line): forward z-FFT, k-space symbol
//   (z3_apply), inverse z-FFT with the reversed plan, store.
#pragma once
#include "fast_kernels.cuh"
#include "pass3_ops.cuh"

namespace qpat {

// Row pairs per CTA of the 3D row pass: about QPAT_ROW3_THREADS threads, i.e.
// one row pair at extent 288 with 48 (measured on GB300 at 288^3 with
// per-thread operand loads: 48 threads 8.7e9, 96 threads 8.3e9, 144 threads
// 8.0e9 forward+adjoint cell-steps/s; with bulk copies, N_t 300: 48 threads
// 1.285e10, 96 threads (no idle lanes) 1.281e10 with 4 and 1.274e10 with 5
// resident CTAs per SM).
#ifndef QPAT_ROW3_THREADS
#define QPAT_ROW3_THREADS 48
#endif
template <int L>
constexpr int rp3() {
  return (QPAT_ROW3_THREADS / SGeom<L>::TPT) > 0 ? (QPAT_ROW3_THREADS / SGeom<L>::TPT) : 1;
}

// The y and z passes run their Stockham stages in one shared buffer per line
// (measured on GB300 at 288^3, 8 lines per CTA: 1.08e10 against 1.00e10
// cell-steps/s with two buffers).
constexpr bool kLine3OneBuf = true;
constexpr int kLine3Bufs = kLine3OneBuf ? 1 : 2;
#ifndef QPAT_LINE3_PAIRS
#define QPAT_LINE3_PAIRS 1
#endif
constexpr bool kLine3Pairs = QPAT_LINE3_PAIRS != 0;

// Spectral lines per CTA of the 3D y and z passes (adjacent kx; measured on
// GB300 at 288^3: 8 lines 9.3e9, 4 lines 8.7e9, 2 lines 6.3e9 cell-steps/s;
// with the present row pass, N_t 300: 8 lines 1.335e10, 16 lines in the z
// pass 1.235e10, 16 lines in the y pass 1.205e10).
#ifndef QPAT_Y3_CBW
#define QPAT_Y3_CBW 8
#endif
#ifndef QPAT_Z3_CBW
#define QPAT_Z3_CBW 8
#endif
template <int L>
constexpr int cbw3() { return QPAT_Y3_CBW; }
template <int L>
constexpr int cbw3z() { return QPAT_Z3_CBW; }
// Resident CTAs per SM the y and z passes are compiled for (two, or one for
// 16 lines per CTA).
constexpr int line3_minb(int cbw) { return cbw >= 16 ? 1 : 2; }

// Resident CTAs per SM the 3D row pass is compiled for (registers capped to
// fit; measured at 288^3: 6 1.171e10, 8 1.199e10, 9 1.174e10 cell-steps/s).
#ifndef QPAT_ROW3_MINB
#define QPAT_ROW3_MINB 8
#endif
constexpr int kRow3MinBlocks = QPAT_ROW3_MINB;

#ifndef QPAT_ROW3_DESC
#define QPAT_ROW3_DESC 1
#endif
constexpr bool kRow3Descending = QPAT_ROW3_DESC != 0;

// Row pass fed by bulk copies (cp.async.bulk issued by one thread onto two
// mbarriers: the incoming half-spectrum rows before the inverse transform,
// the operand rows before the update) instead of per-thread spectrum loads
// and cp.async pieces (measured on GB300 at 288^3, N_t 300: 1.279e10 against
// 1.192e10 forward+adjoint cell-steps/s).
#ifndef QPAT_ROW3_BULK
#define QPAT_ROW3_BULK 1
#endif
template <int L>
constexpr bool row3_bulk() { return QPAT_ROW3_BULK != 0; }
// With bulk copies the stage twiddles W_L^m come into shared memory by one
// more bulk copy (on the spectra's mbarrier) instead of per-thread copies
// (measured on GB300 at 288^3, N_t 300: 1.335e10 against 1.285e10
// forward+adjoint cell-steps/s).
#ifndef QPAT_ROW3_TWBULK
#define QPAT_ROW3_TWBULK 1
#endif

// The row pass runs its Stockham stages in one shared buffer per row pair
// (288^3: 1.11e10 against 1.09e10 cell-steps/s with two buffers).
constexpr bool kRow3OneBuf = true;

// Complex values of the row pass's shared memory before its staging area:
// twiddles and Stockham buffers, rounded up to a 16-byte boundary.
template <int L, int NSX>
constexpr int row3_stage_offset() {
  return (L + rp3<L>() * (kRow3OneBuf ? 1 : 2) * NSX * SGeom<L>::SL + 1) & ~1;
}

template <typename T, int L, int PH>
constexpr size_t row3_fast_smem_base() {
  typedef typename V2<T>::t C;
  constexpr int KIN = r3_kin(PH), KOUT = r3_kout(PH), NSX = (KIN > KOUT ? KIN : KOUT), RP = rp3<L>();
  constexpr bool SCATTER = (PH == A_R1 || PH == A_R1L);
  return (size_t)row3_stage_offset<L, NSX>() * sizeof(C) + (size_t)RP * r3_nfields(PH) * 2 * L * sizeof(T) +
         (SCATTER ? RP * 2 * L * sizeof(T) : 0);
}
// Byte offset of the bulk-copy mbarriers (after everything else, 16-aligned).
template <typename T, int L, int PH>
constexpr size_t row3_bulk_bar_offset() {
  return (row3_fast_smem_base<T, L, PH>() + 15) & ~(size_t)15;
}
template <typename T, int L, int PH>
constexpr size_t row3_fast_smem() {
  return row3_bulk<L>() ? row3_bulk_bar_offset<T, L, PH>() + 16 : row3_fast_smem_base<T, L, PH>();
}

// Operand loader reading the staged rows: field f of row rr at point i.
template <typename T, int PH, int L>
struct R3Staged {
  const T* st;
  int rr, i;
  __device__ __forceinline__ T operator()(int f) const { return st[(r3_slot(PH, f) * 2 + rr) * L + i]; }
};

template <typename T, int L, int PH>
__global__ void __launch_bounds__(rp3<L>() * SGeom<L>::TPT, kRow3MinBlocks)
row3_fast(const Prop3<T> a) {
  constexpr int KIN = r3_kin(PH), KOUT = r3_kout(PH);
  constexpr int NSX = (KIN > KOUT ? KIN : KOUT);
  constexpr int NF = r3_nfields(PH);
  typedef typename V2<T>::t C;
  typedef SGeom<L> G;
  constexpr int TPT = G::TPT, SL = G::SL, RP = rp3<L>();
  constexpr int Q1 = G::Q1, QL = G::QL, P1 = G::P1;
  constexpr bool SCATTER = (PH == A_R1 || PH == A_R1L);
  static_assert((L * sizeof(T)) % 16 == 0, "staged rows are copied in 16-byte pieces");
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int m = threadIdx.x / TPT;
  const int j = threadIdx.x - m * TPT;
  C* tws = reinterpret_cast<C*>(smem_raw);                       // W_L^m table
  constexpr int NB = kRow3OneBuf ? 1 : 2;
  // the staging area starts on a 16-byte boundary (cp.async destinations)
  constexpr int STAGE_OFF = row3_stage_offset<L, NSX>();
  C* bufA = tws + L + m * NB * NSX * SL;
  C* bufB = kRow3OneBuf ? bufA : bufA + NSX * SL;
  T* stage = reinterpret_cast<T*>(tws + STAGE_OFF) + m * NF * 2 * L;
  T* sc = reinterpret_cast<T*>(tws + STAGE_OFF) + RP * NF * 2 * L + m * 2 * L;
  // planes in descending z: the y pass before this one wrote the high planes
  // last, so they are read while still in L2, and the y pass after this one
  // (ascending) starts on the planes written last here
  const int b = blockIdx.z, k = kRow3Descending ? (int)gridDim.y - 1 - (int)blockIdx.y : (int)blockIdx.y;
  const int jp = blockIdx.x * RP + m;
  const bool valid = jp < (a.ny >> 1);
  const int j0 = valid ? 2 * jp : 0;
  C* spec = a.spec + (long long)b * a.sstride + ((long long)k * a.ny + j0) * a.pitch;
  const bool skip_in = (a.flags & kSkipInput) != 0;

  constexpr bool BULK = row3_bulk<L>();
  constexpr int kSpecRow = ((L / 2 + 1) + 1) & ~1;               // complex values per staged row (16-byte pieces)
  static_assert(!BULK || kSpecRow * 2 * KIN <= NSX * SL, "staged spectra must fit the Stockham buffer");
  static_assert(!BULK || (L % 2 == 0 && SL % 2 == 0), "every row pair's buffers start on 16-byte boundaries");
  unsigned long long* bar = reinterpret_cast<unsigned long long*>(smem_raw + row3_bulk_bar_offset<T, L, PH>());
  C* const sp = bufA;
  if constexpr (BULK) {
    // one thread issues bulk copies of the incoming half-spectrum rows (into
    // the Stockham buffer, which the first stage reads before anything writes
    // it; counted on bar[0]) and of the update's operand rows (bar[1], waited
    // for only before the update)
    if (threadIdx.x == 0) {
      mbar_init(bar, 1);
      mbar_init(bar + 1, 1);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      // every row pair mm of the CTA: its spectra into its Stockham buffer,
      // its operand rows into its staging area
      unsigned in_bytes = QPAT_ROW3_TWBULK ? L * (unsigned)sizeof(C) : 0u, op_bytes = 0;
      for (int mm = 0; mm < RP; ++mm) {
        if (blockIdx.x * RP + mm >= (a.ny >> 1)) continue;
        if (!skip_in) in_bytes += 2u * KIN * kSpecRow * (unsigned)sizeof(C);
        op_bytes += 2u * NF * L * (unsigned)sizeof(T);
      }
      mbar_arrive_expect_tx(bar, in_bytes);
      mbar_arrive_expect_tx(bar + 1, op_bytes);
      if (QPAT_ROW3_TWBULK) bulk_g2s(tws, a.twx, L * (unsigned)sizeof(C), bar);
      for (int mm = 0; mm < RP; ++mm) {
        const int jm = blockIdx.x * RP + mm;
        if (jm >= (a.ny >> 1)) continue;
        const int j0m = 2 * jm;
        if (!skip_in) {
          C* spm = tws + L + mm * NB * NSX * SL;
          const C* specm = a.spec + (long long)b * a.sstride + ((long long)k * a.ny + j0m) * a.pitch;
          for (int s = 0; s < KIN; ++s)
            for (int rr = 0; rr < 2; ++rr)
              bulk_g2s(spm + (s * 2 + rr) * kSpecRow, specm + s * a.slot + rr * a.pitch,
                       kSpecRow * (unsigned)sizeof(C), bar);
        }
        T* stm = reinterpret_cast<T*>(tws + STAGE_OFF) + mm * NF * 2 * L;
        for (int f = 0; f < NF; ++f)
          for (int rr = 0; rr < 2; ++rr)
            bulk_g2s(stm + (f * 2 + rr) * L, r3_row<T>(a, r3_field(PH, f), b, (long long)k * a.ny + j0m + rr),
                     L * (unsigned)sizeof(T), bar + 1);
      }
    }
  } else {
    // the update's operands of both rows, copied while the spectra load and the
    // inverse transform runs
    if (valid) {
      constexpr int CH = L * (int)sizeof(T) / 16;                  // 16-byte pieces per row
      constexpr int PW = 16 / (int)sizeof(T);                      // elements per piece
#pragma unroll
      for (int f = 0; f < NF; ++f)
#pragma unroll
        for (int rr = 0; rr < 2; ++rr) {
          const T* src = r3_row<T>(a, r3_field(PH, f), b, (long long)k * a.ny + j0 + rr);
          T* dst = stage + (f * 2 + rr) * L;
          for (int piece = j; piece < CH; piece += TPT) cp_async16(dst + piece * PW, src + piece * PW);
        }
    }
  }
  if (!BULK || !QPAT_ROW3_TWBULK)
    for (int t = threadIdx.x; t < L; t += blockDim.x) tws[t] = a.twx[t];
  if constexpr (BULK) row_bulk_wait(bar, a.err);                 // spectra (and twiddles) in shared memory

  // 1. inverse x-transform of the incoming half spectra (reversed plan)
  C y[KIN][Q1];
  if (!skip_in) {
    C v[KIN][P1];
    if (j < L / P1) {
#pragma unroll
      for (int s = 0; s < KIN; ++s) {
        const C* r0 = BULK ? sp + (s * 2) * kSpecRow : spec + s * a.slot;
        const C* r1 = BULK ? r0 + kSpecRow : r0 + a.pitch;
#pragma unroll
        for (int r = 0; r < P1; ++r) {
          const int n = j + r * (L / P1);
          C P, Q;
          if (2 * n <= L) {
            P = r0[n];
            Q = r1[n];
            if (n == 0 || 2 * n == L) { P.y = (T)0; Q.y = (T)0; }
          } else {
            P = cconj(r0[L - n]);
            Q = cconj(r1[L - n]);
          }
          v[s][r] = cmake<C>(P.x - Q.y, -(P.y + Q.x));   // conj(P + i Q)
        }
      }
    }
    if constexpr (BULK) __syncthreads();                          // staged spectra read before the first stage writes
    fft_stockham<L, G::P1, G::P2, G::P3, KIN, kRow3OneBuf>(v, y, bufA, bufB, SL, j, tws);
  } else {
#pragma unroll
    for (int s = 0; s < KIN; ++s)
#pragma unroll
      for (int r = 0; r < Q1; ++r) y[s][r] = cmake<C>((T)0, (T)0);
  }

  // adjoint sensor source M^T w_n on the two rows
  if (SCATTER) {
    for (int i = j; i < 2 * L; i += TPT) sc[i] = (T)0;
    __syncthreads();
    if (valid) sensor_scatter_rows3<T>(a, b, k * a.ny + j0, sc, j, TPT);
  }
  if constexpr (BULK)
    row_bulk_wait(bar + 1, a.err);
  else
    cp_async_wait_all();
  __syncthreads();

  // 2. pointwise update on grid points i = j + r L/Q1 of both rows;
  //    y = FFT(conj Z) = conj(z): row j0 is Re, row j0+1 is -Im
  C o[KOUT][Q1];
  bool bad = false;
#pragma unroll
  for (int r = 0; r < Q1; ++r) {
    T u[2][3] = {{(T)0, (T)0, (T)0}, {(T)0, (T)0, (T)0}};
    if (j < L / Q1 && valid) {
      const int i = j + r * (L / Q1);
#pragma unroll
      for (int rr = 0; rr < 2; ++rr) {
        T in[3] = {(T)0, (T)0, (T)0};
#pragma unroll
        for (int s = 0; s < KIN; ++s) in[s] = rr ? -y[s][r].y : y[s][r].x;
        const T scv = SCATTER ? sc[rr * L + i] : (T)0;
        const R3Staged<T, PH, L> ld{stage, rr, i};
        row3_point<T>(a, PH, b, i, j0 + rr, k, in, scv, ld, u[rr], bad);
      }
    }
#pragma unroll
    for (int s = 0; s < KOUT; ++s) o[s][r] = cmake<C>(u[0][s], u[1][s]);
  }
  if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr(a.err, 1);
  if (a.flags & kSkipOutput) return;

  // 3. forward x-transform of the packed outgoing rows, split, store
  C X[KOUT][QL];
  fft_stockham<L, G::Q1, G::Q2, G::Q3, KOUT, kRow3OneBuf>(o, X, bufA, bufB, SL, j, tws);
  if (j < L / QL) {
#pragma unroll
    for (int s = 0; s < KOUT; ++s)
#pragma unroll
      for (int r = 0; r < QL; ++r) bufA[s * SL + spad(j + r * (L / QL))] = X[s][r];
  }
  __syncthreads();
  if (valid) {
#pragma unroll
    for (int s = 0; s < KOUT; ++s) {
      C* w0 = spec + s * a.slot;
      C* w1 = w0 + a.pitch;
      for (int q = j; 2 * q <= L; q += TPT) {
        const C Z = bufA[s * SL + spad(q)];
        const C Zm = cconj(bufA[s * SL + spad(q == 0 ? 0 : L - q)]);
        w0[q] = cscale(cadd(Z, Zm), (T)0.5);
        w1[q] = cscale(cmul_mi(csub(Z, Zm)), (T)0.5);
      }
    }
  }
}

// Per-line shared-memory stride of the y and z passes (col_stride with the
// number of Stockham buffers in use).
template <int L, int NSX, int CBW>
__host__ __device__ constexpr int line3_stride() {
  return kLine3Bufs * NSX * SGeom<L>::SL + ((col_pad_target(CBW) - (kLine3Bufs * NSX * SGeom<L>::SL) % 16) + 16) % 16;
}

// y pass over the (z = blockIdx.y, kx) lines of problem blockIdx.z.
template <typename T, int L, int K, int INV>
__global__ void __launch_bounds__(cbw3<L>() * SGeom<L>::TPT, line3_minb(cbw3<L>()))
ypass3_fast(const Prop3<T> a, const int gather) {
  typedef typename V2<T>::t C;
  typedef SGeom<L> G;
  constexpr int SL = G::SL, CBW = cbw3<L>(), Q1 = G::Q1, QL = G::QL;
  constexpr int CS = line3_stride<L, K, CBW>();
  static_assert(CS % 2 == 0 && SL % 2 == 0, "line buffers start on 16-byte boundaries");
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int c = threadIdx.x % CBW;
  const int j = threadIdx.x / CBW;
  C* tws = reinterpret_cast<C*>(smem_raw);
  C* bufA = tws + L + c * CS;
  C* bufB = kLine3OneBuf ? bufA : bufA + K * SL;
  const int b = blockIdx.z, k = blockIdx.y;
  const int kx = blockIdx.x * CBW + c;
  const bool valid = kx < a.nxh;
  C* spec = a.spec + (long long)b * a.sstride + (long long)k * a.ny * a.pitch + (valid ? kx : 0);
  if (gather) {
    const int blk = blockIdx.y * gridDim.x + blockIdx.x;
    gather3<T>(a, b, blk * blockDim.x + threadIdx.x, gridDim.x * gridDim.y * blockDim.x);
  }
  C v[K][Q1];
  if (j < L / Q1) {
#pragma unroll
    for (int s = 0; s < K; ++s)
#pragma unroll
      for (int r = 0; r < Q1; ++r) {
        const C z = spec[s * a.slot + (long long)(j + r * (L / Q1)) * a.pitch];
        v[s][r] = INV ? cconj(z) : z;
      }
  }
  for (int t = threadIdx.x; t < L; t += blockDim.x) tws[t] = a.twy[t];
  C X[K][QL];
  fft_stockham<L, G::Q1, G::Q2, G::Q3, K, kLine3OneBuf, kLine3Pairs>(v, X, bufA, bufB, SL, j, tws);
  if (j < L / QL && valid) {
#pragma unroll
    for (int s = 0; s < K; ++s)
#pragma unroll
      for (int r = 0; r < QL; ++r)
        spec[s * a.slot + (long long)(j + r * (L / QL)) * a.pitch] = INV ? cconj(X[s][r]) : X[s][r];
  }
}

// z pass over the (ky = blockIdx.y, kx) lines of problem blockIdx.z.
template <typename T, int L, int PH>
__global__ void __launch_bounds__(cbw3z<L>() * SGeom<L>::TPT, line3_minb(cbw3z<L>()))
zpass3_fast(const Prop3<T> a) {
  constexpr int KIN = z3_kin(PH), KOUT = z3_kout(PH);
  constexpr int NSX = (KIN > KOUT ? KIN : KOUT);
  typedef typename V2<T>::t C;
  typedef SGeom<L> G;
  constexpr int SL = G::SL, CBW = cbw3z<L>(), Q1 = G::Q1, QL = G::QL;
  constexpr int CS = line3_stride<L, NSX, CBW>();
  static_assert(CS % 2 == 0 && SL % 2 == 0, "line buffers start on 16-byte boundaries");
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int c = threadIdx.x % CBW;
  const int j = threadIdx.x / CBW;
  C* tws = reinterpret_cast<C*>(smem_raw);
  C* bufA = tws + L + c * CS;
  C* bufB = kLine3OneBuf ? bufA : bufA + NSX * SL;
  const int b = blockIdx.z, ky = blockIdx.y;
  const int kx = blockIdx.x * CBW + c;
  const bool valid = kx < a.nxh;
  const int kxs = valid ? kx : 0;
  const long long zs = (long long)a.ny * a.pitch;
  C* spec = a.spec + (long long)b * a.sstride + (long long)ky * a.pitch + kxs;

  C v[KIN][Q1];
  if (j < L / Q1) {
#pragma unroll
    for (int s = 0; s < KIN; ++s)
#pragma unroll
      for (int r = 0; r < Q1; ++r) v[s][r] = spec[s * a.slot + (long long)(j + r * (L / Q1)) * zs];
  }
  // twiddles and the symbol operands of this thread's points before the transforms
  for (int t = threadIdx.x; t < L; t += blockDim.x) tws[t] = a.twz[t];
  Z3In<T, C> st[QL];
#pragma unroll
  for (int r = 0; r < QL; ++r)
    st[r] = (j < L / QL && valid) ? z3_load<T, C>(a, PH, kx, ky, j + r * (L / QL)) : Z3In<T, C>{};
  const C sx = z3_sx<T, C>(a, PH, kxs), sy = z3_sy<T, C>(a, PH, ky);
  C X[KIN][QL];
  fft_stockham<L, G::Q1, G::Q2, G::Q3, KIN, kLine3OneBuf, kLine3Pairs>(v, X, bufA, bufB, SL, j, tws);
  C o[KOUT][QL];
#pragma unroll
  for (int r = 0; r < QL; ++r) {
    C xin[3], out[3];
#pragma unroll
    for (int s = 0; s < 3; ++s) xin[s] = (s < KIN) ? X[s < KIN ? s : 0][r] : cmake<C>((T)0, (T)0);
    if (j < L / QL && valid) z3_apply<T, C>(PH, st[r], sx, sy, xin, out);
    else out[0] = out[1] = out[2] = cmake<C>((T)0, (T)0);
#pragma unroll
    for (int s = 0; s < KOUT; ++s) o[s][r] = cconj(out[s]);
  }
  C Y[KOUT][Q1];
  fft_stockham<L, G::P1, G::P2, G::P3, KOUT, kLine3OneBuf, kLine3Pairs>(o, Y, bufA, bufB, SL, j, tws);
  if (j < L / Q1 && valid) {
#pragma unroll
    for (int s = 0; s < KOUT; ++s)
#pragma unroll
      for (int r = 0; r < Q1; ++r) spec[s * a.slot + (long long)(j + r * (L / Q1)) * zs] = cconj(Y[s][r]);
  }
}

template <typename T, int L, int NSX, int CBW = cbw3<L>()>
constexpr size_t line3_fast_smem() {
  typedef typename V2<T>::t C;
  return ((size_t)L + (size_t)CBW * line3_stride<L, NSX, CBW>()) * sizeof(C);
}

template <typename T, int L, int PH>
void set_row3_fast_attr() {
  cudaFuncSetAttribute(row3_fast<T, L, PH>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)row3_fast_smem<T, L, PH>());
}
template <typename T, int L, int PH>
void set_z3_fast_attr() {
  constexpr int NSX = z3_kin(PH) > z3_kout(PH) ? z3_kin(PH) : z3_kout(PH);
  cudaFuncSetAttribute(zpass3_fast<T, L, PH>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)line3_fast_smem<T, L, NSX, cbw3z<L>()>());
}
template <typename T, int L, int K, int INV>
void set_y3_fast_attr() {
  cudaFuncSetAttribute(ypass3_fast<T, L, K, INV>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)line3_fast_smem<T, L, K>());
}

// Dynamic shared-memory limits of all 3D pass kernels of length L; called at
// context creation, outside any stream capture.
template <typename T, int L>
void prepare3_fast_len() {
  set_row3_fast_attr<T, L, F_R1>(); set_row3_fast_attr<T, L, F_R2>(); set_row3_fast_attr<T, L, F_R3>();
  set_row3_fast_attr<T, L, F_R3L>(); set_row3_fast_attr<T, L, A_R1>(); set_row3_fast_attr<T, L, A_R1L>();
  set_row3_fast_attr<T, L, A_R3>(); set_row3_fast_attr<T, L, A_R5>();
  set_z3_fast_attr<T, L, F_C1>(); set_z3_fast_attr<T, L, F_C2>(); set_z3_fast_attr<T, L, F_C3>();
  set_z3_fast_attr<T, L, A_C2>(); set_z3_fast_attr<T, L, A_C4>(); set_z3_fast_attr<T, L, A_C6>();
  set_y3_fast_attr<T, L, 1, 0>(); set_y3_fast_attr<T, L, 2, 0>(); set_y3_fast_attr<T, L, 3, 0>();
  set_y3_fast_attr<T, L, 1, 1>(); set_y3_fast_attr<T, L, 2, 1>(); set_y3_fast_attr<T, L, 3, 1>();
}

template <typename T, int L, int PH>
void run_row3_fast(const Prop3<T>& a, int batch, cudaStream_t s) {
  constexpr int RP = rp3<L>();
  const dim3 grid((a.ny / 2 + RP - 1) / RP, a.nz, batch);
  row3_fast<T, L, PH><<<grid, RP * SGeom<L>::TPT, row3_fast_smem<T, L, PH>(), s>>>(a);
}
template <typename T, int L, int PH>
void run_z3_fast(const Prop3<T>& a, int batch, cudaStream_t s) {
  typedef SGeom<L> G;
  constexpr int NSX = z3_kin(PH) > z3_kout(PH) ? z3_kin(PH) : z3_kout(PH);
  constexpr int CBW = cbw3z<L>();
  const dim3 grid((a.nxh + CBW - 1) / CBW, a.ny, batch);
  zpass3_fast<T, L, PH><<<grid, CBW * G::TPT, line3_fast_smem<T, L, NSX, CBW>(), s>>>(a);
}
template <typename T, int L, int K, int INV>
void run_y3_fast(const Prop3<T>& a, int gather, int batch, cudaStream_t s) {
  typedef SGeom<L> G;
  constexpr int CBW = cbw3<L>();
  const dim3 grid((a.nxh + CBW - 1) / CBW, a.nz, batch);
  ypass3_fast<T, L, K, INV><<<grid, CBW * G::TPT, line3_fast_smem<T, L, K>(), s>>>(a, gather);
}

template <typename T, int L>
void launch_row3_fast_len(const Prop3<T>& a, int ph, int batch, cudaStream_t s) {
  switch (ph) {
    case F_R1: run_row3_fast<T, L, F_R1>(a, batch, s); break;
    case F_R2: run_row3_fast<T, L, F_R2>(a, batch, s); break;
    case F_R3: run_row3_fast<T, L, F_R3>(a, batch, s); break;
    case F_R3L: run_row3_fast<T, L, F_R3L>(a, batch, s); break;
    case A_R1: run_row3_fast<T, L, A_R1>(a, batch, s); break;
    case A_R1L: run_row3_fast<T, L, A_R1L>(a, batch, s); break;
    case A_R3: run_row3_fast<T, L, A_R3>(a, batch, s); break;
    case A_R5: run_row3_fast<T, L, A_R5>(a, batch, s); break;
    default: break;
  }
}
template <typename T, int L>
void launch_z3_fast_len(const Prop3<T>& a, int ph, int batch, cudaStream_t s) {
  switch (ph) {
    case F_C1: run_z3_fast<T, L, F_C1>(a, batch, s); break;
    case F_C2: run_z3_fast<T, L, F_C2>(a, batch, s); break;
    case F_C3: run_z3_fast<T, L, F_C3>(a, batch, s); break;
    case A_C2: run_z3_fast<T, L, A_C2>(a, batch, s); break;
    case A_C4: run_z3_fast<T, L, A_C4>(a, batch, s); break;
    case A_C6: run_z3_fast<T, L, A_C6>(a, batch, s); break;
    default: break;
  }
}
template <typename T, int L>
void launch_y3_fast_len(const Prop3<T>& a, int K, int inv, int gather, int batch, cudaStream_t s) {
  if (!inv) {
    if (K == 1) run_y3_fast<T, L, 1, 0>(a, gather, batch, s);
    else if (K == 2) run_y3_fast<T, L, 2, 0>(a, gather, batch, s);
    else run_y3_fast<T, L, 3, 0>(a, gather, batch, s);
  } else {
    if (K == 1) run_y3_fast<T, L, 1, 1>(a, gather, batch, s);
    else if (K == 2) run_y3_fast<T, L, 2, 1>(a, gather, batch, s);
    else run_y3_fast<T, L, 3, 1>(a, gather, batch, s);
  }
}

#define QPAT_FAST3_LENGTH(L)                                                                                   \
  template void prepare3_fast_len<float, L>();                                                                 \
  template void launch_row3_fast_len<float, L>(const Prop3<float>&, int, int, cudaStream_t);                 \
  template void launch_y3_fast_len<float, L>(const Prop3<float>&, int, int, int, int, cudaStream_t);         \
  template void launch_z3_fast_len<float, L>(const Prop3<float>&, int, int, cudaStream_t);

}  // namespace qpat
