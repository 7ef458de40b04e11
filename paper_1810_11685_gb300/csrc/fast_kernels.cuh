// Length-specialised propagation passes on compile-time Stockham FFTs.
//
// Row pass (one thread group per pair of grid rows j0, j0 + 1):
//   load the incoming half spectra straight into registers, Hermitian-extend
//   them and pack the two rows into one complex sequence -> inverse x-FFT via
//   conj(FFT(conj .)) with the radices of the forward plan reversed -> each
//   thread ends holding grid points j + r L/Q1 of both rows -> pointwise
//   update (row_point) in registers -> forward x-FFT, whose first stage reads
//   exactly those registers -> split into two half spectra through shared
//   memory -> store.
// Column pass (one thread group per half-spectrum column, CBW adjacent
//   columns per CTA, column index fastest so that global accesses of a warp
//   are contiguous):
//   load rows j + r L/Q1 of the column -> forward y-FFT -> spectral symbol
//   (col_point) on the registers -> inverse y-FFT (reversed radices), which
//   ends in the load layout -> store.
#pragma once
#include "fft_reg.cuh"
#include "pass_ops.cuh"

namespace qpat {

// Forward radix plans (Q3 = 1: two stages).  The inverse uses them reversed.
template <int L> struct SPlan { static constexpr int Q1 = 0, Q2 = 0, Q3 = 0; };
template <> struct SPlan<24> { static constexpr int Q1 = 4, Q2 = 6, Q3 = 1; };
template <> struct SPlan<40> { static constexpr int Q1 = 5, Q2 = 8, Q3 = 1; };
template <> struct SPlan<48> { static constexpr int Q1 = 6, Q2 = 8, Q3 = 1; };
template <> struct SPlan<54> { static constexpr int Q1 = 6, Q2 = 9, Q3 = 1; };
template <> struct SPlan<56> { static constexpr int Q1 = 7, Q2 = 8, Q3 = 1; };
template <> struct SPlan<168> { static constexpr int Q1 = 12, Q2 = 14, Q3 = 1; };
template <> struct SPlan<288> { static constexpr int Q1 = 8, Q2 = 6, Q3 = 6; };
template <> struct SPlan<432> { static constexpr int Q1 = 6, Q2 = 8, Q3 = 9; };
template <> struct SPlan<576> { static constexpr int Q1 = 8, Q2 = 8, Q3 = 9; };
template <> struct SPlan<1024> { static constexpr int Q1 = 8, Q2 = 8, Q3 = 16; };
template <> struct SPlan<1080> { static constexpr int Q1 = 10, Q2 = 12, Q3 = 9; };

template <int L>
struct SGeom {
  static constexpr int Q1 = SPlan<L>::Q1, Q2 = SPlan<L>::Q2, Q3 = SPlan<L>::Q3;
  static constexpr bool three = Q3 > 1;
  static constexpr int QL = three ? Q3 : Q2;                    // last forward radix
  // inverse plan: reversed radices
  static constexpr int P1 = QL, P2 = three ? Q2 : Q1, P3 = three ? Q1 : 1;
  static constexpr int minQ = three ? (Q1 < Q2 ? (Q1 < Q3 ? Q1 : Q3) : (Q2 < Q3 ? Q2 : Q3)) : (Q1 < Q2 ? Q1 : Q2);
  static constexpr int TPT = L / minQ;
  static constexpr int SL = spad_size(L);
  static constexpr int RP = (192 / TPT) > 0 ? (192 / TPT) : 1;   // row pairs per CTA
  // columns per CTA: 8 adjacent columns make each warp access 64 contiguous
  // bytes per row (measured on GB300: 576^2 batch 8 1.92e10 against 1.82e10
  // cell-steps/s with 4 columns; 288^2..576^2 jvp mix 1.9e10 against 1.7e10).
  // Fewer where 8 columns' two-slot double buffers would not fit in the 227
  // KB of shared memory a CTA may use (extents 1024, 1080: 4 columns).
  static constexpr int col_bytes(int cbw) { return (L + cbw * (4 * SL + 16)) * 8; }
  static constexpr int CBW = col_bytes(8) <= 227 * 1024 ? 8 : col_bytes(4) <= 227 * 1024 ? 4 : 2;
};

template <typename T, int L, int PH>
__global__ void __launch_bounds__(SGeom<L>::RP * SGeom<L>::TPT)
row_fast(const PropArgs<T> a) {
  constexpr int ph = PH, KIN = row_kin(PH), KOUT = row_kout(PH);
  typedef typename V2<T>::t C;
  typedef SGeom<L> G;
  constexpr int TPT = G::TPT, SL = G::SL, RP = G::RP, NSX = (KIN > KOUT ? KIN : KOUT);
  constexpr int Q1 = G::Q1, QL = G::QL, P1 = G::P1;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int m = threadIdx.x / TPT;
  const int j = threadIdx.x - m * TPT;
  C* tws = reinterpret_cast<C*>(smem_raw);                       // W_L^m table
  C* bufA = tws + L + m * 2 * NSX * SL;
  C* bufB = bufA + NSX * SL;
  T* sc = reinterpret_cast<T*>(tws + L + RP * 2 * NSX * SL) + m * 2 * L;
  const int b = blockIdx.y;
  const int jp = blockIdx.x * RP + m;
  const bool valid = jp < (a.ny >> 1);
  const int j0 = valid ? 2 * jp : 0;
  C* spec = a.spec + (long long)b * a.sstride;
  const long long slot = (long long)a.ny * a.pitch;
  const bool skip_in = (a.flags & kSkipInput) != 0;

  // twiddle table to shared memory, and every pointwise operand of this
  // thread's grid points into registers, before any transform: their
  // latencies overlap the loads of the spectra and the first FFT stage
  for (int t = threadIdx.x; t < L; t += blockDim.x) tws[t] = a.twx[t];
  RowIn<T> st[2][Q1];
#pragma unroll
  for (int r = 0; r < Q1; ++r)
#pragma unroll
    for (int rr = 0; rr < 2; ++rr)
      st[rr][r] = (j < L / Q1 && valid) ? row_load<T>(a, ph, b, j + r * (L / Q1), j0 + rr) : RowIn<T>{};

  // 1. inverse x-transform of the incoming half spectra (reversed plan)
  C y[KIN][Q1];
  if (!skip_in) {
    C v[KIN][P1];
    if (j < L / P1) {
#pragma unroll
      for (int s = 0; s < KIN; ++s) {
        const C* r0 = spec + s * slot + (long long)j0 * a.pitch;
        const C* r1 = r0 + a.pitch;
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
    fft_stockham<L, G::P1, G::P2, G::P3, KIN>(v, y, bufA, bufB, SL, j, tws);
  } else {
#pragma unroll
    for (int s = 0; s < KIN; ++s)
#pragma unroll
      for (int r = 0; r < Q1; ++r) y[s][r] = cmake<C>((T)0, (T)0);
  }

  // adjoint sensor source M^T w_n on the two rows (A_R1, A_R1L)
  if (KIN == 1) {
    for (int i = j; i < 2 * L; i += TPT) sc[i] = (T)0;
    __syncthreads();
    if (valid) sensor_scatter_rows<T>(a, b, j0, sc, j, TPT);
    __syncthreads();
  }

  // 2. pointwise update on grid points i = j + r L/Q1 of both rows;
  //    y = FFT(conj Z) = conj(z): row j0 is Re, row j0+1 is -Im
  C o[KOUT][Q1];
  bool bad = false;
#pragma unroll
  for (int r = 0; r < Q1; ++r) {
    T u0[2] = {(T)0, (T)0}, u1[2] = {(T)0, (T)0};
    if (j < L / Q1 && valid) {
      const int i = j + r * (L / Q1);
#pragma unroll
      for (int rr = 0; rr < 2; ++rr) {
        const T in0 = rr ? -y[0][r].y : y[0][r].x;
        const T in1 = (KIN > 1) ? (rr ? -y[KIN - 1][r].y : y[KIN - 1][r].x) : (T)0;
        const T scv = (KIN == 1) ? sc[rr * L + i] : (T)0;
        row_point<T>(a, ph, b, i, j0 + rr, in0, in1, scv, st[rr][r], u0[rr], u1[rr], bad);
      }
    }
    o[0][r] = cmake<C>(u0[0], u0[1]);
    if (KOUT > 1) o[KOUT - 1][r] = cmake<C>(u1[0], u1[1]);
  }
  if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr(a.err, 1);
  if (a.flags & kSkipOutput) return;

  // 3. forward x-transform of the packed outgoing rows
  C X[KOUT][QL];
  fft_stockham<L, G::Q1, G::Q2, G::Q3, KOUT>(o, X, bufA, bufB, SL, j, tws);
  // thread j < L/QL holds Z[j + r L/QL]; split Z into the two rows' half
  // spectra A(k) = (Z(k) + conj Z(-k))/2, B(k) = -i (Z(k) - conj Z(-k))/2
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
      C* w0 = spec + s * slot + (long long)j0 * a.pitch;
      C* w1 = w0 + a.pitch;
      for (int k = j; 2 * k <= L; k += TPT) {
        const C Z = bufA[s * SL + spad(k)];
        const C Zm = cconj(bufA[s * SL + spad(k == 0 ? 0 : L - k)]);
        w0[k] = cscale(cadd(Z, Zm), (T)0.5);
        w1[k] = cscale(cmul_mi(csub(Z, Zm)), (T)0.5);
      }
    }
  }
}

// ---- row pass with the pointwise operands staged in shared memory ----------
// The same pass as row_fast, but the state and medium rows that the update
// reads are copied into shared memory with cp.async (issued before the
// spectra loads, waited on just before the update) instead of being held in
// registers across the inverse transform.  Used for extents whose rows are a
// whole number of 16-byte pieces.

// Field of the medium or state staged for RowIn member v (0..4) of phase ph,
// -1 if the update does not read it.
enum RowField : int { RFVX, RFVY, RFRX, RFRY, RFPB, RFCC, RFRHO, RFDX, RFDY, RFETA, RFTAU };
__host__ __device__ constexpr int row_field(int ph, int v) {
  switch (ph) {
    case F_R1: { const int f[5] = {RFRX, RFRY, RFCC, RFETA, RFTAU}; return f[v]; }
    case F_R2: case A_R5: { const int f[5] = {RFVX, RFVY, RFDX, RFDY, -1}; return f[v]; }
    case F_R3: case F_R3L: case A_R1L: { const int f[5] = {RFRX, RFRY, RFRHO, RFCC, -1}; return f[v]; }
    case A_R1: { const int f[5] = {-1, -1, RFCC, RFETA, RFTAU}; return f[v]; }
    case A_R3: { const int f[5] = {RFRX, RFRY, RFRHO, RFCC, RFPB}; return f[v]; }
    default: return -1;
  }
}
// Staging slot of RowIn member v (its rank among the members the phase reads).
__host__ __device__ constexpr int row_stage_slot(int ph, int v) {
  int n = 0;
  for (int u = 0; u < v; ++u) n += row_field(ph, u) >= 0 ? 1 : 0;
  return n;
}
__host__ __device__ constexpr int row_nfields(int ph) { return row_stage_slot(ph, 5); }

// Row-start pointer of field f for grid row j of problem b.
template <typename T>
__device__ __forceinline__ const T* row_field_ptr(const PropArgs<T>& a, int f, int b, int j) {
  const long long o = (long long)j * a.nx, ob = (long long)b * a.gstride + o;
  switch (f) {
    case RFVX: return a.vx + ob;
    case RFVY: return a.vy + ob;
    case RFRX: return a.rx + ob;
    case RFRY: return a.ry + ob;
    case RFPB: return a.pbuf + ob;
    case RFCC: return a.Cc + o;
    case RFRHO: return a.rho0 + o;
    case RFDX: return a.dtrsx + o;
    case RFDY: return a.dtrsy + o;
    case RFETA: return a.eta + o;
    default: return a.tau + o;
  }
}

// c^2 is read by F_R3 and A_R3 only at the source steps.
__device__ __forceinline__ bool row_field_needed(int ph, int f, int flags) {
  if (f != RFCC) return true;
  if (ph == F_R3) return (flags & kSource) != 0;
  if (ph == A_R3) return (flags & (kAccWrite | kAccAdd)) != 0;
  return true;
}

#ifndef QPAT_ROW_STAGED
#define QPAT_ROW_STAGED 1
#endif
template <int L>
__host__ __device__ constexpr bool row_staged() { return QPAT_ROW_STAGED && L % 4 == 0 && L >= 96; }

// Row pairs per CTA of the staged row pass.
#ifndef QPAT_ROWST_RP
#define QPAT_ROWST_RP 1
#endif
template <int L>
__host__ __device__ constexpr int rp_st() { return QPAT_ROWST_RP; }

#ifndef QPAT_ROWST_ONEBUF
#define QPAT_ROWST_ONEBUF 1
#endif
// Staged row pass fed by bulk copies (cp.async.bulk issued by one thread onto
// two mbarriers) instead of per-thread loads of the spectra and cp.async
// pieces of the operand rows (measured at 576^2 batch 12, Nt 600 on GB300:
// 2.325e10 against 2.190e10 cell-steps/s).
#ifndef QPAT_ROWST_BULK
#define QPAT_ROWST_BULK 1
#endif
constexpr bool kRowStOneBuf = QPAT_ROWST_ONEBUF != 0;

// Complex values before the staging area (twiddles and Stockham buffers),
// rounded up to a 16-byte boundary.
// Stage twiddles W_L^m of the staged row pass: a per-CTA shared copy (0),
// which the bulk-copy form fetches with one more copy, or read straight from
// global memory through L1 (1).  Measured on GB300 at 576^2 batch 12, N_t
// 600, with bulk copies: 2.352e10 against 2.322e10 cell-steps/s from L1
// (with per-thread copies the L1 reads were the faster form).
#ifndef QPAT_ROWST_TWG
#define QPAT_ROWST_TWG 0
#endif
constexpr bool kRowStTwGlobal = QPAT_ROWST_TWG != 0;
constexpr int kRowStTwSmem(int L) { return kRowStTwGlobal ? 0 : L; }

template <int L, int NSX, int RP = rp_st<L>()>
__host__ __device__ constexpr int row_st_offset() {
  return (kRowStTwSmem(L) + RP * (kRowStOneBuf ? 1 : 2) * NSX * SGeom<L>::SL + 1) & ~1;
}

// At least six resident CTAs per SM (registers capped to fit; measured at
// 576^2 batch 12, Nt 600: 2.145e10 with no bound, 2.186e10 with 6, 2.148e10
// with 7, 2.163e10 with 8 cell-steps/s).
#ifndef QPAT_ROWST_MINB
#define QPAT_ROWST_MINB 6
#endif
// Body of the staged row pass for row-pair block `blk` of problem b, run by
// RP * TPT threads (threadIdx.x), in the launch's dynamic shared memory
// (row_fast_st_smem bytes), which the body names itself so that every
// access stays a shared-memory access.  Every thread of the CTA must call it.
template <typename T, int L, int PH, int RP>
__device__ __forceinline__ void row_st_body(const PropArgs<T> a, const int b, const int blk) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  constexpr int ph = PH, KIN = row_kin(PH), KOUT = row_kout(PH);
  constexpr int NSX = (KIN > KOUT ? KIN : KOUT), NF = row_nfields(PH);
  typedef typename V2<T>::t C;
  typedef SGeom<L> G;
  constexpr int TPT = G::TPT, SL = G::SL;
  constexpr int Q1 = G::Q1, QL = G::QL, P1 = G::P1;
  constexpr int NB = kRowStOneBuf ? 1 : 2;
  static_assert((L * sizeof(T)) % 16 == 0, "staged rows are copied in 16-byte pieces");
  static_assert(SL % 2 == 0 && row_st_offset<L, NSX, RP>() % 2 == 0,
                "row-group buffers and the staging area must start on 16-byte boundaries");
  const int m = threadIdx.x / TPT;
  const int j = threadIdx.x - m * TPT;
  C* const sbase = reinterpret_cast<C*>(smem_raw);
  C* tws = sbase;                                                // W_L^m table
  const C* tw = kRowStTwGlobal ? a.twx : tws;
  C* bufA = sbase + kRowStTwSmem(L) + m * NB * NSX * SL;
  C* bufB = kRowStOneBuf ? bufA : bufA + NSX * SL;
  constexpr int OFF = row_st_offset<L, NSX, RP>();
  T* stage = reinterpret_cast<T*>(sbase + OFF) + m * NF * 2 * L;
  T* sc = reinterpret_cast<T*>(sbase + OFF) + RP * NF * 2 * L + m * 2 * L;
  const int jp = blk * RP + m;
  const bool valid = jp < (a.ny >> 1);
  const int j0 = valid ? 2 * jp : 0;
  C* spec = a.spec + (long long)b * a.sstride;
  const long long slot = (long long)a.ny * a.pitch;
  const bool skip_in = (a.flags & kSkipInput) != 0;

  // the update's operands of both rows, copied while the spectra load and the
  // inverse transform runs
  if (valid) {
    constexpr int CH = L * (int)sizeof(T) / 16;                  // 16-byte pieces per row
    constexpr int PW = 16 / (int)sizeof(T);                      // elements per piece
#pragma unroll
    for (int v = 0; v < 5; ++v) {
      const int f = row_field(ph, v);
      if (f < 0 || !row_field_needed(ph, f, a.flags)) continue;
      const int sl = row_stage_slot(ph, v);
#pragma unroll
      for (int rr = 0; rr < 2; ++rr) {
        const T* src = row_field_ptr<T>(a, f, b, j0 + rr);
        T* dst = stage + (sl * 2 + rr) * L;
        for (int piece = j; piece < CH; piece += TPT) cp_async16(dst + piece * PW, src + piece * PW);
      }
    }
  }
  if constexpr (!kRowStTwGlobal)
    for (int t = threadIdx.x; t < L; t += RP * TPT) tws[t] = a.twx[t];

  // 1. inverse x-transform of the incoming half spectra (reversed plan)
  C y[KIN][Q1];
  if (!skip_in) {
    C v[KIN][P1];
    if (j < L / P1) {
#pragma unroll
      for (int s = 0; s < KIN; ++s) {
        const C* r0 = spec + s * slot + (long long)j0 * a.pitch;
        const C* r1 = r0 + a.pitch;
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
    fft_stockham<L, G::P1, G::P2, G::P3, KIN, kRowStOneBuf>(v, y, bufA, bufB, SL, j, tw);
  } else {
#pragma unroll
    for (int s = 0; s < KIN; ++s)
#pragma unroll
      for (int r = 0; r < Q1; ++r) y[s][r] = cmake<C>((T)0, (T)0);
  }

  // adjoint sensor source M^T w_n on the two rows (A_R1, A_R1L)
  if (KIN == 1) {
    for (int i = j; i < 2 * L; i += TPT) sc[i] = (T)0;
    __syncthreads();
    if (valid) sensor_scatter_rows<T>(a, b, j0, sc, j, TPT);
  }
  cp_async_wait_all();
  __syncthreads();

  // 2. pointwise update on grid points i = j + r L/Q1 of both rows;
  //    y = FFT(conj Z) = conj(z): row j0 is Re, row j0+1 is -Im
  C o[KOUT][Q1];
  bool bad = false;
#pragma unroll
  for (int r = 0; r < Q1; ++r) {
    T u0[2] = {(T)0, (T)0}, u1[2] = {(T)0, (T)0};
    if (j < L / Q1 && valid) {
      const int i = j + r * (L / Q1);
#pragma unroll
      for (int rr = 0; rr < 2; ++rr) {
        T sv[5];
#pragma unroll
        for (int v = 0; v < 5; ++v)
          sv[v] = row_field(ph, v) >= 0 ? stage[(row_stage_slot(ph, v) * 2 + rr) * L + i] : (T)0;
        const RowIn<T> st{sv[0], sv[1], sv[2], sv[3], sv[4]};
        const T in0 = rr ? -y[0][r].y : y[0][r].x;
        const T in1 = (KIN > 1) ? (rr ? -y[KIN - 1][r].y : y[KIN - 1][r].x) : (T)0;
        const T scv = (KIN == 1) ? sc[rr * L + i] : (T)0;
        row_point<T>(a, ph, b, i, j0 + rr, in0, in1, scv, st, u0[rr], u1[rr], bad);
      }
    }
    o[0][r] = cmake<C>(u0[0], u0[1]);
    if (KOUT > 1) o[KOUT - 1][r] = cmake<C>(u1[0], u1[1]);
  }
  if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr(a.err, 1);
  if (a.flags & kSkipOutput) return;

  // 3. forward x-transform of the packed outgoing rows, split, store
  C X[KOUT][QL];
  fft_stockham<L, G::Q1, G::Q2, G::Q3, KOUT, kRowStOneBuf>(o, X, bufA, bufB, SL, j, tw);
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
      C* w0 = spec + s * slot + (long long)j0 * a.pitch;
      C* w1 = w0 + a.pitch;
      for (int k = j; 2 * k <= L; k += TPT) {
        const C Z = bufA[s * SL + spad(k)];
        const C Zm = cconj(bufA[s * SL + spad(k == 0 ? 0 : L - k)]);
        w0[k] = cscale(cadd(Z, Zm), (T)0.5);
        w1[k] = cscale(cmul_mi(csub(Z, Zm)), (T)0.5);
      }
    }
  }
}

// Wait for phase 0 of a bulk-copy barrier; when the bounded wait gives up,
// flag the context (bit 2) and wait once more so that no copy is still
// landing in shared memory when the block moves on.
__device__ __forceinline__ void row_bulk_wait(unsigned long long* bar, int* err) {
  if (!mbar_wait_bounded(bar, 0)) {
    atomicOr(err, 2);
    mbar_wait_bounded(bar, 0);
  }
}

// Dynamic shared memory of the staged row pass.
template <typename T, int L, int PH, int RP = rp_st<L>()>
constexpr size_t row_fast_st_smem_base() {
  typedef typename V2<T>::t C;
  constexpr int KIN = row_kin(PH), KOUT = row_kout(PH), NSX = (KIN > KOUT ? KIN : KOUT);
  return row_st_offset<L, NSX, RP>() * sizeof(C) + (size_t)RP * (row_nfields(PH) * 2 * L) * sizeof(T) +
         (KIN == 1 ? (size_t)RP * 2 * L * sizeof(T) : 0);
}
// Byte offset of the bulk-copy mbarriers of the single-context staged row
// pass (one row pair per CTA): after everything else, 16-aligned.
template <typename T, int L, int PH>
constexpr size_t row_bulk_bar_offset() {
  return (row_fast_st_smem_base<T, L, PH, 1>() + 15) & ~(size_t)15;
}
// With bulk copies two mbarriers follow, on a 16-byte boundary (the
// multi-problem kernels size their shared memory with this too, for RP row
// pairs, and never touch the barriers).
template <typename T, int L, int PH, int RP = rp_st<L>()>
constexpr size_t row_fast_st_smem() {
  return QPAT_ROWST_BULK ? ((row_fast_st_smem_base<T, L, PH, RP>() + 15) & ~(size_t)15) + 16
                         : row_fast_st_smem_base<T, L, PH, RP>();
}

// The single-context staged row pass.  It keeps its own copy of the body
// above rather than calling row_st_body: the same code reached through the
// device function measured 11% slower at 576^2 (1.96e10 against 2.19e10
// cell-steps/s on GB300, with the body taking its arguments by reference or
// by value, naming the shared memory itself or receiving it), so the
// single-context kernels stay in this form and the body serves the
// multi-problem kernels (multi_kernels.cuh).
template <typename T, int L, int PH>
__global__ void __launch_bounds__(rp_st<L>() * SGeom<L>::TPT, QPAT_ROWST_MINB)
row_fast_st(const PropArgs<T> a) {
  constexpr int ph = PH, KIN = row_kin(PH), KOUT = row_kout(PH);
  constexpr int NSX = (KIN > KOUT ? KIN : KOUT), NF = row_nfields(PH);
  typedef typename V2<T>::t C;
  typedef SGeom<L> G;
  constexpr int TPT = G::TPT, SL = G::SL, RP = rp_st<L>();
  constexpr int Q1 = G::Q1, QL = G::QL, P1 = G::P1;
  constexpr int NB = kRowStOneBuf ? 1 : 2;
  static_assert((L * sizeof(T)) % 16 == 0, "staged rows are copied in 16-byte pieces");
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int m = threadIdx.x / TPT;
  const int j = threadIdx.x - m * TPT;
  C* const sbase = reinterpret_cast<C*>(smem_raw);
  C* tws = sbase;                                                // W_L^m table
  const C* tw = kRowStTwGlobal ? a.twx : tws;
  C* bufA = sbase + kRowStTwSmem(L) + m * NB * NSX * SL;
  C* bufB = kRowStOneBuf ? bufA : bufA + NSX * SL;
  constexpr int OFF = row_st_offset<L, NSX>();
  T* stage = reinterpret_cast<T*>(sbase + OFF) + m * NF * 2 * L;
  T* sc = reinterpret_cast<T*>(sbase + OFF) + RP * NF * 2 * L + m * 2 * L;
  const int b = blockIdx.y;
  const int jp = blockIdx.x * RP + m;
  const bool valid = jp < (a.ny >> 1);
  const int j0 = valid ? 2 * jp : 0;
  C* spec = a.spec + (long long)b * a.sstride;
  const long long slot = (long long)a.ny * a.pitch;
  const bool skip_in = (a.flags & kSkipInput) != 0;

#if QPAT_ROWST_BULK
  // one thread issues bulk copies of the incoming half-spectrum rows (into
  // the Stockham buffer, which the first stage reads before anything writes
  // it; counted on bar[0]) and of the update's operand rows (bar[1], waited
  // for only before the update)
  static_assert(RP == 1, "bulk-copy staging serves one row pair per CTA");
  static_assert(row_bulk_bar_offset<T, L, PH>() + 16 <= row_fast_st_smem<T, L, PH>(), "barriers inside the launch's shared memory");
  constexpr int kSpecRow = ((L / 2 + 1) + 1) & ~1;               // complex values per staged row (16-byte pieces)
  static_assert(kSpecRow * 2 * KIN <= NSX * SL, "staged spectra must fit the Stockham buffer");
  unsigned long long* bar = reinterpret_cast<unsigned long long*>(smem_raw + row_bulk_bar_offset<T, L, PH>());
  C* const sp = bufA;
  if (threadIdx.x == 0) {
    mbar_init(bar, 1);
    mbar_init(bar + 1, 1);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    const bool load_in = valid && !skip_in;
    // (with the twiddles in shared memory, they come by one more copy)
    mbar_arrive_expect_tx(bar, (load_in ? 2u * KIN * kSpecRow * (unsigned)sizeof(C) : 0u) +
                                   (kRowStTwGlobal ? 0u : L * (unsigned)sizeof(C)));
    if constexpr (!kRowStTwGlobal) bulk_g2s(tws, a.twx, L * (unsigned)sizeof(C), bar);
    if (load_in)
      for (int s = 0; s < KIN; ++s)
        for (int rr = 0; rr < 2; ++rr)
          bulk_g2s(sp + (s * 2 + rr) * kSpecRow, spec + s * slot + (long long)(j0 + rr) * a.pitch,
                   kSpecRow * (unsigned)sizeof(C), bar);
    unsigned bytes = 0;
    if (valid) {
#pragma unroll
      for (int v = 0; v < 5; ++v) {
        const int f = row_field(ph, v);
        if (f >= 0 && row_field_needed(ph, f, a.flags)) bytes += 2u * L * (unsigned)sizeof(T);
      }
    }
    mbar_arrive_expect_tx(bar + 1, bytes);
    if (valid) {
#pragma unroll
      for (int v = 0; v < 5; ++v) {
        const int f = row_field(ph, v);
        if (f < 0 || !row_field_needed(ph, f, a.flags)) continue;
        const int sl = row_stage_slot(ph, v);
        for (int rr = 0; rr < 2; ++rr)
          bulk_g2s(stage + (sl * 2 + rr) * L, row_field_ptr<T>(a, f, b, j0 + rr), L * (unsigned)sizeof(T),
                   bar + 1);
      }
    }
  }
#else
  // the update's operands of both rows, copied while the spectra load and the
  // inverse transform runs
  if (valid) {
    constexpr int CH = L * (int)sizeof(T) / 16;                  // 16-byte pieces per row
    constexpr int PW = 16 / (int)sizeof(T);                      // elements per piece
#pragma unroll
    for (int v = 0; v < 5; ++v) {
      const int f = row_field(ph, v);
      if (f < 0 || !row_field_needed(ph, f, a.flags)) continue;
      const int sl = row_stage_slot(ph, v);
#pragma unroll
      for (int rr = 0; rr < 2; ++rr) {
        const T* src = row_field_ptr<T>(a, f, b, j0 + rr);
        T* dst = stage + (sl * 2 + rr) * L;
        for (int piece = j; piece < CH; piece += TPT) cp_async16(dst + piece * PW, src + piece * PW);
      }
    }
  }
#endif
#if QPAT_ROWST_BULK
  row_bulk_wait(bar, a.err);                                     // spectra (and twiddles) in shared memory
#else
  if constexpr (!kRowStTwGlobal)
    for (int t = threadIdx.x; t < L; t += blockDim.x) tws[t] = a.twx[t];
#endif

  // 1. inverse x-transform of the incoming half spectra (reversed plan)
  C y[KIN][Q1];
  if (!skip_in) {
    C v[KIN][P1];
    if (j < L / P1) {
#pragma unroll
      for (int s = 0; s < KIN; ++s) {
#if QPAT_ROWST_BULK
        const C* r0 = sp + (s * 2) * kSpecRow;
        const C* r1 = r0 + kSpecRow;
#else
        const C* r0 = spec + s * slot + (long long)j0 * a.pitch;
        const C* r1 = r0 + a.pitch;
#endif
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
#if QPAT_ROWST_BULK
    __syncthreads();                                              // staged spectra read before the first stage writes
#endif
    fft_stockham<L, G::P1, G::P2, G::P3, KIN, kRowStOneBuf>(v, y, bufA, bufB, SL, j, tw);
  } else {
#pragma unroll
    for (int s = 0; s < KIN; ++s)
#pragma unroll
      for (int r = 0; r < Q1; ++r) y[s][r] = cmake<C>((T)0, (T)0);
  }

  // adjoint sensor source M^T w_n on the two rows (A_R1, A_R1L)
  if (KIN == 1) {
    for (int i = j; i < 2 * L; i += TPT) sc[i] = (T)0;
    __syncthreads();
    if (valid) sensor_scatter_rows<T>(a, b, j0, sc, j, TPT);
  }
#if QPAT_ROWST_BULK
  row_bulk_wait(bar + 1, a.err);
#else
  cp_async_wait_all();
#endif
  __syncthreads();

  // 2. pointwise update on grid points i = j + r L/Q1 of both rows;
  //    y = FFT(conj Z) = conj(z): row j0 is Re, row j0+1 is -Im
  C o[KOUT][Q1];
  bool bad = false;
#pragma unroll
  for (int r = 0; r < Q1; ++r) {
    T u0[2] = {(T)0, (T)0}, u1[2] = {(T)0, (T)0};
    if (j < L / Q1 && valid) {
      const int i = j + r * (L / Q1);
#pragma unroll
      for (int rr = 0; rr < 2; ++rr) {
        T sv[5];
#pragma unroll
        for (int v = 0; v < 5; ++v)
          sv[v] = row_field(ph, v) >= 0 ? stage[(row_stage_slot(ph, v) * 2 + rr) * L + i] : (T)0;
        const RowIn<T> st{sv[0], sv[1], sv[2], sv[3], sv[4]};
        const T in0 = rr ? -y[0][r].y : y[0][r].x;
        const T in1 = (KIN > 1) ? (rr ? -y[KIN - 1][r].y : y[KIN - 1][r].x) : (T)0;
        const T scv = (KIN == 1) ? sc[rr * L + i] : (T)0;
        row_point<T>(a, ph, b, i, j0 + rr, in0, in1, scv, st, u0[rr], u1[rr], bad);
      }
    }
    o[0][r] = cmake<C>(u0[0], u0[1]);
    if (KOUT > 1) o[KOUT - 1][r] = cmake<C>(u1[0], u1[1]);
  }
  if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr(a.err, 1);
  if (a.flags & kSkipOutput) return;

  // 3. forward x-transform of the packed outgoing rows, split, store
  C X[KOUT][QL];
  fft_stockham<L, G::Q1, G::Q2, G::Q3, KOUT, kRowStOneBuf>(o, X, bufA, bufB, SL, j, tw);
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
      C* w0 = spec + s * slot + (long long)j0 * a.pitch;
      C* w1 = w0 + a.pitch;
      for (int k = j; 2 * k <= L; k += TPT) {
        const C Z = bufA[s * SL + spad(k)];
        const C Zm = cconj(bufA[s * SL + spad(k == 0 ? 0 : L - k)]);
        w0[k] = cscale(cadd(Z, Zm), (T)0.5);
        w1[k] = cscale(cmul_mi(csub(Z, Zm)), (T)0.5);
      }
    }
  }
}

// Per-column shared-memory stride: congruent to 16/CBW complex values mod 16
// so that the CBW columns of a half warp fall on distinct banks, and always
// an even number of complex values: the paired Stockham stages move 16-byte
// entries, so every column's buffers must start on a 16-byte boundary (for
// CBW that does not divide 16 the residue is rounded up to an even count).
__host__ __device__ constexpr int col_pad_target(int cbw) {
  return (16 / cbw) < 2 ? 2 : ((16 / cbw) & ~1);
}
template <int L, int NSX, int CBW>
__host__ __device__ constexpr int col_stride() {
  return 2 * NSX * SGeom<L>::SL + ((col_pad_target(CBW) - (2 * NSX * SGeom<L>::SL) % 16) + 16) % 16;
}

#ifndef QPAT_COL_PAIRS
#define QPAT_COL_PAIRS 1
#endif
constexpr bool kColPairs = QPAT_COL_PAIRS != 0;

// Body of the column pass for column block `blk` (CBW adjacent columns) of
// problem b, run by CBW * TPT threads; nblk = column blocks per problem (the
// sensor gather of F_C1 is strided over all of them).  Dynamic shared memory
// of the launch (col_fast_smem bytes), named by the body itself.  Every
// thread of the CTA must call it.
template <typename T, int L, int PH, int CBW>
__device__ __forceinline__ void col_body(const PropArgs<T> a, const int b, const int blk, const int nblk) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  constexpr int ph = PH, KIN = col_kin(PH), KOUT = col_kout(PH);
  typedef typename V2<T>::t C;
  typedef SGeom<L> G;
  constexpr int SL = G::SL, NSX = (KIN > KOUT ? KIN : KOUT);
  constexpr int Q1 = G::Q1, QL = G::QL;
  constexpr int CS = col_stride<L, NSX, CBW>();
  static_assert(CS % 2 == 0 && L % 2 == 0 && SL % 2 == 0, "column buffers must start on 16-byte boundaries");
  const int c = threadIdx.x % CBW;
  const int j = threadIdx.x / CBW;
  C* tws = reinterpret_cast<C*>(smem_raw);                       // W_L^m table
  C* bufA = tws + L + c * CS;
  C* bufB = bufA + NSX * SL;
  const int kx = blk * CBW + c;
  const bool valid = kx < a.nxh;
  const int kxs = valid ? kx : 0;
  C* spec = a.spec + (long long)b * a.sstride;
  const long long slot = (long long)a.ny * a.pitch;

  if (ph == F_C1) sensor_gather<T>(a, b, blk * CBW * G::TPT + threadIdx.x, nblk * CBW * G::TPT);

  C v[KIN][Q1];
  if (j < L / Q1) {
#pragma unroll
    for (int s = 0; s < KIN; ++s)
#pragma unroll
      for (int r = 0; r < Q1; ++r) v[s][r] = spec[s * slot + (long long)(j + r * (L / Q1)) * a.pitch + kxs];
  }
  // twiddles to shared memory and the symbol operands of this thread's
  // points into registers before the transforms
  for (int t = threadIdx.x; t < L; t += CBW * G::TPT) tws[t] = a.twy[t];
  ColIn<T, C> cst[QL];
#pragma unroll
  for (int r = 0; r < QL; ++r)
    cst[r] = (j < L / QL && valid) ? col_load<T, C>(a, ph, kx, j + r * (L / QL)) : ColIn<T, C>{};
  const C sx = col_sx<T, C>(a, ph, kxs);
  C X[KIN][QL];
  fft_stockham<L, G::Q1, G::Q2, G::Q3, KIN, false, kColPairs>(v, X, bufA, bufB, SL, j, tws);
  // thread j < L/QL holds X[ky = j + r L/QL]
  C o[KOUT][QL];
#pragma unroll
  for (int r = 0; r < QL; ++r) {
    C o0 = cmake<C>((T)0, (T)0), o1 = o0;
    if (j < L / QL && valid) col_apply<T, C>(ph, cst[r], sx, X[0][r], X[KIN - 1][r], o0, o1);
    o[0][r] = cconj(o0);
    if (KOUT > 1) o[KOUT - 1][r] = cconj(o1);
  }
  C Y[KOUT][Q1];
  fft_stockham<L, G::P1, G::P2, G::P3, KOUT, false, kColPairs>(o, Y, bufA, bufB, SL, j, tws);
  if (j < L / Q1 && valid) {
#pragma unroll
    for (int s = 0; s < KOUT; ++s)
#pragma unroll
      for (int r = 0; r < Q1; ++r)
        spec[s * slot + (long long)(j + r * (L / Q1)) * a.pitch + kx] = cconj(Y[s][r]);
  }
}

// The single-context column pass, with its own copy of the body of col_body
// for the same reason as row_fast_st.
template <typename T, int L, int PH>
__global__ void __launch_bounds__(SGeom<L>::CBW * SGeom<L>::TPT)
col_fast(const PropArgs<T> a) {
  constexpr int ph = PH, KIN = col_kin(PH), KOUT = col_kout(PH);
  typedef typename V2<T>::t C;
  typedef SGeom<L> G;
  constexpr int SL = G::SL, CBW = G::CBW, NSX = (KIN > KOUT ? KIN : KOUT);
  constexpr int Q1 = G::Q1, QL = G::QL;
  constexpr int CS = col_stride<L, NSX, CBW>();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int c = threadIdx.x % CBW;
  const int j = threadIdx.x / CBW;
  C* tws = reinterpret_cast<C*>(smem_raw);                       // W_L^m table
  C* bufA = tws + L + c * CS;
  C* bufB = bufA + NSX * SL;
  const int b = blockIdx.y;
  const int kx = blockIdx.x * CBW + c;
  const bool valid = kx < a.nxh;
  const int kxs = valid ? kx : 0;
  C* spec = a.spec + (long long)b * a.sstride;
  const long long slot = (long long)a.ny * a.pitch;

  if (ph == F_C1) sensor_gather<T>(a, b, blockIdx.x * blockDim.x + threadIdx.x, gridDim.x * blockDim.x);

  C v[KIN][Q1];
  if (j < L / Q1) {
#pragma unroll
    for (int s = 0; s < KIN; ++s)
#pragma unroll
      for (int r = 0; r < Q1; ++r) v[s][r] = spec[s * slot + (long long)(j + r * (L / Q1)) * a.pitch + kxs];
  }
  // twiddles to shared memory and the symbol operands of this thread's
  // points into registers before the transforms
  for (int t = threadIdx.x; t < L; t += blockDim.x) tws[t] = a.twy[t];
  ColIn<T, C> cst[QL];
#pragma unroll
  for (int r = 0; r < QL; ++r)
    cst[r] = (j < L / QL && valid) ? col_load<T, C>(a, ph, kx, j + r * (L / QL)) : ColIn<T, C>{};
  const C sx = col_sx<T, C>(a, ph, kxs);
  C X[KIN][QL];
  fft_stockham<L, G::Q1, G::Q2, G::Q3, KIN, false, kColPairs>(v, X, bufA, bufB, SL, j, tws);
  // thread j < L/QL holds X[ky = j + r L/QL]
  C o[KOUT][QL];
#pragma unroll
  for (int r = 0; r < QL; ++r) {
    C o0 = cmake<C>((T)0, (T)0), o1 = o0;
    if (j < L / QL && valid) col_apply<T, C>(ph, cst[r], sx, X[0][r], X[KIN - 1][r], o0, o1);
    o[0][r] = cconj(o0);
    if (KOUT > 1) o[KOUT - 1][r] = cconj(o1);
  }
  C Y[KOUT][Q1];
  fft_stockham<L, G::P1, G::P2, G::P3, KOUT, false, kColPairs>(o, Y, bufA, bufB, SL, j, tws);
  if (j < L / Q1 && valid) {
#pragma unroll
    for (int s = 0; s < KOUT; ++s)
#pragma unroll
      for (int r = 0; r < Q1; ++r)
        spec[s * slot + (long long)(j + r * (L / Q1)) * a.pitch + kx] = cconj(Y[s][r]);
  }
}


template <typename T, int L, int PH>
constexpr size_t row_fast_smem() {
  typedef typename V2<T>::t C;
  constexpr int KIN = row_kin(PH), KOUT = row_kout(PH), NSX = (KIN > KOUT ? KIN : KOUT);
  return (L + SGeom<L>::RP * 2 * NSX * SGeom<L>::SL) * sizeof(C) + (KIN == 1 ? SGeom<L>::RP * 2 * L * sizeof(T) : 0);
}
template <typename T, int L, int PH, int CBW = SGeom<L>::CBW>
constexpr size_t col_fast_smem() {
  typedef typename V2<T>::t C;
  constexpr int KIN = col_kin(PH), KOUT = col_kout(PH), NSX = (KIN > KOUT ? KIN : KOUT);
  return ((size_t)L + (size_t)CBW * col_stride<L, NSX, CBW>()) * sizeof(C);
}

template <typename T, int L, int PH>
void set_row_fast_attr() {
  static_assert(row_fast_st_smem<T, L, PH>() <= 227 * 1024 && row_fast_smem<T, L, PH>() <= 227 * 1024,
                "row pass shared memory above the 227 KB a CTA may use");
  if constexpr (row_staged<L>())
    cudaFuncSetAttribute(row_fast_st<T, L, PH>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)row_fast_st_smem<T, L, PH>());
  else
    cudaFuncSetAttribute(row_fast<T, L, PH>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)row_fast_smem<T, L, PH>());
}
template <typename T, int L, int PH>
void set_col_fast_attr() {
  static_assert(col_fast_smem<T, L, PH>() <= 227 * 1024, "column pass shared memory above the 227 KB a CTA may use");
  cudaFuncSetAttribute(col_fast<T, L, PH>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)col_fast_smem<T, L, PH>());
}

// Dynamic shared-memory limits of all pass kernels of length L; called at
// context creation, outside any stream capture.
template <typename T, int L>
void prepare_fast_len() {
  set_row_fast_attr<T, L, F_R1>(); set_row_fast_attr<T, L, F_R2>(); set_row_fast_attr<T, L, F_R3>();
  set_row_fast_attr<T, L, F_R3L>(); set_row_fast_attr<T, L, A_R1>(); set_row_fast_attr<T, L, A_R1L>();
  set_row_fast_attr<T, L, A_R3>(); set_row_fast_attr<T, L, A_R5>();
  set_col_fast_attr<T, L, F_C1>(); set_col_fast_attr<T, L, F_C2>(); set_col_fast_attr<T, L, F_C3>();
  set_col_fast_attr<T, L, A_C2>(); set_col_fast_attr<T, L, A_C4>(); set_col_fast_attr<T, L, A_C6>();
}

template <typename T, int L, int PH>
void run_row_fast(const PropArgs<T>& a, int batch, cudaStream_t s) {
  typedef SGeom<L> G;
  if constexpr (row_staged<L>()) {
    constexpr int RP = rp_st<L>();
    dim3 grid((a.ny / 2 + RP - 1) / RP, batch);
    row_fast_st<T, L, PH><<<grid, RP * G::TPT, row_fast_st_smem<T, L, PH>(), s>>>(a);
  } else {
    dim3 grid((a.ny / 2 + G::RP - 1) / G::RP, batch);
    row_fast<T, L, PH><<<grid, G::RP * G::TPT, row_fast_smem<T, L, PH>(), s>>>(a);
  }
}

template <typename T, int L, int PH>
void run_col_fast(const PropArgs<T>& a, int batch, cudaStream_t s) {
  typedef SGeom<L> G;
  dim3 grid((a.nxh + G::CBW - 1) / G::CBW, batch);
  col_fast<T, L, PH><<<grid, G::CBW * G::TPT, col_fast_smem<T, L, PH>(), s>>>(a);
}

// Entry points of one specialised length L (one translation unit each).
template <typename T, int L>
void launch_row_fast_len(const PropArgs<T>& a, int ph, int batch, cudaStream_t s) {
  switch (ph) {
    case F_R1: run_row_fast<T, L, F_R1>(a, batch, s); break;
    case F_R2: run_row_fast<T, L, F_R2>(a, batch, s); break;
    case F_R3: run_row_fast<T, L, F_R3>(a, batch, s); break;
    case F_R3L: run_row_fast<T, L, F_R3L>(a, batch, s); break;
    case A_R1: run_row_fast<T, L, A_R1>(a, batch, s); break;
    case A_R1L: run_row_fast<T, L, A_R1L>(a, batch, s); break;
    case A_R3: run_row_fast<T, L, A_R3>(a, batch, s); break;
    case A_R5: run_row_fast<T, L, A_R5>(a, batch, s); break;
    default: break;
  }
}

template <typename T, int L>
void launch_col_fast_len(const PropArgs<T>& a, int ph, int batch, cudaStream_t s) {
  switch (ph) {
    case F_C1: run_col_fast<T, L, F_C1>(a, batch, s); break;
    case F_C2: run_col_fast<T, L, F_C2>(a, batch, s); break;
    case F_C3: run_col_fast<T, L, F_C3>(a, batch, s); break;
    case A_C2: run_col_fast<T, L, A_C2>(a, batch, s); break;
    case A_C4: run_col_fast<T, L, A_C4>(a, batch, s); break;
    case A_C6: run_col_fast<T, L, A_C6>(a, batch, s); break;
    default: break;
  }
}

// FP32 only: in FP64 the generic passes are faster on GB300.
#define QPAT_FAST_LENGTH(L)                                                                              \
  template void prepare_fast_len<float, L>();                                                            \
  template void launch_row_fast_len<float, L>(const PropArgs<float>&, int, int, cudaStream_t);         \
  template void launch_col_fast_len<float, L>(const PropArgs<float>&, int, int, cudaStream_t);

}  // namespace qpat
