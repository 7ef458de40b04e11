// Per-element work of the propagation passes, shared by the generic
// (any FFT length) and the length-specialised kernels.
#pragma once
#include "qpat_internal.h"

namespace qpat {

// A of the register-FFT split L = A * B used for each specialised FFT
// extent (0: the extent uses the generic shared-memory passes).
__host__ __device__ constexpr int fast_split_a(int L) {
  return L == 24 ? 4 : L == 40 ? 5 : L == 48 ? 6 : L == 54 ? 6 : L == 56 ? 7 : L == 168 ? 12
       : L == 288 ? 16 : L == 432 ? 24 : L == 576 ? 24 : 0;
}

__host__ __device__ constexpr int row_kin(int ph) { return (ph == A_R1 || ph == A_R1L) ? 1 : 2; }
__host__ __device__ constexpr int row_kout(int ph) { return (ph == F_R1 || ph == F_R3L) ? 1 : 2; }
__host__ __device__ constexpr int col_kin(int ph) { return ph == F_C1 ? 1 : 2; }
__host__ __device__ constexpr int col_kout(int ph) { return ph == A_C6 ? 1 : 2; }

// Operands a row pass needs at one grid point, loaded before the transforms
// so that their latency overlaps the FFT (row_load), then consumed by
// row_point.  The meaning of v0..v4 depends on the phase.
template <typename T>
struct RowIn {
  T v0, v1, v2, v3, v4;
};

template <typename T>
__device__ __forceinline__ RowIn<T> row_load(const PropArgs<T>& a, const int ph, const int b, const int i,
                                             const int j) {
  const long long g = (long long)j * a.nx + i;
  const long long gb = (long long)b * a.gstride + g;
  RowIn<T> r;
  r.v0 = r.v1 = r.v2 = r.v3 = r.v4 = (T)0;
  if (ph == F_R1) {
    r.v0 = a.rx[gb]; r.v1 = a.ry[gb]; r.v2 = a.Cc[g]; r.v3 = a.eta[g]; r.v4 = a.tau[g];
  } else if (ph == F_R2 || ph == A_R5) {
    r.v0 = a.vx[gb]; r.v1 = a.vy[gb]; r.v2 = a.dtrsx[g]; r.v3 = a.dtrsy[g];
  } else if (ph == F_R3 || ph == F_R3L) {
    // c^2 only enters through the source (F_R3) or the pressure (F_R3L)
    r.v0 = a.rx[gb]; r.v1 = a.ry[gb]; r.v2 = a.rho0[g];
    if (ph == F_R3L || (a.flags & kSource)) r.v3 = a.Cc[g];
  } else if (ph == A_R1) {
    r.v2 = a.Cc[g]; r.v3 = a.eta[g]; r.v4 = a.tau[g];
  } else if (ph == A_R1L) {
    r.v0 = a.rx[gb]; r.v1 = a.ry[gb]; r.v2 = a.rho0[g]; r.v3 = a.Cc[g];
  } else if (ph == A_R3) {
    // c^2 only enters through the source adjoint (accumulation steps)
    r.v0 = a.rx[gb]; r.v1 = a.ry[gb]; r.v2 = a.rho0[g]; r.v4 = a.pbuf[gb];
    if (a.flags & (kAccWrite | kAccAdd)) r.v3 = a.Cc[g];
  }
  return r;
}

// 16-byte asynchronous global -> shared copy (both addresses 16-byte aligned).
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(s), "l"(gmem) : "memory");
}
// Commit this thread's outstanding cp.async copies and wait for all of them.
__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.commit_group;\n\tcp.async.wait_group 0;" ::: "memory");
}

// ---- bulk copies (cp.async.bulk) completing on a shared-memory mbarrier ------
__device__ __forceinline__ unsigned smem_u32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void mbar_init(unsigned long long* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
// Arrive once and add `bytes` to the transfer count the phase waits for.
__device__ __forceinline__ void mbar_arrive_expect_tx(unsigned long long* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}
// Global -> shared copy of `bytes` (a multiple of 16; both addresses 16-byte
// aligned) by the bulk-copy unit, counted on `bar` when it lands.
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, unsigned bytes, unsigned long long* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_u32(dst)),
               "l"(src), "r"(bytes), "r"(smem_u32(bar))
               : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(unsigned long long* bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Wait for phase `parity` of `bar` with a bounded number of polls (each poll
// may suspend the thread for a while); false when the limit ran out.
__device__ __forceinline__ bool mbar_wait_bounded(unsigned long long* bar, unsigned parity) {
  for (int i = 0; i < (1 << 22); ++i)
    if (mbar_try_wait(bar, parity)) return true;
  return false;
}

// Pointwise update of one grid point (i, j) of problem b in a row pass.
// in0/in1: the incoming fields after the inverse transforms (already
// normalised); scv: M^T w at this point (adjoint sensor source, A_R1*);
// st: the operands from row_load.  Writes the outgoing fields to out0/out1
// (to be forward transformed) and the updated state to global memory.
template <typename T>
__device__ __forceinline__ void row_point(const PropArgs<T>& a, const int ph, const int b, const int i, const int j,
                                          const T in0, const T in1, const T scv, const RowIn<T>& st, T& out0,
                                          T& out1, bool& bad) {
  const long long g = (long long)j * a.nx + i;
  const long long gb = (long long)b * a.gstride;
  const bool interior = (i >= a.pml) && (i < a.pml + a.n0) && (j >= a.pml) && (j < a.pml + a.n1);
  const long long ii = interior ? (long long)(j - a.pml) * a.n0 + (i - a.pml) : 0;
  out0 = (T)0;
  out1 = (T)0;
  if (ph == F_R1) {
    // eq. num-p: p = c^2 [ (I - eta Y_dis) sum rho_i + tau Y_abs u ]
    const T r = st.v0 + st.v1;
    const T p = st.v2 * ((r - st.v3 * in0) + st.v4 * in1);
    a.pbuf[gb + g] = p;
    bad |= !isfinite(p);
    out0 = p;
  } else if (ph == F_R2) {
    // eq. num-vel: v_i <- A_i (A_i v_i - dt/rho_i d/dr_i^+ p)
    const T sx = a.asx[i], sy = a.asy[j];
    const T vx = sx * (sx * st.v0 - st.v2 * in0);
    const T vy = sy * (sy * st.v1 - st.v3 * in1);
    a.vx[gb + g] = vx;
    a.vy[gb + g] = vy;
    out0 = vx;
    out1 = vy;
  } else if (ph == F_R3 || ph == F_R3L) {
    // eq. num-rho with the additive source of eq. s1 (dt s_i = P0 / (2 d c^2))
    T q = (T)0;
    if ((a.flags & kSource) && interior) q = a.io->p0[(long long)b * a.n0 * a.n1 + ii] / ((T)4 * st.v3);
    const T ax = a.ax[i], ay = a.ay[j], r0 = st.v2;
    const T rx = ax * (ax * st.v0 - a.dt * r0 * in0) + q;
    const T ry = ay * (ay * st.v1 - a.dt * r0 * in1) + q;
    a.rx[gb + g] = rx;
    a.ry[gb + g] = ry;
    if (ph == F_R3) {
      out0 = rx + ry;                            // sum_i rho_i
      out1 = ax * r0 * in0 + ay * r0 * in1;      // sum_i A_i rho0 d/dr_i^- v_i
    } else {
      const T p = st.v3 * (rx + ry);
      a.pbuf[gb + g] = p;
      bad |= !isfinite(p);
      out0 = p;
    }
  } else if (ph == A_R1) {
    // transpose of num-m and of the pressure update: C p-bar feeds Y_dis^T, Y_abs^T
    const T Cp = st.v2 * (in0 + scv);
    a.pbuf[gb + g] = Cp;
    out0 = st.v3 * Cp;
    out1 = st.v4 * Cp;
  } else if (ph == A_R1L || ph == A_R3) {
    // transpose of the density update (and of the source injection)
    T Cp, ya = (T)0;
    if (ph == A_R1L) {
      Cp = st.v3 * (in0 + scv);
    } else {
      Cp = st.v4;
      ya = in1;
    }
    const T rpart = (ph == A_R1L) ? Cp : Cp - in0;   // (I - Y_dis eta) C p-bar
    const T ax = a.ax[i], ay = a.ay[j], r0 = st.v2;
    const T rtx = st.v0 + rpart;
    const T rty = st.v1 + rpart;
    out0 = r0 * ax * (ya - a.dt * rtx);
    out1 = r0 * ay * (ya - a.dt * rty);
    a.rx[gb + g] = ax * ax * rtx;
    a.ry[gb + g] = ay * ay * rty;
    bad |= !isfinite(rtx + rty);
    if (interior && (a.flags & (kAccWrite | kAccAdd))) {
      T* dst = a.io->p0adj + (long long)b * a.n0 * a.n1 + ii;
      const T val = (rtx + rty) / ((T)4 * st.v3);
      if (a.flags & kAccWrite) *dst = val;
      else *dst += val;
    }
  } else if (ph == A_R5) {
    // transpose of the velocity update
    const T sx = a.asx[i], sy = a.asy[j];
    const T vtx = st.v0 + in0;
    const T vty = st.v1 + in1;
    a.vx[gb + g] = sx * sx * vtx;
    a.vy[gb + g] = sy * sy * vty;
    out0 = sx * st.v2 * vtx;
    out1 = sy * st.v3 * vty;
  }
}

// Operands of a column pass at one half-spectrum point, loaded early.
template <typename T, typename C>
struct ColIn {
  T k1, k2;      // kappa (or |k|^(y-1)) and |k|^(y-2)
  C sy;          // y shift-derivative factor
};

template <typename T, typename C>
__device__ __forceinline__ ColIn<T, C> col_load(const PropArgs<T>& a, const int ph, const int kx, const int ky) {
  const long long t = (long long)ky * a.nxh + kx;
  ColIn<T, C> r;
  r.k1 = (T)0;
  r.k2 = (T)0;
  r.sy = cmake<C>((T)0, (T)0);
  if (ph == F_C3 || ph == A_C2) {
    r.k1 = a.kp1[t];
    r.k2 = a.kp2[t];
  } else {
    r.k1 = a.kap[t];
    r.sy = (ph == F_C1 || ph == A_C6) ? a.shyp[ky] : a.shym[ky];
  }
  return r;
}

// Spectral symbol of a column pass from preloaded operands; sx is the x
// shift-derivative factor of the column (shxp or shxm by phase).
template <typename T, typename C>
__device__ __forceinline__ void col_apply(const int ph, const ColIn<T, C>& st, const C sx, const C X0, const C X1,
                                          C& o0, C& o1) {
  if (ph == F_C1) {          // d/dr_x^+, d/dr_y^+ of p (eq. grr)
    o0 = cscale(cmul(sx, X0), st.k1);
    o1 = cscale(cmul(st.sy, X0), st.k1);
  } else if (ph == F_C2) {   // d/dr_x^- v_x, d/dr_y^- v_y
    o0 = cscale(cmul(sx, X0), st.k1);
    o1 = cscale(cmul(st.sy, X1), st.k1);
  } else if (ph == F_C3 || ph == A_C2) {   // Y_dis, Y_abs (real, even symbols)
    o0 = cscale(X0, st.k1);
    o1 = cscale(X1, st.k2);
  } else if (ph == A_C4) {   // (d/dr_i^-)^T: conjugate symbols
    o0 = cscale(cmul(cconj(sx), X0), st.k1);
    o1 = cscale(cmul(cconj(st.sy), X1), st.k1);
  } else {                   // A_C6: -sum_i (d/dr_i^+)^T
    o0 = cscale(cadd(cmul(cconj(sx), X0), cmul(cconj(st.sy), X1)), -st.k1);
    o1 = o0;
  }
}

template <typename T, typename C>
__device__ __forceinline__ C col_sx(const PropArgs<T>& a, const int ph, const int kx) {
  return (ph == F_C1 || ph == A_C6) ? a.shxp[kx] : a.shxm[kx];
}

// Spectral symbol of a column pass at half-spectrum point (kx, ky).
template <typename T, typename C>
__device__ __forceinline__ void col_point(const PropArgs<T>& a, const int ph, const int kx, const int ky, const C X0,
                                          const C X1, C& o0, C& o1) {
  const ColIn<T, C> st = col_load<T, C>(a, ph, kx, ky);
  col_apply<T, C>(ph, st, col_sx<T, C>(a, ph, kx), X0, X1, o0, o1);
}

// M^T w_n for the grid points of rows j0, j0 + 1 into sc[rr * nx + i]
// (deterministic: each point sums its own entries).  Threads tid0..tid0+nth-1.
template <typename T>
__device__ __forceinline__ void sensor_scatter_rows(const PropArgs<T>& a, int b, int j0, T* sc, int tid, int nth) {
  const T* wn = a.io->w + ((long long)b * a.nt + a.n) * a.ns;
  for (int rr = 0; rr < 2; ++rr) {
    const int j = j0 + rr;
    for (int q = a.rowptr[j] + tid; q < a.rowptr[j + 1]; q += nth) {
      T acc = (T)0;
      for (int e = a.pent[q]; e < a.pent[q + 1]; ++e) acc += a.ew[e] * wn[a.esens[e]];
      sc[rr * a.nx + a.pcol[q]] = acc;
    }
  }
}

// eq. num-m: bilinear samples of p_n for problem b, sensors strided over the grid.
template <typename T>
__device__ __forceinline__ void sensor_gather(const PropArgs<T>& a, int b, int first, int stride) {
  const T* pb = a.pbuf + (long long)b * a.gstride;
  T* dn = a.io->data + ((long long)b * a.nt + a.n) * a.ns;
  for (int s = first; s < a.ns; s += stride) {
    T acc = (T)0;
#pragma unroll
    for (int c = 0; c < 4; ++c) acc += a.sw[4 * s + c] * pb[a.sidx[4 * s + c]];
    dn[s] = acc;
  }
}

}  // namespace qpat
