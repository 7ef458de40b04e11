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

// Pointwise update of one grid point (i, j) of problem b in a row pass.
// in0/in1: the incoming fields after the inverse transforms (already
// normalised); scv: M^T w at this point (adjoint sensor source, A_R1*).
// Writes the outgoing fields to out0/out1 (to be forward transformed).
template <typename T>
__device__ __forceinline__ void row_point(const PropArgs<T>& a, const int ph, const int b, const int i, const int j,
                                          const T in0, const T in1, const T scv, T& out0, T& out1, bool& bad) {
  const long long g = (long long)j * a.nx + i;
  const long long gb = (long long)b * a.gstride;
  const bool interior = (i >= a.pml) && (i < a.pml + a.n0) && (j >= a.pml) && (j < a.pml + a.n1);
  const long long ii = interior ? (long long)(j - a.pml) * a.n0 + (i - a.pml) : 0;
  out0 = (T)0;
  out1 = (T)0;
  if (ph == F_R1) {
    // eq. num-p: p = c^2 [ (I - eta Y_dis) sum rho_i + tau Y_abs u ]
    const T r = a.rx[gb + g] + a.ry[gb + g];
    const T p = a.Cc[g] * ((r - a.eta[g] * in0) + a.tau[g] * in1);
    a.pbuf[gb + g] = p;
    bad |= !isfinite(p);
    out0 = p;
  } else if (ph == F_R2) {
    // eq. num-vel: v_i <- A_i (A_i v_i - dt/rho_i d/dr_i^+ p)
    const T sx = a.asx[i], sy = a.asy[j];
    const T vx = sx * (sx * a.vx[gb + g] - a.dtrsx[g] * in0);
    const T vy = sy * (sy * a.vy[gb + g] - a.dtrsy[g] * in1);
    a.vx[gb + g] = vx;
    a.vy[gb + g] = vy;
    out0 = vx;
    out1 = vy;
  } else if (ph == F_R3 || ph == F_R3L) {
    // eq. num-rho with the additive source of eq. s1 (dt s_i = P0 / (2 d c^2))
    T q = (T)0;
    if ((a.flags & kSource) && interior) q = a.p0[(long long)b * a.n0 * a.n1 + ii] / ((T)4 * a.Cc[g]);
    const T ax = a.ax[i], ay = a.ay[j], r0 = a.rho0[g];
    const T rx = ax * (ax * a.rx[gb + g] - a.dt * r0 * in0) + q;
    const T ry = ay * (ay * a.ry[gb + g] - a.dt * r0 * in1) + q;
    a.rx[gb + g] = rx;
    a.ry[gb + g] = ry;
    if (ph == F_R3) {
      out0 = rx + ry;                            // sum_i rho_i
      out1 = ax * r0 * in0 + ay * r0 * in1;      // sum_i A_i rho0 d/dr_i^- v_i
    } else {
      const T p = a.Cc[g] * (rx + ry);
      a.pbuf[gb + g] = p;
      bad |= !isfinite(p);
      out0 = p;
    }
  } else if (ph == A_R1) {
    // transpose of num-m and of the pressure update: C p-bar feeds Y_dis^T, Y_abs^T
    const T Cp = a.Cc[g] * (in0 + scv);
    a.pbuf[gb + g] = Cp;
    out0 = a.eta[g] * Cp;
    out1 = a.tau[g] * Cp;
  } else if (ph == A_R1L || ph == A_R3) {
    // transpose of the density update (and of the source injection)
    T Cp, ya = (T)0;
    if (ph == A_R1L) {
      Cp = a.Cc[g] * (in0 + scv);
    } else {
      Cp = a.pbuf[gb + g];
      ya = in1;
    }
    const T rpart = (ph == A_R1L) ? Cp : Cp - in0;   // (I - Y_dis eta) C p-bar
    const T ax = a.ax[i], ay = a.ay[j], r0 = a.rho0[g];
    const T rtx = a.rx[gb + g] + rpart;
    const T rty = a.ry[gb + g] + rpart;
    out0 = r0 * ax * (ya - a.dt * rtx);
    out1 = r0 * ay * (ya - a.dt * rty);
    a.rx[gb + g] = ax * ax * rtx;
    a.ry[gb + g] = ay * ay * rty;
    bad |= !isfinite(rtx + rty);
    if (interior && (a.flags & (kAccWrite | kAccAdd))) {
      T* dst = a.p0adj + (long long)b * a.n0 * a.n1 + ii;
      const T val = (rtx + rty) / ((T)4 * a.Cc[g]);
      if (a.flags & kAccWrite) *dst = val;
      else *dst += val;
    }
  } else if (ph == A_R5) {
    // transpose of the velocity update
    const T sx = a.asx[i], sy = a.asy[j];
    const T vtx = a.vx[gb + g] + in0;
    const T vty = a.vy[gb + g] + in1;
    a.vx[gb + g] = sx * sx * vtx;
    a.vy[gb + g] = sy * sy * vty;
    out0 = sx * a.dtrsx[g] * vtx;
    out1 = sy * a.dtrsy[g] * vty;
  }
}

// Spectral symbol of a column pass at half-spectrum point (kx, ky):
// o0/o1 from the y-transformed inputs X0/X1.
template <typename T, typename C>
__device__ __forceinline__ void col_point(const PropArgs<T>& a, const int ph, const int kx, const int ky, const C X0,
                                          const C X1, C& o0, C& o1) {
  const long long t = (long long)ky * a.nxh + kx;
  if (ph == F_C1) {          // d/dr_x^+, d/dr_y^+ of p (eq. grr)
    const T k = a.kap[t];
    o0 = cscale(cmul(a.shxp[kx], X0), k);
    o1 = cscale(cmul(a.shyp[ky], X0), k);
  } else if (ph == F_C2) {   // d/dr_x^- v_x, d/dr_y^- v_y
    const T k = a.kap[t];
    o0 = cscale(cmul(a.shxm[kx], X0), k);
    o1 = cscale(cmul(a.shym[ky], X1), k);
  } else if (ph == F_C3 || ph == A_C2) {   // Y_dis, Y_abs (real, even symbols)
    o0 = cscale(X0, a.kp1[t]);
    o1 = cscale(X1, a.kp2[t]);
  } else if (ph == A_C4) {   // (d/dr_i^-)^T: conjugate symbols
    const T k = a.kap[t];
    o0 = cscale(cmul(cconj(a.shxm[kx]), X0), k);
    o1 = cscale(cmul(cconj(a.shym[ky]), X1), k);
  } else {                   // A_C6: -sum_i (d/dr_i^+)^T
    const T k = a.kap[t];
    o0 = cscale(cadd(cmul(cconj(a.shxp[kx]), X0), cmul(cconj(a.shyp[ky]), X1)), -k);
    o1 = o0;
  }
}

// M^T w_n for the grid points of rows j0, j0 + 1 into sc[rr * nx + i]
// (deterministic: each point sums its own entries).  Threads tid0..tid0+nth-1.
template <typename T>
__device__ __forceinline__ void sensor_scatter_rows(const PropArgs<T>& a, int b, int j0, T* sc, int tid, int nth) {
  const T* wn = a.w + ((long long)b * a.nt + a.n) * a.ns;
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
  T* dn = a.data + ((long long)b * a.nt + a.n) * a.ns;
  for (int s = first; s < a.ns; s += stride) {
    T acc = (T)0;
#pragma unroll
    for (int c = 0; c < 4; ++c) acc += a.sw[4 * s + c] * pb[a.sidx[4 * s + c]];
    dn[s] = acc;
  }
}

}  // namespace qpat
