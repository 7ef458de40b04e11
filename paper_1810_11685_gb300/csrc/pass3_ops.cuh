// Per-element work of the 3D propagation passes, shared by the generic
// (runtime-radix) and the length-specialised kernels.
#pragma once
#include "prop3d.h"

namespace qpat {

__host__ __device__ constexpr int r3_kin(int ph) {
  return (ph == F_R1) ? 2 : (ph == A_R1 || ph == A_R1L) ? 1 : (ph == A_R3) ? 2 : 3;
}
__host__ __device__ constexpr int r3_kout(int ph) {
  return (ph == F_R1 || ph == F_R3L) ? 1 : (ph == F_R3 || ph == A_R1) ? 2 : 3;
}
__host__ __device__ constexpr int z3_kin(int ph) { return ph == F_C1 ? 1 : (ph == F_C3 || ph == A_C2) ? 2 : 3; }
__host__ __device__ constexpr int z3_kout(int ph) { return ph == A_C6 ? 1 : (ph == F_C3 || ph == A_C2) ? 2 : 3; }

constexpr int k3Threads = 256;

// ---- pointwise update of one grid point (i, j, k) -------------------------
template <typename T>
__device__ __forceinline__ void row3_point(const Prop3<T>& a, const int ph, const int b, const int i, const int j,
                                           const int k, const T* in, const T scv, T* out, bool& bad) {
  const long long g = ((long long)k * a.ny + j) * a.nx + i;
  const long long gb = (long long)b * a.gstride + g;
  const bool interior = i >= a.pml && i < a.pml + a.n0 && j >= a.pml && j < a.pml + a.n1 && k >= a.pml &&
                        k < a.pml + a.n2;
  const long long ii = interior ? ((long long)(k - a.pml) * a.n1 + (j - a.pml)) * a.n0 + (i - a.pml) : 0;
  const long long N = (long long)a.n0 * a.n1 * a.n2;
  out[0] = out[1] = out[2] = (T)0;
  if (ph == F_R1) {
    // eq. num-p with sum_i rho_i over three components
    const T r = a.rx[gb] + a.ry[gb] + a.rz[gb];
    const T p = a.Cc[g] * ((r - a.eta[g] * in[0]) + a.tau[g] * in[1]);
    a.pbuf[gb] = p;
    bad |= !isfinite(p);
    out[0] = p;
  } else if (ph == F_R2) {
    // eq. num-vel per axis
    const T sx = a.asx[i], sy = a.asy[j], sz = a.asz[k];
    const T vx = sx * (sx * a.vx[gb] - a.dtrsx[g] * in[0]);
    const T vy = sy * (sy * a.vy[gb] - a.dtrsy[g] * in[1]);
    const T vz = sz * (sz * a.vz[gb] - a.dtrsz[g] * in[2]);
    a.vx[gb] = vx;
    a.vy[gb] = vy;
    a.vz[gb] = vz;
    out[0] = vx;
    out[1] = vy;
    out[2] = vz;
  } else if (ph == F_R3 || ph == F_R3L) {
    // eq. num-rho with the additive source of eq. s1, dt s_i = P0 / (2 d c^2), d = 3
    T q = (T)0;
    if ((a.flags & kSource) && interior) q = a.io->p0[(long long)b * N + ii] / ((T)6 * a.Cc[g]);
    const T ax = a.ax[i], ay = a.ay[j], az = a.az[k], r0 = a.rho0[g];
    const T rx = ax * (ax * a.rx[gb] - a.dt * r0 * in[0]) + q;
    const T ry = ay * (ay * a.ry[gb] - a.dt * r0 * in[1]) + q;
    const T rz = az * (az * a.rz[gb] - a.dt * r0 * in[2]) + q;
    a.rx[gb] = rx;
    a.ry[gb] = ry;
    a.rz[gb] = rz;
    if (ph == F_R3) {
      out[0] = rx + ry + rz;
      out[1] = r0 * (ax * in[0] + ay * in[1] + az * in[2]);
    } else {
      const T p = a.Cc[g] * (rx + ry + rz);
      a.pbuf[gb] = p;
      bad |= !isfinite(p);
      out[0] = p;
    }
  } else if (ph == A_R1) {
    const T Cp = a.Cc[g] * (in[0] + scv);
    a.pbuf[gb] = Cp;
    out[0] = a.eta[g] * Cp;
    out[1] = a.tau[g] * Cp;
  } else if (ph == A_R1L || ph == A_R3) {
    T Cp, ya = (T)0;
    if (ph == A_R1L) {
      Cp = a.Cc[g] * (in[0] + scv);
    } else {
      Cp = a.pbuf[gb];
      ya = in[1];
    }
    const T rpart = (ph == A_R1L) ? Cp : Cp - in[0];
    const T A[3] = {a.ax[i], a.ay[j], a.az[k]};
    T* R[3] = {a.rx, a.ry, a.rz};
    const T r0 = a.rho0[g];
    T sum = (T)0;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const T rt = R[c][gb] + rpart;
      out[c] = r0 * A[c] * (ya - a.dt * rt);
      R[c][gb] = A[c] * A[c] * rt;
      sum += rt;
    }
    bad |= !isfinite(sum);
    if (interior && (a.flags & (kAccWrite | kAccAdd))) {
      T* dst = a.io->p0adj + (long long)b * N + ii;
      const T val = sum / ((T)6 * a.Cc[g]);
      if (a.flags & kAccWrite) *dst = val;
      else *dst += val;
    }
  } else if (ph == A_R5) {
    const T S[3] = {a.asx[i], a.asy[j], a.asz[k]};
    const T D[3] = {a.dtrsx[g], a.dtrsy[g], a.dtrsz[g]};
    T* V[3] = {a.vx, a.vy, a.vz};
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const T vt = V[c][gb] + in[c];
      V[c][gb] = S[c] * S[c] * vt;
      out[c] = S[c] * D[c] * vt;
    }
  }
}

// ---- z pass symbols ----------------------------------------------------------
// Operands of the symbol at half-spectrum point (kx, ky, kz): kappa (or the
// fractional-Laplacian powers k^(y-1), k^(y-2)) and the z shift factor.
template <typename T, typename C>
struct Z3In {
  T k1, k2;
  C sz;
};

template <typename T, typename C>
__device__ __forceinline__ Z3In<T, C> z3_load(const Prop3<T>& a, const int ph, const int kx, const int ky,
                                              const int kz) {
  const long long t = ((long long)kz * a.ny + ky) * a.nxh + kx;
  Z3In<T, C> r;
  r.k1 = (T)0;
  r.k2 = (T)0;
  r.sz = cmake<C>((T)0, (T)0);
  if (ph == F_C3 || ph == A_C2) {
    r.k1 = a.kp1[t];
    r.k2 = a.kp2[t];
  } else {
    r.k1 = a.kap[t];
    r.sz = (ph == F_C1 || ph == A_C6) ? a.shzp[kz] : a.shzm[kz];
  }
  return r;
}
template <typename T, typename C>
__device__ __forceinline__ C z3_sx(const Prop3<T>& a, const int ph, const int kx) {
  return (ph == F_C1 || ph == A_C6) ? a.shxp[kx] : a.shxm[kx];
}
template <typename T, typename C>
__device__ __forceinline__ C z3_sy(const Prop3<T>& a, const int ph, const int ky) {
  return (ph == F_C1 || ph == A_C6) ? a.shyp[ky] : a.shym[ky];
}

// The k-space symbol of a z pass on the forward-transformed slots X.
template <typename T, typename C>
__device__ __forceinline__ void z3_apply(const int ph, const Z3In<T, C>& st, const C sx, const C sy, const C (&X)[3],
                                         C (&o)[3]) {
  o[0] = o[1] = o[2] = cmake<C>((T)0, (T)0);
  if (ph == F_C1) {          // d/dr_i^+ of p, i = x, y, z (eq. grr)
    o[0] = cscale(cmul(sx, X[0]), st.k1);
    o[1] = cscale(cmul(sy, X[0]), st.k1);
    o[2] = cscale(cmul(st.sz, X[0]), st.k1);
  } else if (ph == F_C2) {   // d/dr_i^- v_i
    o[0] = cscale(cmul(sx, X[0]), st.k1);
    o[1] = cscale(cmul(sy, X[1]), st.k1);
    o[2] = cscale(cmul(st.sz, X[2]), st.k1);
  } else if (ph == F_C3 || ph == A_C2) {   // Y_dis, Y_abs
    o[0] = cscale(X[0], st.k1);
    o[1] = cscale(X[1], st.k2);
  } else if (ph == A_C4) {   // (d/dr_i^-)^T
    o[0] = cscale(cmul(cconj(sx), X[0]), st.k1);
    o[1] = cscale(cmul(cconj(sy), X[1]), st.k1);
    o[2] = cscale(cmul(cconj(st.sz), X[2]), st.k1);
  } else {                   // A_C6: -sum_i (d/dr_i^+)^T
    o[0] = cscale(cadd(cadd(cmul(cconj(sx), X[0]), cmul(cconj(sy), X[1])), cmul(cconj(st.sz), X[2])), -st.k1);
  }
}

// eq. num-m, trilinear: samples of p_n for problem b
template <typename T>
__device__ __forceinline__ void gather3(const Prop3<T>& a, int b, int first, int stride) {
  const T* pb = a.pbuf + (long long)b * a.gstride;
  T* dn = a.io->data + ((long long)b * a.nt + a.n) * a.ns;
  for (int s = first; s < a.ns; s += stride) {
    T acc = (T)0;
#pragma unroll
    for (int c = 0; c < 8; ++c) acc += a.sw[8 * s + c] * pb[a.sidx[8 * s + c]];
    dn[s] = acc;
  }
}

// M^T w_n for grid rows r0 = k ny + j0 and r0 + 1 into sc[rr * nx + i]
// (deterministic: each point sums its own entries).  Threads tid0..tid0+nth-1.
template <typename T>
__device__ __forceinline__ void sensor_scatter_rows3(const Prop3<T>& a, int b, int r0, T* sc, int tid, int nth) {
  const T* wn = a.io->w + ((long long)b * a.nt + a.n) * a.ns;
  for (int rr = 0; rr < 2; ++rr) {
    const int r = r0 + rr;
    for (int q = a.rowptr[r] + tid; q < a.rowptr[r + 1]; q += nth) {
      T acc = (T)0;
      for (int e = a.pent[q]; e < a.pent[q + 1]; ++e) acc += a.ew[e] * wn[a.esens[e]];
      sc[rr * a.nx + a.pcol[q]] = acc;
    }
  }
}

}  // namespace qpat
