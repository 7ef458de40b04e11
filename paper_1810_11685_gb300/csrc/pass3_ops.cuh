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

// ---- operands of the pointwise updates --------------------------------------
// Per-point fields a row pass reads: state of problem b (v_i, rho_i, the
// sampling buffer) and medium diagonals shared by the batch.
enum R3Field : int { FVX, FVY, FVZ, FRX, FRY, FRZ, FPB, MCC, MRHO, MDX, MDY, MDZ, META, MTAU, kR3Fields };

// Fields read by the update of phase ph, in staging order (-1: unused slot).
__host__ __device__ constexpr int r3_field(int ph, int slot) {
  switch (ph) {
    case F_R1: { const int f[6] = {FRX, FRY, FRZ, MCC, META, MTAU}; return f[slot]; }
    case F_R2: case A_R5: { const int f[6] = {FVX, FVY, FVZ, MDX, MDY, MDZ}; return f[slot]; }
    case F_R3: case F_R3L: case A_R1L: { const int f[6] = {FRX, FRY, FRZ, MRHO, MCC, -1}; return f[slot]; }
    case A_R1: { const int f[6] = {MCC, META, MTAU, -1, -1, -1}; return f[slot]; }
    case A_R3: { const int f[6] = {FRX, FRY, FRZ, MRHO, FPB, MCC}; return f[slot]; }
    default: return -1;
  }
}
__host__ __device__ constexpr int r3_nfields(int ph) {
  int n = 0;
  for (int s = 0; s < 6; ++s) n += r3_field(ph, s) >= 0 ? 1 : 0;
  return n;
}
__host__ __device__ constexpr int r3_slot(int ph, int field) {
  for (int s = 0; s < 6; ++s)
    if (r3_field(ph, s) == field) return s;
  return -1;
}

// Row-start pointer of field f for grid row r = k ny + j of problem b.
template <typename T>
__device__ __forceinline__ const T* r3_row(const Prop3<T>& a, int f, int b, long long r) {
  const long long o = r * a.nx, ob = (long long)b * a.gstride + o;
  switch (f) {
    case FVX: return a.vx + ob;
    case FVY: return a.vy + ob;
    case FVZ: return a.vz + ob;
    case FRX: return a.rx + ob;
    case FRY: return a.ry + ob;
    case FRZ: return a.rz + ob;
    case FPB: return a.pbuf + ob;
    case MCC: return a.Cc + o;
    case MRHO: return a.rho0 + o;
    case MDX: return a.dtrsx + o;
    case MDY: return a.dtrsy + o;
    case MDZ: return a.dtrsz + o;
    case META: return a.eta + o;
    default: return a.tau + o;
  }
}

// Operand loader reading global memory at grid point g of problem b.
template <typename T>
struct R3Global {
  const Prop3<T>& a;
  long long g, gb;
  __device__ __forceinline__ T operator()(int f) const {
    switch (f) {
      case FVX: return a.vx[gb];
      case FVY: return a.vy[gb];
      case FVZ: return a.vz[gb];
      case FRX: return a.rx[gb];
      case FRY: return a.ry[gb];
      case FRZ: return a.rz[gb];
      case FPB: return a.pbuf[gb];
      case MCC: return a.Cc[g];
      case MRHO: return a.rho0[g];
      case MDX: return a.dtrsx[g];
      case MDY: return a.dtrsy[g];
      case MDZ: return a.dtrsz[g];
      case META: return a.eta[g];
      default: return a.tau[g];
    }
  }
};

// ---- pointwise update of one grid point (i, j, k) -------------------------
// ld(f) returns field f at this point (from global memory or a staged copy);
// results go to global memory and to out[] (the fields to be transformed).
template <typename T, class Ld>
__device__ __forceinline__ void row3_point(const Prop3<T>& a, const int ph, const int b, const int i, const int j,
                                           const int k, const T* in, const T scv, const Ld& ld, T* out, bool& bad) {
  const long long g = ((long long)k * a.ny + j) * a.nx + i;
  const long long gb = (long long)b * a.gstride + g;
  const bool interior = i >= a.pml && i < a.pml + a.n0 && j >= a.pml && j < a.pml + a.n1 && k >= a.pml &&
                        k < a.pml + a.n2;
  const long long ii = interior ? ((long long)(k - a.pml) * a.n1 + (j - a.pml)) * a.n0 + (i - a.pml) : 0;
  const long long N = (long long)a.n0 * a.n1 * a.n2;
  out[0] = out[1] = out[2] = (T)0;
  if (ph == F_R1) {
    // eq. num-p with sum_i rho_i over three components
    const T r = ld(FRX) + ld(FRY) + ld(FRZ);
    const T p = ld(MCC) * ((r - ld(META) * in[0]) + ld(MTAU) * in[1]);
    a.pbuf[gb] = p;
    bad |= !isfinite(p);
    out[0] = p;
  } else if (ph == F_R2) {
    // eq. num-vel per axis
    const T sx = a.asx[i], sy = a.asy[j], sz = a.asz[k];
    const T vx = sx * (sx * ld(FVX) - ld(MDX) * in[0]);
    const T vy = sy * (sy * ld(FVY) - ld(MDY) * in[1]);
    const T vz = sz * (sz * ld(FVZ) - ld(MDZ) * in[2]);
    a.vx[gb] = vx;
    a.vy[gb] = vy;
    a.vz[gb] = vz;
    out[0] = vx;
    out[1] = vy;
    out[2] = vz;
  } else if (ph == F_R3 || ph == F_R3L) {
    // eq. num-rho with the additive source of eq. s1, dt s_i = P0 / (2 d c^2), d = 3
    T q = (T)0;
    if ((a.flags & kSource) && interior) q = a.io->p0[(long long)b * N + ii] / ((T)6 * ld(MCC));
    const T ax = a.ax[i], ay = a.ay[j], az = a.az[k], r0 = ld(MRHO);
    const T rx = ax * (ax * ld(FRX) - a.dt * r0 * in[0]) + q;
    const T ry = ay * (ay * ld(FRY) - a.dt * r0 * in[1]) + q;
    const T rz = az * (az * ld(FRZ) - a.dt * r0 * in[2]) + q;
    a.rx[gb] = rx;
    a.ry[gb] = ry;
    a.rz[gb] = rz;
    if (ph == F_R3) {
      out[0] = rx + ry + rz;
      out[1] = r0 * (ax * in[0] + ay * in[1] + az * in[2]);
    } else {
      const T p = ld(MCC) * (rx + ry + rz);
      a.pbuf[gb] = p;
      bad |= !isfinite(p);
      out[0] = p;
    }
  } else if (ph == A_R1) {
    const T Cp = ld(MCC) * (in[0] + scv);
    a.pbuf[gb] = Cp;
    out[0] = ld(META) * Cp;
    out[1] = ld(MTAU) * Cp;
  } else if (ph == A_R1L || ph == A_R3) {
    T Cp, ya = (T)0;
    if (ph == A_R1L) {
      Cp = ld(MCC) * (in[0] + scv);
    } else {
      Cp = ld(FPB);
      ya = in[1];
    }
    const T rpart = (ph == A_R1L) ? Cp : Cp - in[0];
    const T A[3] = {a.ax[i], a.ay[j], a.az[k]};
    const T Rin[3] = {ld(FRX), ld(FRY), ld(FRZ)};
    T* R[3] = {a.rx, a.ry, a.rz};
    const T r0 = ld(MRHO);
    T sum = (T)0;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const T rt = Rin[c] + rpart;
      out[c] = r0 * A[c] * (ya - a.dt * rt);
      R[c][gb] = A[c] * A[c] * rt;
      sum += rt;
    }
    bad |= !isfinite(sum);
    if (interior && (a.flags & (kAccWrite | kAccAdd))) {
      T* dst = a.io->p0adj + (long long)b * N + ii;
      const T val = sum / ((T)6 * ld(MCC));
      if (a.flags & kAccWrite) *dst = val;
      else *dst += val;
    }
  } else if (ph == A_R5) {
    const T S[3] = {a.asx[i], a.asy[j], a.asz[k]};
    const T D[3] = {ld(MDX), ld(MDY), ld(MDZ)};
    const T Vin[3] = {ld(FVX), ld(FVY), ld(FVZ)};
    T* V[3] = {a.vx, a.vy, a.vz};
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const T vt = Vin[c] + in[c];
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
