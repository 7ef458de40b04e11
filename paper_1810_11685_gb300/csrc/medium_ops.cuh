// Derivatives of the acoustic data in the medium (sound speed c, ambient
// density rho), 2D, with the sweeps in the context's precision (FP64 or FP32)
// and the gradient sums in FP64.
//
// The paper's Discussion names a joint reconstruction of the optical
// coefficients and the sound speed as the next step.  Its Jacobian needs the
// derivative of H_a in c and rho, taken here of the discretised map itself,
// as for H_a^* (Section 3.2.4, Lemma 2):
//
//  * c enters through C = c^2 in eq. num-p, through tau = -2 alpha0 c^(y-1)
//    and eta = 2 alpha0 c^y tan(pi y / 2) (eq. Twelve), so that
//    d tau / dc = (y - 1) tau / c and d eta / dc = y eta / c, and through the
//    source dt s_i = P0 / (2 d C) of eq. s1;
//  * rho enters through rho-bar at the nodes (eq. num-rho and the absorption
//    term of num-p) and through the staggered rho-bar_i of eq. num-vel, the
//    mean of the two neighbouring nodes.
//
// c_ref (the k-space correction kappa and the PML scale) and dt are held
// fixed: they are parameters of the discretisation.
//
// The tangent loop (jvp) steps the fields and their derivatives together.
// The adjoint (vjp) runs the forward loop, keeping the spectral quantities
// each step's derivative needs (for every step, or recomputed segment by
// segment from checkpoints), and then runs the exact transpose backwards.
// Spectral operators are full complex 2D FFTs in three launches: the x
// transforms of the real inputs; per group of adjacent columns the y
// transforms, the symbol products (the context's half-spectrum tables,
// mirrored) and the inverse y transforms; the inverse x transforms keeping
// the real part.  Each CTA transforms several grid lines in shared memory
// (mixed-radix Stockham), and up to four fields (a field and its tangent,
// the velocity components, the absorption inputs) share each launch.
//
// Every per-element body is a functor templated on the sweep's real type R;
// the loops are templates over R and the executor type, whose one
// implementation (GpuEx in medium.cu) launches each functor as a grid-stride
// kernel on the context's stream.  The directions (dc, drho), the sensor
// weights w and every output are FP64 whatever R is; the products that feed
// the gradient are formed and summed in FP64 over the N_t steps, so that an
// FP32 sweep rounds each step's contribution once instead of the running sum.
#pragma once

#include <math.h>
#include <vector_types.h>

#include <initializer_list>

#ifdef __CUDACC__
#define QPAT_HD __host__ __device__ __forceinline__
#else
#define QPAT_HD inline
#endif

namespace qpat {
namespace med {

// Complex type of a real type.
template <typename R>
struct CplxOf;
template <>
struct CplxOf<double> { typedef double2 t; };
template <>
struct CplxOf<float> { typedef float2 t; };
template <typename R>
using Cplx = typename CplxOf<R>::t;

template <typename R>
QPAT_HD Cplx<R> z(R a, R b) { Cplx<R> r; r.x = a; r.y = b; return r; }
template <typename C>
QPAT_HD C zadd(C a, C b) { C r; r.x = a.x + b.x; r.y = a.y + b.y; return r; }
template <typename C>
QPAT_HD C zmul(C a, C b) { C r; r.x = a.x * b.x - a.y * b.y; r.y = a.x * b.y + a.y * b.x; return r; }
template <typename C>
QPAT_HD C zconj(C a) { a.y = -a.y; return a; }
template <typename C, typename R>
QPAT_HD C zscale(C a, R s) { a.x *= s; a.y *= s; return a; }

constexpr int kMaxStages = 16;
struct Plan {
  int L = 0, nstages = 0;
  int radix[kMaxStages] = {};
};

// Tables of one 2D FP64 context (device pointers on the GPU, host pointers
// in a host run).  Layouts as the propagation passes use them:
// full-grid diagonals [ny][nx]; PML per axis; k-space symbols on the half
// spectrum [ny][nxh] divided by nx*ny; shift factors i k e^{+-i k dx/2}
// ([nxh] along x, [ny] along y); twiddles W_L^m = e^{-2 pi i m / L};
// sensors in gather form ([ns][4] indices and bilinear weights) and in the
// row-wise scatter form (rowptr [ny+1], point columns, per-point entries).
template <typename R>
struct Tables {
  typedef Cplx<R> C;
  int nx, ny, nxh, pml, n0, n1, ns, nt, lossless;
  R dt;
  double y;
  const R *Cc, *rho0, *dtrsx, *dtrsy, *tau, *eta;
  const R *ax, *asx, *ay, *asy;
  const R *kap, *kp1, *kp2;
  const C *shxp, *shxm, *shyp, *shym, *twx, *twy;
  const int* sidx;
  const R* sw;
  const int *rowptr, *pcol, *pent, *esens;
  const R* ew;
  Plan px, py;
};

enum Symbol { kDPX = 0, kDPY = 1, kDMX = 2, kDMY = 3, kYDIS = 4, kYABS = 5 };

// Symbol at spectral bin (j, i) of the full nx x ny spectrum.  Bins
// i >= nxh mirror i' = nx - i: |k| is even in kx and i kx e^{+-i kx dx/2} is
// Hermitian, so the value there is the conjugate of the stored one.
template <typename R>
QPAT_HD Cplx<R> symbol(const Tables<R>& t, int which, int j, int i) {
  const bool mir = i >= t.nxh;
  const int im = mir ? t.nx - i : i;
  const long long kt = (long long)j * t.nxh + im;
  Cplx<R> s;
  switch (which) {
    case kDPX: s = t.shxp[im]; if (mir) s = zconj(s); return zscale(s, t.kap[kt]);
    case kDMX: s = t.shxm[im]; if (mir) s = zconj(s); return zscale(s, t.kap[kt]);
    case kDPY: return zscale(t.shyp[j], t.kap[kt]);
    case kDMY: return zscale(t.shym[j], t.kap[kt]);
    case kYDIS: return z<R>(t.kp1[kt], (R)0);
    default: return z<R>(t.kp2[kt], (R)0);
  }
}

constexpr int kMaxBatch = 4;

// The terms of the outputs of one spectral product: output o is the sum
// over its nterm[o] terms q of sym[o][q] (conjugated when conj) times input
// spectrum in[o][q].
struct Terms {
  int no;
  int nterm[kMaxBatch], in[kMaxBatch][2], sym[kMaxBatch][2];
  int conj;
};
// Up to kMaxBatch field pointers, passed by value to a kernel.
template <typename P>
struct FieldPtrs {
  P p[kMaxBatch];
};

// Interior p0 [n1][n0] (FP64) -> full grid in the sweep's precision, zero
// in the PML.
template <typename R>
struct Embed {
  Tables<R> t;
  const double* p0;
  R* P;
  QPAT_HD void operator()(long long g) const {
    const int i = (int)(g % t.nx) - t.pml, j = (int)(g / t.nx) - t.pml;
    P[g] = (i >= 0 && i < t.n0 && j >= 0 && j < t.n1) ? (R)p0[(long long)j * t.n0 + i] : (R)0;
  }
};

// Staggered density perturbation of axis x / y at node g: the mean of the
// node and its + neighbour (periodic), as for rho-bar_i itself.
// (F: the field's type.)
template <class Tb, typename F>
QPAT_HD F stag_x(const Tb& t, const F* f, long long g) {
  const int i = (int)(g % t.nx);
  return (F)0.5 * (f[g] + f[g - i + (i + 1) % t.nx]);
}
template <class Tb, typename F>
QPAT_HD F stag_y(const Tb& t, const F* f, long long g) {
  const long long G = (long long)t.nx * t.ny;
  const long long gn = g + t.nx;
  return (F)0.5 * (f[g] + f[gn >= G ? gn - G : gn]);
}
// Transpose of stag_x / stag_y: the mean of the node and its - neighbour.
template <class Tb, typename F>
QPAT_HD F stag_x_T(const Tb& t, const F* f, long long g) {
  const int i = (int)(g % t.nx);
  return (F)0.5 * (f[g] + f[g - i + (i + t.nx - 1) % t.nx]);
}
template <class Tb, typename F>
QPAT_HD F stag_y_T(const Tb& t, const F* f, long long g) {
  const long long G = (long long)t.nx * t.ny;
  const long long gp = g - t.nx;
  return (F)0.5 * (f[g] + f[gp < 0 ? gp + G : gp]);
}

// Sensor gather of one time sample: out[s] = sum of the 4 bilinear corners
// (summed and stored in FP64).
template <typename R>
struct Gather {
  Tables<R> t;
  const R* f;
  double* out;
  QPAT_HD void operator()(long long s) const {
    double a = 0.0;
    for (int q = 0; q < 4; ++q) a += (double)t.sw[4 * s + q] * f[t.sidx[4 * s + q]];
    out[s] = a;
  }
};
// Transposed sensor gather, one thread per grid row: f += M^T w (w FP64).
template <typename R>
struct Scatter {
  Tables<R> t;
  const double* w;
  R* f;
  QPAT_HD void operator()(long long row) const {
    for (int p = t.rowptr[row]; p < t.rowptr[row + 1]; ++p) {
      double a = 0.0;
      for (int e = t.pent[p]; e < t.pent[p + 1]; ++e) a += (double)t.ew[e] * w[t.esens[e]];
      f[row * t.nx + t.pcol[p]] += (R)a;
    }
  }
};

}  // namespace med
}  // namespace qpat

namespace qpat {
namespace med {

// ---------------------------------------------------------------------------
// Per-cell steps of the loop (2D: axis x = array axis 1, axis y = axis 0)
// ---------------------------------------------------------------------------

// eq. num-vel, and along (dc, drho) its tangent when dvx != nullptr:
// v_i = A_i (A_i v_i - (dt / rho_i) g_i), d(dt / rho_i) = -(dt / rho_i)^2 drho_i / dt.
template <typename R>
struct Vel {
  Tables<R> t;
  const R *gx, *gy, *dgx, *dgy;
  const double* drho;
  R *vx, *vy, *dvx, *dvy;
  QPAT_HD void operator()(long long g) const {
    const int i = (int)(g % t.nx), j = (int)(g / t.nx);
    const R ax = t.asx[i], ay = t.asy[j], bx = t.dtrsx[g], by = t.dtrsy[g];
    vx[g] = ax * (ax * vx[g] - bx * gx[g]);
    vy[g] = ay * (ay * vy[g] - by * gy[g]);
    if (dvx) {
      dvx[g] = ax * (ax * dvx[g] - bx * dgx[g] + bx * bx / t.dt * (R)stag_x(t, drho, g) * gx[g]);
      dvy[g] = ay * (ay * dvy[g] - by * dgy[g] + by * by / t.dt * (R)stag_y(t, drho, g) * gy[g]);
    }
  }
};

// eq. num-rho with the source of eq. s1 (src: n = -1, 0), the sums
// r = sum rho_i and u = sum A_i rho divergence_i that eq. num-p needs, and the
// tangents when drx != nullptr.  dt s_i = P0 / (4 C), so d(dt s_i) = -dt s_i dC / C.
template <typename R>
struct Rho {
  Tables<R> t;
  const R *dx, *dy, *ddx, *ddy;
  const double *drho, *dc;
  const R* P0;
  int src;
  R *rx, *ry, *r, *u, *drx, *dry, *dr, *du;
  QPAT_HD void operator()(long long g) const {
    const int i = (int)(g % t.nx), j = (int)(g / t.nx);
    const R ax = t.ax[i], ay = t.ay[j], r0 = t.rho0[g], dt = t.dt;
    R q = (R)0, dq = (R)0;
    if (src) {
      const R C = t.Cc[g];
      q = P0[g] / ((R)4 * C);
      if (drx) dq = -q * (R)2 * sqrt(C) * (R)dc[g] / C;
    }
    rx[g] = ax * (ax * rx[g] - dt * r0 * dx[g]) + q;
    ry[g] = ay * (ay * ry[g] - dt * r0 * dy[g]) + q;
    r[g] = rx[g] + ry[g];
    if (!t.lossless) u[g] = ax * r0 * dx[g] + ay * r0 * dy[g];
    if (drx) {
      const R dr0 = (R)drho[g];
      drx[g] = ax * (ax * drx[g] - dt * (dr0 * dx[g] + r0 * ddx[g])) + dq;
      dry[g] = ay * (ay * dry[g] - dt * (dr0 * dy[g] + r0 * ddy[g])) + dq;
      dr[g] = drx[g] + dry[g];
      if (!t.lossless) du[g] = ax * (dr0 * dx[g] + r0 * ddx[g]) + ay * (dr0 * dy[g] + r0 * ddy[g]);
    }
  }
};

// eq. num-p: p = C X, X = r (lossless) or r - eta Y_dis r + tau Y_abs u; keeps X
// when Xo != nullptr and forms the tangent dp = dC X + C dX when dp != nullptr.
template <typename R>
struct Pres {
  Tables<R> t;
  const R *r, *Yr, *Yu, *dr, *YdR, *Ydu;
  const double* dc;
  R *p, *Xo, *dp;
  QPAT_HD void operator()(long long g) const {
    const R C = t.Cc[g];
    R X = r[g];
    if (!t.lossless) X += -t.eta[g] * Yr[g] + t.tau[g] * Yu[g];
    p[g] = C * X;
    if (Xo) Xo[g] = X;
    if (dp) {
      const R c = sqrt(C), dcg = (R)dc[g];
      R dX = dr[g];
      if (!t.lossless) {
        const R dtau = (R)(t.y - 1.0) * t.tau[g] / c * dcg, deta = (R)t.y * t.eta[g] / c * dcg;
        dX += -deta * Yr[g] - t.eta[g] * YdR[g] + dtau * Yu[g] + t.tau[g] * Ydu[g];
      }
      dp[g] = (R)2 * c * dcg * X + C * dX;
    }
  }
};

// Reverse of eq. num-p at one step: pb is the adjoint of p_(n+1) (sensor
// scatter already added).  gC += pb X; Cp = C pb; lossy: g_eta -= Cp Y_dis r,
// g_tau += Cp Y_abs u and the two fields eta Cp, tau Cp whose transposed
// spectral products come next.
template <typename R>
struct RevP {
  Tables<R> t;
  const R *pb, *X, *Yr, *Yu;
  double *gC, *geta, *gtau;
  R *Cp, *e1, *e2;
  QPAT_HD void operator()(long long g) const {
    const R cp = t.Cc[g] * pb[g];
    gC[g] += (double)pb[g] * X[g];
    Cp[g] = cp;
    if (!t.lossless) {
      geta[g] -= (double)cp * Yr[g];
      gtau[g] += (double)cp * Yu[g];
      e1[g] = t.eta[g] * cp;
      e2[g] = t.tau[g] * cp;
    }
  }
};

// Reverse of eq. num-rho (and of the u term of num-p): with
// rtot_i = rb_i + (Cp - Y_dis^T eta Cp) and ub = Y_abs^T tau Cp,
// db_i = rho A_i (ub - dt rtot_i), g_rho += A_i div_i (ub - dt rtot_i),
// rb_i = A_i^2 rtot_i, and the source adjoint qb += sum rtot_i (src).
template <typename R>
struct RevRho {
  Tables<R> t;
  const R *Cp, *t1, *ub, *dx, *dy;
  int src;
  R *rbx, *rby, *dbx, *dby;
  double *grho, *qb;
  QPAT_HD void operator()(long long g) const {
    const int i = (int)(g % t.nx), j = (int)(g / t.nx);
    const R ax = t.ax[i], ay = t.ay[j], r0 = t.rho0[g], dt = t.dt;
    R rp = Cp[g], u = (R)0;
    if (!t.lossless) {
      rp -= t1[g];
      u = ub[g];
    }
    const R tx = rbx[g] + rp, ty = rby[g] + rp;
    const R hx = u - dt * tx, hy = u - dt * ty;
    dbx[g] = r0 * ax * hx;
    dby[g] = r0 * ay * hy;
    grho[g] += (double)ax * dx[g] * hx + (double)ay * dy[g] * hy;
    rbx[g] = ax * ax * tx;
    rby[g] = ay * ay * ty;
    if (src) qb[g] += (double)tx + ty;
  }
};

// Reverse of eq. num-vel: vtot_i = vb_i + (D-_i)^T db_i;
// g_rho_i += vtot_i A_i (dt / rho_i)^2 / dt g_i (g_i = D+_i p of the forward
// step); vb_i = A_i^2 vtot_i; f_i = A_i (dt / rho_i) vtot_i, whose transposed
// D+_i products make the adjoint of p_n (with a minus sign).
template <typename R>
struct RevVel {
  Tables<R> t;
  const R *ex, *ey, *gx, *gy;
  R *vbx, *vby;
  double *grsx, *grsy;
  R *fx, *fy;
  QPAT_HD void operator()(long long g) const {
    const int i = (int)(g % t.nx), j = (int)(g / t.nx);
    const R ax = t.asx[i], ay = t.asy[j], bx = t.dtrsx[g], by = t.dtrsy[g];
    const R tx = vbx[g] + ex[g], ty = vby[g] + ey[g];
    grsx[g] += (double)tx * ax * bx * bx / t.dt * gx[g];
    grsy[g] += (double)ty * ay * by * by / t.dt * gy[g];
    vbx[g] = ax * ax * tx;
    vby[g] = ay * ay * ty;
    fx[g] = ax * bx * tx;
    fy[g] = ay * by * ty;
  }
};

// The gradients in c and rho on the full grid: the source term of eq. s1
// (dt s_i = P0 / (4 C)), the chain rule through C = c^2, tau and eta, and
// the transposed staggered means.
template <typename R>
struct Finish {
  Tables<R> t;
  const double *gC, *gtau, *geta, *qb;
  const R* P0;
  const double *grsx, *grsy, *grho;
  double *g_c, *g_rho;
  QPAT_HD void operator()(long long g) const {
    const double C = t.Cc[g], c = sqrt(C);
    const double gc = gC[g] - qb[g] * (double)P0[g] / (4.0 * C) / C;
    double v = 2.0 * c * gc;
    if (!t.lossless) v += (t.y - 1.0) * (double)t.tau[g] / c * gtau[g] + t.y * (double)t.eta[g] / c * geta[g];
    g_c[g] = v;
    g_rho[g] = grho[g] + stag_x_T(t, grsx, g) + stag_y_T(t, grsy, g);
  }
};

}  // namespace med
}  // namespace qpat

namespace qpat {
namespace med {

// Spectral products F^-1 { S F{f} } on the full complex spectrum, several
// fields per launch, in three launches: the x transforms of the real inputs
// (forward), then per group of adjacent columns the y transforms, the
// symbol products and the inverse y transforms, then the inverse x
// transforms keeping alpha times the real part (apply).  Zi holds up to
// kMaxBatch x-transformed inputs, Zc the combined products (each
// kMaxBatch * G).
template <class Ex, typename R>
struct Spectral {
  Ex& ex;
  const Tables<R>& t;
  long long G;
  Cplx<R> *Zi, *Zc;
  int nin = 0;                                    // inputs of the last forward()

  // x transforms of the fields f[0..nb) into Zi
  void forward(std::initializer_list<const R*> f) {
    if (f.size() < 1 || f.size() > (size_t)kMaxBatch) {
      ex.fail(cudaErrorInvalidValue);
      return;
    }
    FieldPtrs<const R*> in{};
    int nb = 0;
    for (const R* p : f) in.p[nb++] = p;
    nin = nb;
    ex.rows_forward(in, nb, Zi, t, G);
  }
  // outputs o: out[o] = alpha Re F^-1{ sum_q S_(o,q) F{f_(in_(o,q))} }; terms
  // list (in, symbol) pairs per output; conj: the transposed operators.
  void apply(std::initializer_list<std::initializer_list<int>> terms, int conj,
             std::initializer_list<R*> out, R alpha) {
    // at most kMaxBatch outputs, each of one or two (input, symbol) terms
    // over the inputs of the last forward()
    bool ok = terms.size() >= 1 && terms.size() <= (size_t)kMaxBatch && out.size() == terms.size();
    for (const auto& tl : terms) ok = ok && tl.size() >= 2 && tl.size() <= 4 && tl.size() % 2 == 0;
    Terms tm{};
    tm.conj = conj;
    int no = 0;
    if (ok) {
      for (const auto& tl : terms) {
        int q = 0, k = 0;
        for (int v : tl) {
          if (k % 2 == 0) {
            ok = ok && v >= 0 && v < nin;
            tm.in[no][q] = v;
          } else {
            tm.sym[no][q++] = v;
          }
          ++k;
        }
        tm.nterm[no++] = q;
      }
    }
    if (!ok) {
      ex.fail(cudaErrorInvalidValue);
      return;
    }
    tm.no = no;
    ex.cols_combine(Zi, nin, Zc, tm, t, G);
    FieldPtrs<R*> o{};
    int nb = 0;
    for (R* p : out) o.p[nb++] = p;
    ex.rows_inverse(Zc, o, no, alpha, t, G);
  }
};

// Fields of one loop, all [G] in the sweep's precision.
template <typename R>
struct Fields {
  R *P0, *p, *vx, *vy, *rx, *ry, *r, *u;
  R *gx, *gy, *dx, *dy, *Yr, *Yu, *X;
  R *dp, *dvx, *dvy, *drx, *dry, *dr, *du, *dgx, *dgy, *ddx, *ddy, *YdR, *Ydu;
};

// Tangent loop: dP[n] = M dp_n for n = 0 .. nt-1 along (dc, drho), both full
// grid.  The loop runs n = -1 .. nt-2 from zero fields (samples n + 1).
template <class Ex, typename R>
void jvp_loop(Ex& ex, const Tables<R>& t, Spectral<Ex, R>& S, const Fields<R>& f, const double* dc,
              const double* drho, double* dP) {
  const long long G = (long long)t.nx * t.ny;
  for (int it = 0; it < t.nt; ++it) {
    const int src = it <= 1;
    S.forward({f.p, f.dp});
    S.apply({{0, kDPX}, {0, kDPY}, {1, kDPX}, {1, kDPY}}, 0, {f.gx, f.gy, f.dgx, f.dgy}, 1.0);
    ex.run(G, Vel<R>{t, f.gx, f.gy, f.dgx, f.dgy, drho, f.vx, f.vy, f.dvx, f.dvy});
    S.forward({f.vx, f.vy, f.dvx, f.dvy});
    S.apply({{0, kDMX}, {1, kDMY}, {2, kDMX}, {3, kDMY}}, 0, {f.dx, f.dy, f.ddx, f.ddy}, 1.0);
    ex.run(G, Rho<R>{t, f.dx, f.dy, f.ddx, f.ddy, drho, dc, f.P0, src, f.rx, f.ry, f.r, f.u, f.drx, f.dry, f.dr,
                     f.du});
    if (!t.lossless) {
      S.forward({f.r, f.u, f.dr, f.du});
      S.apply({{0, kYDIS}, {1, kYABS}, {2, kYDIS}, {3, kYABS}}, 0, {f.Yr, f.Yu, f.YdR, f.Ydu}, 1.0);
    }
    ex.run(G, Pres<R>{t, f.r, f.Yr, f.Yu, f.dr, f.YdR, f.Ydu, dc, f.p, nullptr, f.dp});
    ex.run(t.ns, Gather<R>{t, f.dp, dP + (long long)it * t.ns});
  }
}

// Fields of one forward step that the reverse step needs: g_i = D+_i p_n,
// the divergences D-_i v_i, X = p_(n+1) / C and (lossy) Y_dis r, Y_abs u.
// Tape holds them for a run of consecutive steps ([steps][G] each).
template <typename R>
struct Tape {
  R *gx, *gy, *dx, *dy, *X, *Yr, *Yu;
};

// Reverse-loop fields, all [G]: the adjoint fields in the sweep's precision,
// the gradient sums in FP64.
template <typename R>
struct RevFields {
  R *pb, *Cp, *e1, *e2, *t1, *ub, *rbx, *rby, *dbx, *dby, *vbx, *vby, *fx, *fy, *ex, *ey;
  double *qb, *gC, *gtau, *geta, *grho, *grsx, *grsy;
};

// Copy the loop state (p, v_x, v_y, rho_x, rho_y) to or from a checkpoint
// [5][G].
template <typename R>
struct StateCopy {
  const R* src[5];
  R* dst[5];
  long long G;
  QPAT_HD void operator()(long long u) const {
    const long long k = u / G, g = u - k * G;
    dst[k][g] = src[k][g];
  }
};

// Forward step it (loop index n = it - 1) of the gradient's forward sweep,
// writing its tape fields to slot k of tp.
template <class Ex, typename R>
void tape_step(Ex& ex, const Tables<R>& t, Spectral<Ex, R>& S, const Fields<R>& f, const Tape<R>& tp, int it,
               int k) {
  const long long G = (long long)t.nx * t.ny, o = (long long)k * G;
  S.forward({f.p});
  S.apply({{0, kDPX}, {0, kDPY}}, 0, {tp.gx + o, tp.gy + o}, 1.0);
  ex.run(G, Vel<R>{t, tp.gx + o, tp.gy + o, nullptr, nullptr, nullptr, f.vx, f.vy, nullptr, nullptr});
  S.forward({f.vx, f.vy});
  S.apply({{0, kDMX}, {1, kDMY}}, 0, {tp.dx + o, tp.dy + o}, 1.0);
  ex.run(G, Rho<R>{t, tp.dx + o, tp.dy + o, nullptr, nullptr, nullptr, nullptr, f.P0, it <= 1, f.rx, f.ry, f.r,
                   f.u, nullptr, nullptr, nullptr, nullptr});
  R* Yr = t.lossless ? nullptr : tp.Yr + o;
  R* Yu = t.lossless ? nullptr : tp.Yu + o;
  if (!t.lossless) {
    S.forward({f.r, f.u});
    S.apply({{0, kYDIS}, {1, kYABS}}, 0, {Yr, Yu}, 1.0);
  }
  ex.run(G, Pres<R>{t, f.r, Yr, Yu, nullptr, nullptr, nullptr, nullptr, f.p, tp.X + o, nullptr});
}

// Transposed step it, reading the tape fields of step it from slot k.
template <class Ex, typename R>
void reverse_step(Ex& ex, const Tables<R>& t, Spectral<Ex, R>& S, const Tape<R>& tp, const RevFields<R>& b,
                  const double* W, int it, int k) {
  const long long G = (long long)t.nx * t.ny, o = (long long)k * G;
  const R* Yr = t.lossless ? nullptr : tp.Yr + o;
  const R* Yu = t.lossless ? nullptr : tp.Yu + o;
  ex.run(t.ny, Scatter<R>{t, W + (long long)it * t.ns, b.pb});
  ex.run(G, RevP<R>{t, b.pb, tp.X + o, Yr, Yu, b.gC, b.geta, b.gtau, b.Cp, b.e1, b.e2});
  if (!t.lossless) {
    S.forward({b.e1, b.e2});
    S.apply({{0, kYDIS}, {1, kYABS}}, 1, {b.t1, b.ub}, 1.0);
  }
  ex.run(G, RevRho<R>{t, b.Cp, b.t1, b.ub, tp.dx + o, tp.dy + o, it <= 1, b.rbx, b.rby, b.dbx, b.dby, b.grho,
                      b.qb});
  S.forward({b.dbx, b.dby});
  S.apply({{0, kDMX}, {1, kDMY}}, 1, {b.ex, b.ey}, 1.0);
  ex.run(G, RevVel<R>{t, b.ex, b.ey, tp.gx + o, tp.gy + o, b.vbx, b.vby, b.grsx, b.grsy, b.fx, b.fy});
  S.forward({b.fx, b.fy});
  S.apply({{0, kDPX, 1, kDPY}}, 1, {b.pb}, -1.0);
}

// The gradient: the forward loop, then its exact transpose backwards.
// K >= nt: the tape holds every step (nt slots), written by the one forward
// sweep.  K < nt: the tape holds K steps; the forward sweep stores the loop
// state at the start of every segment of K steps in ck ([ceil(nt/K)][5][G]),
// and the reverse sweep, segment by segment from the last, restores that
// state, recomputes the segment's tape and runs its transposed steps.  The
// recomputation repeats the same kernels on the same inputs, so the tape
// and the gradient are the same bit for bit for every K.
template <class Ex, typename R>
void vjp_loop(Ex& ex, const Tables<R>& t, Spectral<Ex, R>& S, const Fields<R>& f, const Tape<R>& tp,
              const RevFields<R>& b, int K, R* ck, const double* W, double* g_c, double* g_rho) {
  const long long G = (long long)t.nx * t.ny;
  if (K >= t.nt) {
    for (int it = 0; it < t.nt; ++it) tape_step(ex, t, S, f, tp, it, it);
    for (int it = t.nt - 1; it >= 0; --it) reverse_step(ex, t, S, tp, b, W, it, it);
  } else {
    auto state = [&](int seg, bool save) {
      R* c = ck + (long long)seg * 5 * G;
      R* live[5] = {f.p, f.vx, f.vy, f.rx, f.ry};
      StateCopy<R> op{};
      for (int q = 0; q < 5; ++q) {
        op.src[q] = save ? live[q] : c + q * G;
        op.dst[q] = save ? c + q * G : live[q];
      }
      op.G = G;
      ex.run(5 * G, op);
    };
    const int nseg = (t.nt + K - 1) / K;
    for (int it = 0; it < t.nt; ++it) {
      if (it % K == 0) state(it / K, true);
      tape_step(ex, t, S, f, tp, it, 0);                   // slot 0 as scratch
    }
    for (int seg = nseg - 1; seg >= 0; --seg) {
      const int first = seg * K, end = first + K < t.nt ? first + K : t.nt;
      state(seg, false);
      for (int it = first; it < end; ++it) tape_step(ex, t, S, f, tp, it, it - first);
      for (int it = end - 1; it >= first; --it) reverse_step(ex, t, S, tp, b, W, it, it - first);
    }
  }
  ex.run(G, Finish<R>{t, b.gC, b.gtau, b.geta, b.qb, f.P0, b.grsx, b.grsy, b.grho, g_c, g_rho});
}

}  // namespace med
}  // namespace qpat
