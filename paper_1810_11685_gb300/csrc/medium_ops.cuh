// Derivatives of the acoustic data in the medium (sound speed c, ambient
// density rho), FP64, 2D.
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
// The adjoint (vjp) runs the forward loop once, keeping the spectral
// quantities each step's derivative needs (the whole history stays in HBM),
// and then runs the exact transpose backwards.  Spectral operators are full
// complex 2D FFTs: one launch per axis, each CTA transforming several grid
// lines in shared memory (mixed-radix Stockham), then the symbol multiply
// (the context's FP64 half-spectrum tables, mirrored), then the inverse FFT;
// up to four fields (a field and its tangent, the velocity components, the
// absorption inputs) share each launch.
//
// Every per-element body is a functor; the loops are templates over the
// executor type, whose one implementation (GpuEx in medium.cu) launches each
// functor as a grid-stride kernel on the context's stream.
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

QPAT_HD double2 z(double a, double b) { double2 r; r.x = a; r.y = b; return r; }
QPAT_HD double2 zadd(double2 a, double2 b) { return z(a.x + b.x, a.y + b.y); }
QPAT_HD double2 zmul(double2 a, double2 b) { return z(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x); }
QPAT_HD double2 zconj(double2 a) { return z(a.x, -a.y); }
QPAT_HD double2 zscale(double2 a, double s) { return z(a.x * s, a.y * s); }

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
struct Tables {
  int nx, ny, nxh, pml, n0, n1, ns, nt, lossless;
  double dt, y;
  const double *Cc, *rho0, *dtrsx, *dtrsy, *tau, *eta;
  const double *ax, *asx, *ay, *asy;
  const double *kap, *kp1, *kp2;
  const double2 *shxp, *shxm, *shyp, *shym, *twx, *twy;
  const int* sidx;
  const double* sw;
  const int *rowptr, *pcol, *pent, *esens;
  const double* ew;
  Plan px, py;
};

enum Symbol { kDPX = 0, kDPY = 1, kDMX = 2, kDMY = 3, kYDIS = 4, kYABS = 5 };

// Symbol at spectral bin (j, i) of the full nx x ny spectrum.  Bins
// i >= nxh mirror i' = nx - i: |k| is even in kx and i kx e^{+-i kx dx/2} is
// Hermitian, so the value there is the conjugate of the stored one.
QPAT_HD double2 symbol(const Tables& t, int which, int j, int i) {
  const bool mir = i >= t.nxh;
  const int im = mir ? t.nx - i : i;
  const long long kt = (long long)j * t.nxh + im;
  double2 s;
  switch (which) {
    case kDPX: s = t.shxp[im]; if (mir) s = zconj(s); return zscale(s, t.kap[kt]);
    case kDMX: s = t.shxm[im]; if (mir) s = zconj(s); return zscale(s, t.kap[kt]);
    case kDPY: return zscale(t.shyp[j], t.kap[kt]);
    case kDMY: return zscale(t.shym[j], t.kap[kt]);
    case kYDIS: return z(t.kp1[kt], 0.0);
    default: return z(t.kp2[kt], 0.0);
  }
}

constexpr int kMaxBatch = 4;

// Z[b G + g] = f_b[g] + 0 i for nb fields
struct LoadReal {
  const double* f[kMaxBatch];
  double2* Z;
  long long G;
  QPAT_HD void operator()(long long t) const {
    const long long b = t / G;
    Z[t] = z(f[b][t - b * G], 0.0);
  }
};
// out_b = alpha Re(Z[b G + .]), or out_b += alpha Re(...) when acc
struct StoreReal {
  const double2* Z;
  double* out[kMaxBatch];
  double alpha;
  int acc;
  long long G;
  QPAT_HD void operator()(long long t) const {
    const long long b = t / G, g = t - b * G;
    const double v = alpha * Z[t].x;
    out[b][g] = acc ? out[b][g] + v : v;
  }
};
// Output o: Zo[o G + g] = sum over its nterm[o] terms q of sym[o][q]
// (conjugated when conj) * Zi[in[o][q] G + g].
struct Combine {
  Tables t;
  const double2* Zi;
  double2* Zo;
  int nterm[kMaxBatch], in[kMaxBatch][2], sym[kMaxBatch][2];
  int conj;
  long long G;
  QPAT_HD void operator()(long long u) const {
    const long long o = u / G, g = u - o * G;
    const int i = (int)(g % t.nx), j = (int)(g / t.nx);
    double2 r = z(0.0, 0.0);
    for (int q = 0; q < nterm[o]; ++q) {
      double2 a = symbol(t, sym[o][q], j, i);
      if (conj) a = zconj(a);
      r = zadd(r, zmul(a, Zi[in[o][q] * G + g]));
    }
    Zo[u] = r;
  }
};

// Interior p0 [n1][n0] -> full grid, zero in the PML.
struct Embed {
  Tables t;
  const double* p0;
  double* P;
  QPAT_HD void operator()(long long g) const {
    const int i = (int)(g % t.nx) - t.pml, j = (int)(g / t.nx) - t.pml;
    P[g] = (i >= 0 && i < t.n0 && j >= 0 && j < t.n1) ? p0[(long long)j * t.n0 + i] : 0.0;
  }
};

// Staggered density perturbation of axis x / y at node g: the mean of the
// node and its + neighbour (periodic), as for rho-bar_i itself.
QPAT_HD double stag_x(const Tables& t, const double* f, long long g) {
  const int i = (int)(g % t.nx);
  return 0.5 * (f[g] + f[g - i + (i + 1) % t.nx]);
}
QPAT_HD double stag_y(const Tables& t, const double* f, long long g) {
  const long long G = (long long)t.nx * t.ny;
  const long long gn = g + t.nx;
  return 0.5 * (f[g] + f[gn >= G ? gn - G : gn]);
}
// Transpose of stag_x / stag_y: the mean of the node and its - neighbour.
QPAT_HD double stag_x_T(const Tables& t, const double* f, long long g) {
  const int i = (int)(g % t.nx);
  return 0.5 * (f[g] + f[g - i + (i + t.nx - 1) % t.nx]);
}
QPAT_HD double stag_y_T(const Tables& t, const double* f, long long g) {
  const long long G = (long long)t.nx * t.ny;
  const long long gp = g - t.nx;
  return 0.5 * (f[g] + f[gp < 0 ? gp + G : gp]);
}

// Sensor gather of one time sample: out[s] = sum of the 4 bilinear corners.
struct Gather {
  Tables t;
  const double* f;
  double* out;
  QPAT_HD void operator()(long long s) const {
    double a = 0.0;
    for (int q = 0; q < 4; ++q) a += t.sw[4 * s + q] * f[t.sidx[4 * s + q]];
    out[s] = a;
  }
};
// Transposed sensor gather, one thread per grid row: f += M^T w.
struct Scatter {
  Tables t;
  const double* w;
  double* f;
  QPAT_HD void operator()(long long row) const {
    for (int p = t.rowptr[row]; p < t.rowptr[row + 1]; ++p) {
      double a = 0.0;
      for (int e = t.pent[p]; e < t.pent[p + 1]; ++e) a += t.ew[e] * w[t.esens[e]];
      f[row * t.nx + t.pcol[p]] += a;
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
struct Vel {
  Tables t;
  const double *gx, *gy, *dgx, *dgy, *drho;
  double *vx, *vy, *dvx, *dvy;
  QPAT_HD void operator()(long long g) const {
    const int i = (int)(g % t.nx), j = (int)(g / t.nx);
    const double ax = t.asx[i], ay = t.asy[j], bx = t.dtrsx[g], by = t.dtrsy[g];
    vx[g] = ax * (ax * vx[g] - bx * gx[g]);
    vy[g] = ay * (ay * vy[g] - by * gy[g]);
    if (dvx) {
      dvx[g] = ax * (ax * dvx[g] - bx * dgx[g] + bx * bx / t.dt * stag_x(t, drho, g) * gx[g]);
      dvy[g] = ay * (ay * dvy[g] - by * dgy[g] + by * by / t.dt * stag_y(t, drho, g) * gy[g]);
    }
  }
};

// eq. num-rho with the source of eq. s1 (src: n = -1, 0), the sums
// r = sum rho_i and u = sum A_i rho divergence_i that eq. num-p needs, and the
// tangents when drx != nullptr.  dt s_i = P0 / (4 C), so d(dt s_i) = -dt s_i dC / C.
struct Rho {
  Tables t;
  const double *dx, *dy, *ddx, *ddy, *drho, *dc, *P0;
  int src;
  double *rx, *ry, *r, *u, *drx, *dry, *dr, *du;
  QPAT_HD void operator()(long long g) const {
    const int i = (int)(g % t.nx), j = (int)(g / t.nx);
    const double ax = t.ax[i], ay = t.ay[j], r0 = t.rho0[g], dt = t.dt;
    double q = 0.0, dq = 0.0;
    if (src) {
      const double C = t.Cc[g];
      q = P0[g] / (4.0 * C);
      if (drx) dq = -q * 2.0 * sqrt(C) * dc[g] / C;
    }
    rx[g] = ax * (ax * rx[g] - dt * r0 * dx[g]) + q;
    ry[g] = ay * (ay * ry[g] - dt * r0 * dy[g]) + q;
    r[g] = rx[g] + ry[g];
    if (!t.lossless) u[g] = ax * r0 * dx[g] + ay * r0 * dy[g];
    if (drx) {
      const double dr0 = drho[g];
      drx[g] = ax * (ax * drx[g] - dt * (dr0 * dx[g] + r0 * ddx[g])) + dq;
      dry[g] = ay * (ay * dry[g] - dt * (dr0 * dy[g] + r0 * ddy[g])) + dq;
      dr[g] = drx[g] + dry[g];
      if (!t.lossless) du[g] = ax * (dr0 * dx[g] + r0 * ddx[g]) + ay * (dr0 * dy[g] + r0 * ddy[g]);
    }
  }
};

// eq. num-p: p = C X, X = r (lossless) or r - eta Y_dis r + tau Y_abs u; keeps X
// when Xo != nullptr and forms the tangent dp = dC X + C dX when dp != nullptr.
struct Pres {
  Tables t;
  const double *r, *Yr, *Yu, *dr, *YdR, *Ydu, *dc;
  double *p, *Xo, *dp;
  QPAT_HD void operator()(long long g) const {
    const double C = t.Cc[g];
    double X = r[g];
    if (!t.lossless) X += -t.eta[g] * Yr[g] + t.tau[g] * Yu[g];
    p[g] = C * X;
    if (Xo) Xo[g] = X;
    if (dp) {
      const double c = sqrt(C), dcg = dc[g];
      double dX = dr[g];
      if (!t.lossless) {
        const double dtau = (t.y - 1.0) * t.tau[g] / c * dcg, deta = t.y * t.eta[g] / c * dcg;
        dX += -deta * Yr[g] - t.eta[g] * YdR[g] + dtau * Yu[g] + t.tau[g] * Ydu[g];
      }
      dp[g] = 2.0 * c * dcg * X + C * dX;
    }
  }
};

// Reverse of eq. num-p at one step: pb is the adjoint of p_(n+1) (sensor
// scatter already added).  gC += pb X; Cp = C pb; lossy: g_eta -= Cp Y_dis r,
// g_tau += Cp Y_abs u and the two fields eta Cp, tau Cp whose transposed
// spectral products come next.
struct RevP {
  Tables t;
  const double *pb, *X, *Yr, *Yu;
  double *gC, *geta, *gtau, *Cp, *e1, *e2;
  QPAT_HD void operator()(long long g) const {
    const double cp = t.Cc[g] * pb[g];
    gC[g] += pb[g] * X[g];
    Cp[g] = cp;
    if (!t.lossless) {
      geta[g] -= cp * Yr[g];
      gtau[g] += cp * Yu[g];
      e1[g] = t.eta[g] * cp;
      e2[g] = t.tau[g] * cp;
    }
  }
};

// Reverse of eq. num-rho (and of the u term of num-p): with
// rtot_i = rb_i + (Cp - Y_dis^T eta Cp) and ub = Y_abs^T tau Cp,
// db_i = rho A_i (ub - dt rtot_i), g_rho += A_i div_i (ub - dt rtot_i),
// rb_i = A_i^2 rtot_i, and the source adjoint qb += sum rtot_i (src).
struct RevRho {
  Tables t;
  const double *Cp, *t1, *ub, *dx, *dy;
  int src;
  double *rbx, *rby, *dbx, *dby, *grho, *qb;
  QPAT_HD void operator()(long long g) const {
    const int i = (int)(g % t.nx), j = (int)(g / t.nx);
    const double ax = t.ax[i], ay = t.ay[j], r0 = t.rho0[g], dt = t.dt;
    double rp = Cp[g], u = 0.0;
    if (!t.lossless) {
      rp -= t1[g];
      u = ub[g];
    }
    const double tx = rbx[g] + rp, ty = rby[g] + rp;
    const double hx = u - dt * tx, hy = u - dt * ty;
    dbx[g] = r0 * ax * hx;
    dby[g] = r0 * ay * hy;
    grho[g] += ax * dx[g] * hx + ay * dy[g] * hy;
    rbx[g] = ax * ax * tx;
    rby[g] = ay * ay * ty;
    if (src) qb[g] += tx + ty;
  }
};

// Reverse of eq. num-vel: vtot_i = vb_i + (D-_i)^T db_i;
// g_rho_i += vtot_i A_i (dt / rho_i)^2 / dt g_i (g_i = D+_i p of the forward
// step); vb_i = A_i^2 vtot_i; f_i = A_i (dt / rho_i) vtot_i, whose transposed
// D+_i products make the adjoint of p_n (with a minus sign).
struct RevVel {
  Tables t;
  const double *ex, *ey, *gx, *gy;
  double *vbx, *vby, *grsx, *grsy, *fx, *fy;
  QPAT_HD void operator()(long long g) const {
    const int i = (int)(g % t.nx), j = (int)(g / t.nx);
    const double ax = t.asx[i], ay = t.asy[j], bx = t.dtrsx[g], by = t.dtrsy[g];
    const double tx = vbx[g] + ex[g], ty = vby[g] + ey[g];
    grsx[g] += tx * ax * bx * bx / t.dt * gx[g];
    grsy[g] += ty * ay * by * by / t.dt * gy[g];
    vbx[g] = ax * ax * tx;
    vby[g] = ay * ay * ty;
    fx[g] = ax * bx * tx;
    fy[g] = ay * by * ty;
  }
};

// The gradients in c and rho on the full grid: the source term of eq. s1
// (dt s_i = P0 / (4 C)), the chain rule through C = c^2, tau and eta, and
// the transposed staggered means.
struct Finish {
  Tables t;
  const double *gC, *gtau, *geta, *qb, *P0, *grsx, *grsy, *grho;
  double *g_c, *g_rho;
  QPAT_HD void operator()(long long g) const {
    const double C = t.Cc[g], c = sqrt(C);
    const double gc = gC[g] - qb[g] * P0[g] / (4.0 * C) / C;
    double v = 2.0 * c * gc;
    if (!t.lossless) v += (t.y - 1.0) * t.tau[g] / c * gtau[g] + t.y * t.eta[g] / c * geta[g];
    g_c[g] = v;
    g_rho[g] = grho[g] + stag_x_T(t, grsx, g) + stag_y_T(t, grsy, g);
  }
};

}  // namespace med
}  // namespace qpat

namespace qpat {
namespace med {

// Spectral products F^-1 { S F{f} } on the full complex spectrum, several
// fields per launch.  Zi holds up to kMaxBatch forward spectra, Zc the
// combined products (each kMaxBatch * G).
template <class Ex>
struct Spectral {
  Ex& ex;
  const Tables& t;
  long long G;
  double2 *Zi, *Zc;

  // 2D FFT of nb fields in place (inv: the unnormalised inverse), one launch
  // per axis: every grid line is transformed in shared memory
  void fft(double2* Z, int nb, int inv) { ex.fft2(Z, nb, inv, t, G); }
  // spectra of the fields f[0..nb) into Zi
  void forward(std::initializer_list<const double*> f) {
    if (f.size() < 1 || f.size() > (size_t)kMaxBatch) {
      ex.fail(cudaErrorInvalidValue);
      return;
    }
    LoadReal op{};
    int nb = 0;
    for (const double* p : f) op.f[nb++] = p;
    op.Z = Zi;
    op.G = G;
    ex.run(nb * G, op);
    fft(Zi, nb, 0);
  }
  // outputs o: out[o] = alpha Re F^-1{ sum_q S_(o,q) Zi[in_(o,q)] }; terms
  // list (in, symbol) pairs per output; conj: the transposed operators.
  void apply(std::initializer_list<std::initializer_list<int>> terms, int conj,
             std::initializer_list<double*> out, double alpha) {
    // at most kMaxBatch outputs, each of one or two (input, symbol) terms
    bool ok = terms.size() >= 1 && terms.size() <= (size_t)kMaxBatch && out.size() == terms.size();
    for (const auto& tl : terms) ok = ok && tl.size() >= 2 && tl.size() <= 4 && tl.size() % 2 == 0;
    if (!ok) {
      ex.fail(cudaErrorInvalidValue);
      return;
    }
    Combine cb{};
    cb.t = t;
    cb.Zi = Zi;
    cb.Zo = Zc;
    cb.conj = conj;
    cb.G = G;
    int no = 0;
    for (const auto& tl : terms) {
      int q = 0, k = 0;
      for (int v : tl) {
        if (k % 2 == 0) cb.in[no][q] = v;
        else cb.sym[no][q++] = v;
        ++k;
      }
      cb.nterm[no++] = q;
    }
    ex.run(no * G, cb);
    fft(Zc, no, 1);
    StoreReal st{};
    st.Z = Zc;
    int nb = 0;
    for (double* p : out) st.out[nb++] = p;
    st.alpha = alpha;
    st.acc = 0;
    st.G = G;
    ex.run(nb * G, st);
  }
};

// Fields of one loop, all [G] doubles (tape fields [nt][G]).
struct Fields {
  double *P0, *p, *vx, *vy, *rx, *ry, *r, *u;
  double *gx, *gy, *dx, *dy, *Yr, *Yu, *X;
  double *dp, *dvx, *dvy, *drx, *dry, *dr, *du, *dgx, *dgy, *ddx, *ddy, *YdR, *Ydu;
};

// Tangent loop: dP[n] = M dp_n for n = 0 .. nt-1 along (dc, drho), both full
// grid.  The loop runs n = -1 .. nt-2 from zero fields (samples n + 1).
template <class Ex>
void jvp_loop(Ex& ex, const Tables& t, Spectral<Ex>& S, const Fields& f, const double* dc, const double* drho,
              double* dP) {
  const long long G = (long long)t.nx * t.ny;
  for (int it = 0; it < t.nt; ++it) {
    const int src = it <= 1;
    S.forward({f.p, f.dp});
    S.apply({{0, kDPX}, {0, kDPY}, {1, kDPX}, {1, kDPY}}, 0, {f.gx, f.gy, f.dgx, f.dgy}, 1.0);
    ex.run(G, Vel{t, f.gx, f.gy, f.dgx, f.dgy, drho, f.vx, f.vy, f.dvx, f.dvy});
    S.forward({f.vx, f.vy, f.dvx, f.dvy});
    S.apply({{0, kDMX}, {1, kDMY}, {2, kDMX}, {3, kDMY}}, 0, {f.dx, f.dy, f.ddx, f.ddy}, 1.0);
    ex.run(G, Rho{t, f.dx, f.dy, f.ddx, f.ddy, drho, dc, f.P0, src, f.rx, f.ry, f.r, f.u, f.drx, f.dry, f.dr, f.du});
    if (!t.lossless) {
      S.forward({f.r, f.u, f.dr, f.du});
      S.apply({{0, kYDIS}, {1, kYABS}, {2, kYDIS}, {3, kYABS}}, 0, {f.Yr, f.Yu, f.YdR, f.Ydu}, 1.0);
    }
    ex.run(G, Pres{t, f.r, f.Yr, f.Yu, f.dr, f.YdR, f.Ydu, dc, f.p, nullptr, f.dp});
    ex.run(t.ns, Gather{t, f.dp, dP + (long long)it * t.ns});
  }
}

// Fields of one forward step that the reverse step needs: g_i = D+_i p_n,
// the divergences D-_i v_i, X = p_(n+1) / C and (lossy) Y_dis r, Y_abs u.
// Tape holds them for a run of consecutive steps ([steps][G] each).
struct Tape {
  double *gx, *gy, *dx, *dy, *X, *Yr, *Yu;
};

// Reverse-loop fields, all [G]
struct RevFields {
  double *pb, *Cp, *e1, *e2, *t1, *ub, *rbx, *rby, *dbx, *dby, *vbx, *vby, *fx, *fy, *ex, *ey, *qb;
  double *gC, *gtau, *geta, *grho, *grsx, *grsy;
};

// Copy the loop state (p, v_x, v_y, rho_x, rho_y) to or from a checkpoint
// [5][G].
struct StateCopy {
  const double* src[5];
  double* dst[5];
  long long G;
  QPAT_HD void operator()(long long u) const {
    const long long k = u / G, g = u - k * G;
    dst[k][g] = src[k][g];
  }
};

// Forward step it (loop index n = it - 1) of the gradient's forward sweep,
// writing its tape fields to slot k of tp.
template <class Ex>
void tape_step(Ex& ex, const Tables& t, Spectral<Ex>& S, const Fields& f, const Tape& tp, int it, int k) {
  const long long G = (long long)t.nx * t.ny, o = (long long)k * G;
  S.forward({f.p});
  S.apply({{0, kDPX}, {0, kDPY}}, 0, {tp.gx + o, tp.gy + o}, 1.0);
  ex.run(G, Vel{t, tp.gx + o, tp.gy + o, nullptr, nullptr, nullptr, f.vx, f.vy, nullptr, nullptr});
  S.forward({f.vx, f.vy});
  S.apply({{0, kDMX}, {1, kDMY}}, 0, {tp.dx + o, tp.dy + o}, 1.0);
  ex.run(G, Rho{t, tp.dx + o, tp.dy + o, nullptr, nullptr, nullptr, nullptr, f.P0, it <= 1, f.rx, f.ry, f.r, f.u,
                nullptr, nullptr, nullptr, nullptr});
  double* Yr = t.lossless ? nullptr : tp.Yr + o;
  double* Yu = t.lossless ? nullptr : tp.Yu + o;
  if (!t.lossless) {
    S.forward({f.r, f.u});
    S.apply({{0, kYDIS}, {1, kYABS}}, 0, {Yr, Yu}, 1.0);
  }
  ex.run(G, Pres{t, f.r, Yr, Yu, nullptr, nullptr, nullptr, nullptr, f.p, tp.X + o, nullptr});
}

// Transposed step it, reading the tape fields of step it from slot k.
template <class Ex>
void reverse_step(Ex& ex, const Tables& t, Spectral<Ex>& S, const Tape& tp, const RevFields& b, const double* W,
                  int it, int k) {
  const long long G = (long long)t.nx * t.ny, o = (long long)k * G;
  const double* Yr = t.lossless ? nullptr : tp.Yr + o;
  const double* Yu = t.lossless ? nullptr : tp.Yu + o;
  ex.run(t.ny, Scatter{t, W + (long long)it * t.ns, b.pb});
  ex.run(G, RevP{t, b.pb, tp.X + o, Yr, Yu, b.gC, b.geta, b.gtau, b.Cp, b.e1, b.e2});
  if (!t.lossless) {
    S.forward({b.e1, b.e2});
    S.apply({{0, kYDIS}, {1, kYABS}}, 1, {b.t1, b.ub}, 1.0);
  }
  ex.run(G, RevRho{t, b.Cp, b.t1, b.ub, tp.dx + o, tp.dy + o, it <= 1, b.rbx, b.rby, b.dbx, b.dby, b.grho, b.qb});
  S.forward({b.dbx, b.dby});
  S.apply({{0, kDMX}, {1, kDMY}}, 1, {b.ex, b.ey}, 1.0);
  ex.run(G, RevVel{t, b.ex, b.ey, tp.gx + o, tp.gy + o, b.vbx, b.vby, b.grsx, b.grsy, b.fx, b.fy});
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
template <class Ex>
void vjp_loop(Ex& ex, const Tables& t, Spectral<Ex>& S, const Fields& f, const Tape& tp, const RevFields& b, int K,
              double* ck, const double* W, double* g_c, double* g_rho) {
  const long long G = (long long)t.nx * t.ny;
  if (K >= t.nt) {
    for (int it = 0; it < t.nt; ++it) tape_step(ex, t, S, f, tp, it, it);
    for (int it = t.nt - 1; it >= 0; --it) reverse_step(ex, t, S, tp, b, W, it, it);
  } else {
    auto state = [&](int seg, bool save) {
      double* c = ck + (long long)seg * 5 * G;
      double* live[5] = {f.p, f.vx, f.vy, f.rx, f.ry};
      StateCopy op{};
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
  ex.run(G, Finish{t, b.gC, b.gtau, b.geta, b.qb, f.P0, b.grsx, b.grsy, b.grho, g_c, g_rho});
}

}  // namespace med
}  // namespace qpat
