// C ABI of the direct-QPAT propagation library (see include/qpat.h).
//
// A context owns the device tables and the workspace for up to max_batch
// problems on one grid and medium.  The forward operator H_a is the launch
// sequence of Section 3.2.3 (one row/column pass chain per time step, from
// n = -1 to Nt - 2); H_a^* runs the transposed steps in reverse (Section
// 3.2.4).  The composite maps chain the FP64 diffusion solve, the heating
// map and H_a / H_a^* (eqs. com_des, J_des, Lemma 1).
#include <math.h>
#include <string.h>

#include <algorithm>
#include <map>
#include <memory>
#include <cstdio>
#include <string>
#include <tuple>
#include <vector>

#include "qpat.h"
#include "qpat_internal.h"
#include "prop3d.h"
#include "multi.h"

using namespace qpat;

struct qpat_ctx {
  int prec = QPAT_FP32;
  cudaStream_t stream = nullptr;
  qpat_config cfg{};
  int dim = 2;
  int nx = 0, ny = 0, nz = 1, nxh = 0, pitch = 0, n0 = 0, n1 = 0, n2 = 1, pml = 0, ns = 0, nt = 0, maxb = 1;
  long long N = 0, G = 0;
  double dx = 0, dt = 0, c_ref = 0, c_max = 0;
  std::string err;
  std::vector<void*> dev_allocs;
  std::vector<void*> host_allocs;
  PropArgs<float> pf{};
  PropArgs<double> pd{};
  Prop3<float> p3f{};
  Prop3<double> p3d{};
  DAArgs da{};
  PCGWork pcg{};
  std::unique_ptr<MGHierarchy> mg;
  int* d_err = nullptr;
  int* h_err = nullptr;
  void* tw_p0 = nullptr;       // [B][N] prec: heating handed to H_a
  void* tw_hbar = nullptr;     // [B][N] prec: H_a^* output
  double* d_kappa = nullptr;   // [N] optical diffusion (qpat_set_kappa replaces it)
  double* d_phi = nullptr;     // [B][N]
  double* d_rhs = nullptr;     // [B][N]
  double* d_tmp = nullptr;     // [B][N]
  double* d_dot_partial = nullptr;
  double* d_dot_out = nullptr;
  double* h_dot_out = nullptr;
  // launch accounting and per-phase event timing
  long long launches = 0;
  long long last_pcg_iters = 0;
  int prof_phase = -1;
  cudaStream_t cap_stream = nullptr;
  std::map<int, std::pair<cudaGraphExec_t, long long>> graphs;   // (dir, batch) -> graph, kernels
  std::vector<cudaEvent_t> prof_events;
  size_t prof_used = 0;
  int medium_k = 0;            // checkpoint interval of the medium gradient (0: automatic)
};

namespace qpat {
bool ctx_view(const qpat_ctx* c, CtxView* v) {
  if (!c || !v) return false;
  v->prec = c->prec;
  v->dim = c->dim;
  v->n0 = c->n0;
  v->n1 = c->n1;
  v->n2 = c->dim == 3 ? c->n2 : 1;
  v->nt = c->nt;
  v->ns = c->ns;
  v->maxb = c->maxb;
  v->N = c->N;
  v->dx = c->dx;
  v->stream = c->stream;
  return true;
}
int ctx_fail(qpat_ctx* c, int st, const char* msg) {
  if (c) c->err = msg;
  return st;
}
const PropArgs<double>* ctx_tables64(const qpat_ctx* c, double* y, int* lossless, cudaStream_t* stream) {
  if (!c || c->prec != QPAT_FP64 || c->dim != 2) return nullptr;
  *y = c->cfg.y;
  *lossless = c->cfg.lossless;
  *stream = c->stream;
  return &c->pd;
}
const PropArgs<float>* ctx_tables32(const qpat_ctx* c, double* y, int* lossless, cudaStream_t* stream) {
  if (!c || c->prec != QPAT_FP32 || c->dim != 2) return nullptr;
  *y = c->cfg.y;
  *lossless = c->cfg.lossless;
  *stream = c->stream;
  return &c->pf;
}
void ctx_add_launches(qpat_ctx* c, long long n) {
  if (c) c->launches += n;
}
int ctx_medium_k(const qpat_ctx* c) { return c ? c->medium_k : 0; }
}  // namespace qpat

namespace {

qpat_status fail(qpat_ctx* c, qpat_status st, const std::string& msg) {
  if (c) c->err = msg;
  return st;
}

qpat_status cuda_fail(qpat_ctx* c, cudaError_t e, const char* where) {
  return fail(c, e == cudaErrorMemoryAllocation ? QPAT_ENOMEM : QPAT_ECUDA,
              std::string(where) + ": " + cudaGetErrorString(e));
}

#define QCK(expr)                                                  \
  do {                                                             \
    cudaError_t e_ = (expr);                                       \
    if (e_ != cudaSuccess) return cuda_fail(c, e_, #expr);         \
  } while (0)

#define QCK2(ctx, expr)                                            \
  do {                                                             \
    cudaError_t e_ = (expr);                                       \
    if (e_ != cudaSuccess) return cuda_fail(ctx, e_, #expr);       \
  } while (0)

template <typename P>
cudaError_t dalloc(qpat_ctx* c, P** p, size_t bytes) {
  void* v = nullptr;
  cudaError_t e = cudaMalloc(&v, bytes < 16 ? 16 : bytes);
  if (e == cudaSuccess) {
    c->dev_allocs.push_back(v);
    *p = reinterpret_cast<P*>(v);
  }
  return e;
}

cudaError_t dalloc_cb(void* owner, void** p, size_t bytes) { return dalloc((qpat_ctx*)owner, p, bytes); }

bool factor_plan(int L, FFTPlan& p) {
  p.L = L;
  p.nstages = 0;
  int r = L;
  int twos = 0;
  while (r % 2 == 0) { r /= 2; ++twos; }
  while (twos >= 3) { p.radix[p.nstages++] = 8; twos -= 3; }
  if (twos == 2) p.radix[p.nstages++] = 4;
  if (twos == 1) p.radix[p.nstages++] = 2;
  for (int q : {3, 5, 7}) {
    while (r % q == 0) {
      if (p.nstages >= kMaxStages) return false;
      p.radix[p.nstages++] = q;
      r /= q;
    }
  }
  return r == 1 && p.nstages <= kMaxStages;
}

template <typename T>
PropArgs<T>& args(qpat_ctx* c);
template <>
PropArgs<float>& args<float>(qpat_ctx* c) { return c->pf; }
template <>
PropArgs<double>& args<double>(qpat_ctx* c) { return c->pd; }

template <typename T>
Prop3<T>& args3(qpat_ctx* c);
template <>
Prop3<float>& args3<float>(qpat_ctx* c) { return c->p3f; }
template <>
Prop3<double>& args3<double>(qpat_ctx* c) { return c->p3d; }

// Sensor tables for a 2D or 3D node grid: the gather form (2^d corners per
// sensor, multilinear weights) and the transposed scatter as a deterministic
// per-row gather over the grid points the sensors touch; rows are indexed
// k ny + j.
template <typename T>
qpat_status build_sensors(qpat_ctx* c, const double* pos, const int** d_sidx, const T** d_sw, const int** d_rowptr,
                          const int** d_pcol, const int** d_pent, const int** d_esens, const T** d_ew) {
  const int d = c->dim, nc = 1 << d;
  const int Nax[3] = {c->nx, c->ny, c->nz};
  std::vector<int> sidx((size_t)nc * c->ns);
  std::vector<T> sw((size_t)nc * c->ns);
  std::vector<std::tuple<int, int, int, double>> ent;   // row, col, sensor, weight
  for (int s = 0; s < c->ns; ++s) {
    int base[3] = {0, 0, 0};
    double frac[3] = {0, 0, 0};
    for (int ax = 0; ax < d; ++ax) {
      const double g = pos[d * s + ax] / c->dx + (Nax[ax] - 1) / 2.0;
      const int j0 = (int)floor(g);
      const double f = g - j0;
      if (!(g == g) || j0 < 0 || j0 > Nax[ax] - 1 || (j0 == Nax[ax] - 1 && f > 0))
        return fail(c, QPAT_EINVAL, "sensor " + std::to_string(s) + " lies outside the grid");
      base[ax] = j0;
      frac[ax] = f;
    }
    for (int corner = 0; corner < nc; ++corner) {
      double wgt = 1.0;
      int idx[3] = {0, 0, 0};
      for (int ax = 0; ax < d; ++ax) {
        const int bit = (corner >> ax) & 1;
        wgt *= bit ? frac[ax] : 1.0 - frac[ax];
        idx[ax] = std::min(base[ax] + bit, Nax[ax] - 1);
      }
      const long long g = ((long long)idx[2] * c->ny + idx[1]) * c->nx + idx[0];
      sidx[(size_t)nc * s + corner] = (int)g;
      sw[(size_t)nc * s + corner] = (T)wgt;
      if (wgt != 0.0) ent.emplace_back(idx[2] * c->ny + idx[1], idx[0], s, wgt);
    }
  }
  std::sort(ent.begin(), ent.end());
  const int nrows = c->nz * c->ny;
  std::vector<int> rowptr(nrows + 1, 0), pcol, pent, esens;
  std::vector<T> ew;
  int prev_r = -1, prev_c = -1;
  for (size_t e = 0; e < ent.size(); ++e) {
    const int r = std::get<0>(ent[e]), col = std::get<1>(ent[e]);
    if (r != prev_r || col != prev_c) {
      pcol.push_back(col);
      pent.push_back((int)e);
      rowptr[r + 1] += 1;
      prev_r = r;
      prev_c = col;
    }
    esens.push_back(std::get<2>(ent[e]));
    ew.push_back((T)std::get<3>(ent[e]));
  }
  pent.push_back((int)ent.size());
  for (int r = 0; r < nrows; ++r) rowptr[r + 1] += rowptr[r];
  int *a_sidx, *a_rowptr, *a_pcol, *a_pent, *a_esens;
  T *a_sw, *a_ew;
  QCK(dalloc(c, &a_sidx, sidx.size() * sizeof(int)));
  QCK(dalloc(c, &a_sw, sw.size() * sizeof(T)));
  QCK(dalloc(c, &a_rowptr, rowptr.size() * sizeof(int)));
  QCK(dalloc(c, &a_pcol, std::max<size_t>(1, pcol.size()) * sizeof(int)));
  QCK(dalloc(c, &a_pent, pent.size() * sizeof(int)));
  QCK(dalloc(c, &a_esens, std::max<size_t>(1, esens.size()) * sizeof(int)));
  QCK(dalloc(c, &a_ew, std::max<size_t>(1, ew.size()) * sizeof(T)));
  QCK(cudaMemcpy(a_sidx, sidx.data(), sidx.size() * sizeof(int), cudaMemcpyHostToDevice));
  QCK(cudaMemcpy(a_sw, sw.data(), sw.size() * sizeof(T), cudaMemcpyHostToDevice));
  QCK(cudaMemcpy(a_rowptr, rowptr.data(), rowptr.size() * sizeof(int), cudaMemcpyHostToDevice));
  if (!pcol.empty()) QCK(cudaMemcpy(a_pcol, pcol.data(), pcol.size() * sizeof(int), cudaMemcpyHostToDevice));
  QCK(cudaMemcpy(a_pent, pent.data(), pent.size() * sizeof(int), cudaMemcpyHostToDevice));
  if (!esens.empty()) QCK(cudaMemcpy(a_esens, esens.data(), esens.size() * sizeof(int), cudaMemcpyHostToDevice));
  if (!ew.empty()) QCK(cudaMemcpy(a_ew, ew.data(), ew.size() * sizeof(T), cudaMemcpyHostToDevice));
  *d_sidx = a_sidx; *d_sw = a_sw; *d_rowptr = a_rowptr; *d_pcol = a_pcol; *d_pent = a_pent; *d_esens = a_esens;
  *d_ew = a_ew;
  return QPAT_OK;
}

// 3D device tables + workspace for working precision T.
template <typename T>
qpat_status build_context3(qpat_ctx* c, const qpat_medium* med, const double* sensor_xy) {
  typedef typename V2<T>::t C;
  Prop3<T>& a = args3<T>(c);
  a.nx = c->nx; a.ny = c->ny; a.nz = c->nz; a.nxh = c->nxh; a.pitch = c->pitch; a.pml = c->pml;
  a.n0 = c->n0; a.n1 = c->n1; a.n2 = c->n2; a.ns = c->ns; a.nt = c->nt;
  if (!factor_plan(c->nx, a.px) || !factor_plan(c->ny, a.py) || !factor_plan(c->nz, a.pz))
    return fail(c, QPAT_EINVAL, "FFT extents must factor into 2, 3, 5 and 7");
  a.cby = a.cbz = 1;
  for (int cb : {8, 4, 2}) {
    if (prop3_smem_col<T>(c->ny, cb) <= 100 * 1024 && cb * 4 <= c->nxh) { a.cby = cb; break; }
  }
  for (int cb : {8, 4, 2}) {
    if (prop3_smem_col<T>(c->nz, cb) <= 100 * 1024 && cb * 4 <= c->nxh) { a.cbz = cb; break; }
  }
  if (prop3_smem_col<T>(c->ny, a.cby) > 227 * 1024 || prop3_smem_col<T>(c->nz, a.cbz) > 227 * 1024)
    return fail(c, QPAT_EINVAL, "grid too large for the shared-memory FFT passes");
  a.dt = (T)c->dt;
  const long long G = c->G;
  const int B = c->maxb;
  Tables3<T> o{};
  for (T** p : {&o.Cc, &o.rho0, &o.dtrsx, &o.dtrsy, &o.dtrsz, &o.tau, &o.eta}) QCK(dalloc(c, p, G * sizeof(T)));
  QCK(dalloc(c, &o.ax, c->nx * sizeof(T)));
  QCK(dalloc(c, &o.asx, c->nx * sizeof(T)));
  QCK(dalloc(c, &o.ay, c->ny * sizeof(T)));
  QCK(dalloc(c, &o.asy, c->ny * sizeof(T)));
  QCK(dalloc(c, &o.az, c->nz * sizeof(T)));
  QCK(dalloc(c, &o.asz, c->nz * sizeof(T)));
  const long long KT = (long long)c->nz * c->ny * c->nxh;
  for (T** p : {&o.kap, &o.kp1, &o.kp2}) QCK(dalloc(c, p, KT * sizeof(T)));
  QCK(dalloc(c, &o.shxp, c->nxh * sizeof(C)));
  QCK(dalloc(c, &o.shxm, c->nxh * sizeof(C)));
  QCK(dalloc(c, &o.shyp, c->ny * sizeof(C)));
  QCK(dalloc(c, &o.shym, c->ny * sizeof(C)));
  QCK(dalloc(c, &o.shzp, c->nz * sizeof(C)));
  QCK(dalloc(c, &o.shzm, c->nz * sizeof(C)));
  QCK(dalloc(c, &o.twx, c->nx * sizeof(C)));
  QCK(dalloc(c, &o.twy, c->ny * sizeof(C)));
  QCK(dalloc(c, &o.twz, c->nz * sizeof(C)));
  double *dc = nullptr, *drho = nullptr, *dal = nullptr;
  QCK(cudaMalloc(&dc, G * sizeof(double)));
  QCK(cudaMalloc(&drho, G * sizeof(double)));
  QCK(cudaMalloc(&dal, G * sizeof(double)));
  QCK(cudaMemcpyAsync(dc, med->c, G * sizeof(double), cudaMemcpyHostToDevice, c->stream));
  QCK(cudaMemcpyAsync(drho, med->rho, G * sizeof(double), cudaMemcpyHostToDevice, c->stream));
  if (!c->cfg.lossless) QCK(cudaMemcpyAsync(dal, med->alpha0_db, G * sizeof(double), cudaMemcpyHostToDevice, c->stream));
  QCK(build_tables3<T>(o, dc, drho, dal, c->nx, c->ny, c->nz, c->nxh, c->pml, c->dx, c->dt, c->c_ref,
                       c->cfg.pml_alpha, c->cfg.y, c->cfg.lossless, c->stream));
  QCK(cudaStreamSynchronize(c->stream));
  cudaFree(dc);
  cudaFree(drho);
  cudaFree(dal);
  a.Cc = o.Cc; a.rho0 = o.rho0; a.dtrsx = o.dtrsx; a.dtrsy = o.dtrsy; a.dtrsz = o.dtrsz; a.tau = o.tau;
  a.eta = o.eta; a.ax = o.ax; a.asx = o.asx; a.ay = o.ay; a.asy = o.asy; a.az = o.az; a.asz = o.asz;
  a.kap = o.kap; a.kp1 = o.kp1; a.kp2 = o.kp2;
  a.shxp = o.shxp; a.shxm = o.shxm; a.shyp = o.shyp; a.shym = o.shym; a.shzp = o.shzp; a.shzm = o.shzm;
  a.twx = o.twx; a.twy = o.twy; a.twz = o.twz;
  qpat_status st = build_sensors<T>(c, sensor_xy, &a.sidx, &a.sw, &a.rowptr, &a.pcol, &a.pent, &a.esens, &a.ew);
  if (st != QPAT_OK) return st;
  a.gstride = G;
  a.slot = (long long)c->nz * c->ny * c->pitch;
  a.sstride = 3 * a.slot;
  for (T** p : {&a.vx, &a.vy, &a.vz, &a.rx, &a.ry, &a.rz, &a.pbuf}) QCK(dalloc(c, p, (size_t)B * G * sizeof(T)));
  C* spec;
  QCK(dalloc(c, &spec, (size_t)B * a.sstride * sizeof(C)));
  QCK(cudaMemset(spec, 0, (size_t)B * a.sstride * sizeof(C)));
  a.spec = spec;
  QCK(dalloc(c, &c->tw_p0, (size_t)B * c->N * sizeof(T)));
  QCK(dalloc(c, &c->tw_hbar, (size_t)B * c->N * sizeof(T)));
  IoPtrs<T>* io = nullptr;
  QCK(dalloc(c, &io, sizeof(IoPtrs<T>)));
  a.io = io;
  a.err = c->d_err;
  prop3_init_attributes<T>();
  a.fast_x = !c->cfg.generic_fft && fast3_supported(c->nx, (int)sizeof(T));
  a.fast_y = !c->cfg.generic_fft && fast3_supported(c->ny, (int)sizeof(T));
  a.fast_z = !c->cfg.generic_fft && fast3_supported(c->nz, (int)sizeof(T));
  prop3_init_fast<T>(a);
  return QPAT_OK;
}

// Device tables + workspace for working precision T.
template <typename T>
qpat_status build_context(qpat_ctx* c, const qpat_medium* med, const double* sensor_xy) {
  typedef typename V2<T>::t C;
  PropArgs<T>& a = args<T>(c);
  a.nx = c->nx; a.ny = c->ny; a.nxh = c->nxh; a.pitch = c->pitch; a.pml = c->pml;
  a.n0 = c->n0; a.n1 = c->n1; a.ns = c->ns; a.nt = c->nt;
  if (!factor_plan(c->nx, a.px) || !factor_plan(c->ny, a.py))
    return fail(c, QPAT_EINVAL, "FFT extents must factor into 2, 3, 5 and 7");
  // column tile width: widest of 8/4/2/1 columns whose tile fits 100 KB of shared memory
  a.cb = 1;
  for (int cb : {8, 4, 2}) {
    if (col_smem_bytes<T>(c->ny, cb) <= 100 * 1024 && cb * 4 <= c->nxh) { a.cb = cb; break; }
  }
  if (row_smem_bytes<T>(c->nx) > 227 * 1024 || col_smem_bytes<T>(c->ny, a.cb) > 227 * 1024)
    return fail(c, QPAT_EINVAL, "grid too large for the shared-memory FFT passes");
  a.dt = (T)c->dt;
  const long long G = c->G, N = c->N;
  const int B = c->maxb;
  TableOut<T> o{};
  QCK(dalloc(c, &o.Cc, G * sizeof(T)));
  QCK(dalloc(c, &o.rho0, G * sizeof(T)));
  QCK(dalloc(c, &o.dtrsx, G * sizeof(T)));
  QCK(dalloc(c, &o.dtrsy, G * sizeof(T)));
  QCK(dalloc(c, &o.tau, G * sizeof(T)));
  QCK(dalloc(c, &o.eta, G * sizeof(T)));
  QCK(dalloc(c, &o.ax, c->nx * sizeof(T)));
  QCK(dalloc(c, &o.asx, c->nx * sizeof(T)));
  QCK(dalloc(c, &o.ay, c->ny * sizeof(T)));
  QCK(dalloc(c, &o.asy, c->ny * sizeof(T)));
  const long long KT = (long long)c->ny * c->nxh;
  QCK(dalloc(c, &o.kap, KT * sizeof(T)));
  QCK(dalloc(c, &o.kp1, KT * sizeof(T)));
  QCK(dalloc(c, &o.kp2, KT * sizeof(T)));
  QCK(dalloc(c, &o.shxp, c->nxh * sizeof(C)));
  QCK(dalloc(c, &o.shxm, c->nxh * sizeof(C)));
  QCK(dalloc(c, &o.shyp, c->ny * sizeof(C)));
  QCK(dalloc(c, &o.shym, c->ny * sizeof(C)));
  QCK(dalloc(c, &o.twx, c->nx * sizeof(C)));
  QCK(dalloc(c, &o.twy, c->ny * sizeof(C)));
  // FP64 medium staging
  double *dc = nullptr, *drho = nullptr, *dal = nullptr;
  QCK(cudaMalloc(&dc, G * sizeof(double)));
  QCK(cudaMalloc(&drho, G * sizeof(double)));
  QCK(cudaMalloc(&dal, G * sizeof(double)));
  QCK(cudaMemcpyAsync(dc, med->c, G * sizeof(double), cudaMemcpyHostToDevice, c->stream));
  QCK(cudaMemcpyAsync(drho, med->rho, G * sizeof(double), cudaMemcpyHostToDevice, c->stream));
  if (!c->cfg.lossless) QCK(cudaMemcpyAsync(dal, med->alpha0_db, G * sizeof(double), cudaMemcpyHostToDevice, c->stream));
  QCK(build_tables<T>(o, dc, drho, dal, c->nx, c->ny, c->nxh, c->pml, c->dx, c->dt, c->c_ref,
                      c->cfg.pml_alpha, c->cfg.y, c->cfg.lossless, c->stream));
  QCK(cudaStreamSynchronize(c->stream));
  cudaFree(dc);
  cudaFree(drho);
  cudaFree(dal);
  a.Cc = o.Cc; a.rho0 = o.rho0; a.dtrsx = o.dtrsx; a.dtrsy = o.dtrsy; a.tau = o.tau; a.eta = o.eta;
  a.ax = o.ax; a.asx = o.asx; a.ay = o.ay; a.asy = o.asy;
  a.kap = o.kap; a.kp1 = o.kp1; a.kp2 = o.kp2;
  a.shxp = o.shxp; a.shxm = o.shxm; a.shyp = o.shyp; a.shym = o.shym;
  a.twx = o.twx; a.twy = o.twy;
  // length-specialised passes where the extent has them (unless disabled)
  a.fast_rows = !c->cfg.generic_fft && fast_rows_supported(c->nx, (int)sizeof(T));
  a.fast_cols = !c->cfg.generic_fft && fast_cols_supported(c->ny, (int)sizeof(T));

  // sensors: bilinear weights on the node grid (gather form) and the
  // transposed scatter as a per-row, per-point gather (deterministic)
  std::vector<int> sidx(4 * (size_t)c->ns);
  std::vector<T> sw(4 * (size_t)c->ns);
  std::vector<std::tuple<int, int, int, double>> ent;   // row, col, sensor, weight
  for (int s = 0; s < c->ns; ++s) {
    int base[2];
    double frac[2];
    const int Nax[2] = {c->nx, c->ny};
    for (int ax = 0; ax < 2; ++ax) {
      const double g = sensor_xy[2 * s + ax] / c->dx + (Nax[ax] - 1) / 2.0;
      const int j0 = (int)floor(g);
      const double f = g - j0;
      if (!(g == g) || j0 < 0 || j0 > Nax[ax] - 1 || (j0 == Nax[ax] - 1 && f > 0))
        return fail(c, QPAT_EINVAL, "sensor " + std::to_string(s) + " lies outside the grid");
      base[ax] = j0;
      frac[ax] = f;
    }
    for (int corner = 0; corner < 4; ++corner) {
      const int bx = corner & 1, by = (corner >> 1) & 1;
      const double wgt = (bx ? frac[0] : 1.0 - frac[0]) * (by ? frac[1] : 1.0 - frac[1]);
      const int ix = std::min(base[0] + bx, c->nx - 1), iy = std::min(base[1] + by, c->ny - 1);
      sidx[4 * s + corner] = iy * c->nx + ix;
      sw[4 * s + corner] = (T)wgt;
      if (wgt != 0.0) ent.emplace_back(iy, ix, s, wgt);
    }
  }
  std::sort(ent.begin(), ent.end());
  std::vector<int> rowptr(c->ny + 1, 0), pcol, pent, esens;
  std::vector<T> ew;
  {
    int prev_r = -1, prev_c = -1;
    for (size_t e = 0; e < ent.size(); ++e) {
      const int r = std::get<0>(ent[e]), col = std::get<1>(ent[e]);
      if (r != prev_r || col != prev_c) {
        pcol.push_back(col);
        pent.push_back((int)e);
        rowptr[r + 1] += 1;
        prev_r = r;
        prev_c = col;
      }
      esens.push_back(std::get<2>(ent[e]));
      ew.push_back((T)std::get<3>(ent[e]));
    }
    pent.push_back((int)ent.size());
    for (int r = 0; r < c->ny; ++r) rowptr[r + 1] += rowptr[r];
  }
  int *d_sidx, *d_rowptr, *d_pcol, *d_pent, *d_esens;
  T *d_sw, *d_ew;
  QCK(dalloc(c, &d_sidx, sidx.size() * sizeof(int)));
  QCK(dalloc(c, &d_sw, sw.size() * sizeof(T)));
  QCK(dalloc(c, &d_rowptr, rowptr.size() * sizeof(int)));
  QCK(dalloc(c, &d_pcol, std::max<size_t>(1, pcol.size()) * sizeof(int)));
  QCK(dalloc(c, &d_pent, pent.size() * sizeof(int)));
  QCK(dalloc(c, &d_esens, std::max<size_t>(1, esens.size()) * sizeof(int)));
  QCK(dalloc(c, &d_ew, std::max<size_t>(1, ew.size()) * sizeof(T)));
  QCK(cudaMemcpy(d_sidx, sidx.data(), sidx.size() * sizeof(int), cudaMemcpyHostToDevice));
  QCK(cudaMemcpy(d_sw, sw.data(), sw.size() * sizeof(T), cudaMemcpyHostToDevice));
  QCK(cudaMemcpy(d_rowptr, rowptr.data(), rowptr.size() * sizeof(int), cudaMemcpyHostToDevice));
  if (!pcol.empty()) QCK(cudaMemcpy(d_pcol, pcol.data(), pcol.size() * sizeof(int), cudaMemcpyHostToDevice));
  QCK(cudaMemcpy(d_pent, pent.data(), pent.size() * sizeof(int), cudaMemcpyHostToDevice));
  if (!esens.empty()) QCK(cudaMemcpy(d_esens, esens.data(), esens.size() * sizeof(int), cudaMemcpyHostToDevice));
  if (!ew.empty()) QCK(cudaMemcpy(d_ew, ew.data(), ew.size() * sizeof(T), cudaMemcpyHostToDevice));
  a.sidx = d_sidx; a.sw = d_sw; a.rowptr = d_rowptr; a.pcol = d_pcol; a.pent = d_pent; a.esens = d_esens; a.ew = d_ew;

  // workspace
  a.gstride = G;
  a.sstride = 2LL * c->ny * c->pitch;
  T *vx, *vy, *rx, *ry, *pbuf;
  C* spec;
  QCK(dalloc(c, &vx, (size_t)B * G * sizeof(T)));
  QCK(dalloc(c, &vy, (size_t)B * G * sizeof(T)));
  QCK(dalloc(c, &rx, (size_t)B * G * sizeof(T)));
  QCK(dalloc(c, &ry, (size_t)B * G * sizeof(T)));
  QCK(dalloc(c, &pbuf, (size_t)B * G * sizeof(T)));
  QCK(dalloc(c, &spec, (size_t)B * a.sstride * sizeof(C)));
  QCK(cudaMemset(spec, 0, (size_t)B * a.sstride * sizeof(C)));
  a.vx = vx; a.vy = vy; a.rx = rx; a.ry = ry; a.pbuf = pbuf; a.spec = spec;
  QCK(dalloc(c, &c->tw_p0, (size_t)B * N * sizeof(T)));
  QCK(dalloc(c, &c->tw_hbar, (size_t)B * N * sizeof(T)));
  IoPtrs<T>* io = nullptr;
  QCK(dalloc(c, &io, sizeof(IoPtrs<T>)));
  a.io = io;
  a.err = c->d_err;
  prop_init_attributes<T>(c->nx, c->ny, a.fast_rows, a.fast_cols);
  return QPAT_OK;
}

template <typename T>
void zero_state(qpat_ctx* c, int batch, cudaStream_t s) {
  PropArgs<T>& a = args<T>(c);
  const size_t bytes = (size_t)batch * c->G * sizeof(T);
  cudaMemsetAsync(a.vx, 0, bytes, s);
  cudaMemsetAsync(a.vy, 0, bytes, s);
  cudaMemsetAsync(a.rx, 0, bytes, s);
  cudaMemsetAsync(a.ry, 0, bytes, s);
}

// Launch one pass on stream s, counting it and, when this phase is being
// profiled (direct launches only), bracketing it with CUDA events.
template <typename T>
void pass(qpat_ctx* c, const PropArgs<T>& a, int phase, int batch, bool is_row, cudaStream_t s, long long& count) {
  const bool prof = (c->prof_phase == phase);
  if (prof) {
    while (c->prof_events.size() < c->prof_used + 2) {
      cudaEvent_t e;
      if (cudaEventCreate(&e) != cudaSuccess) break;
      c->prof_events.push_back(e);
    }
    if (c->prof_events.size() >= c->prof_used + 2) cudaEventRecord(c->prof_events[c->prof_used], s);
  }
  if (is_row) launch_row<T>(a, phase, batch, s);
  else launch_col<T>(a, phase, batch, s);
  ++count;
  if (prof && c->prof_events.size() >= c->prof_used + 2) {
    cudaEventRecord(c->prof_events[c->prof_used + 1], s);
    c->prof_used += 2;
  }
}

// H_a: launch sequence of the forward loop n = -1 .. Nt - 2 (Section 3.2.3),
// enqueued on stream s; the caller's buffers are read through a.io.
// Checkpointing (K > 0): after loop iteration n with (n + 1) % K == 0 the
// full state is copied to checkpoint m = (n + 1)/K - 1 (store = true), or the
// loop starts after checkpoint `resume_m` from its restored state, producing
// samples (resume_m + 1) K .. Nt - 1 only.
template <typename T>
long long seq_forward(qpat_ctx* c, int batch, cudaStream_t s, int K = 0, bool store = false, int resume_m = -1) {
  PropArgs<T> a = args<T>(c);
  long long cnt = 0;
  const int nt = c->nt;
  int n_first = 0;
  if (resume_m >= 0) {
    launch_ckpt_copy<T>(a, batch, resume_m, 0, s);
    n_first = (resume_m + 1) * K;
  } else {
    zero_state<T>(c, batch, s);
  }
  auto checkpoint = [&](int n) {
    if (store && K > 0 && (n + 1) % K == 0) launch_ckpt_copy<T>(a, batch, (n + 1) / K - 1, 1, s);
  };
  if (!c->cfg.lossless) {
    if (resume_m < 0) {
      a.n = 0;
      a.flags = kSkipInput | kSource;          // step n = -1 from zero fields
      pass<T>(c, a, F_R3, batch, true, s, cnt);
      a.flags = 0;
      pass<T>(c, a, F_C3, batch, false, s, cnt);
    }
    for (int n = n_first; n <= nt - 2; ++n) {
      a.n = n;
      a.flags = 0;
      pass<T>(c, a, F_R1, batch, true, s, cnt);    // p_n
      pass<T>(c, a, F_C1, batch, false, s, cnt);   // sample n, d/dr^+ p_n
      pass<T>(c, a, F_R2, batch, true, s, cnt);    // v^(n+1/2)
      pass<T>(c, a, F_C2, batch, false, s, cnt);   // d/dr^- v
      a.flags = (n == 0) ? kSource : 0;
      pass<T>(c, a, F_R3, batch, true, s, cnt);    // rho^(n+1)
      a.flags = 0;
      pass<T>(c, a, F_C3, batch, false, s, cnt);   // Y_dis, Y_abs
      checkpoint(n);
    }
    a.n = nt - 1;
    a.flags = kSkipOutput;
    pass<T>(c, a, F_R1, batch, true, s, cnt);      // p_(Nt-1)
  } else {
    if (resume_m < 0) {
      a.n = 0;
      a.flags = kSkipInput | kSource;
      pass<T>(c, a, F_R3L, batch, true, s, cnt);   // p_0
    }
    for (int n = n_first; n <= nt - 2; ++n) {
      a.n = n;
      a.flags = 0;
      pass<T>(c, a, F_C1, batch, false, s, cnt);
      pass<T>(c, a, F_R2, batch, true, s, cnt);
      pass<T>(c, a, F_C2, batch, false, s, cnt);
      a.flags = (n == 0) ? kSource : 0;
      pass<T>(c, a, F_R3L, batch, true, s, cnt);   // p_(n+1)
      checkpoint(n);
    }
    a.n = nt - 1;
  }
  launch_gather<T>(a, batch, s);
  return cnt + 1;
}

// H_a^*: transposed steps in reverse, n = Nt - 2 .. -1 (Section 3.2.4).
template <typename T>
long long seq_adjoint(qpat_ctx* c, int batch, cudaStream_t s) {
  PropArgs<T> a = args<T>(c);
  long long cnt = 0;
  zero_state<T>(c, batch, s);
  const int nt = c->nt;
  for (int n = nt - 2; n >= -1; --n) {
    a.n = n + 1;                                   // the sample p_(n+1) produced
    const int first = (n == nt - 2) ? kSkipInput : 0;
    const int acc = (n == 0) ? kAccWrite : (n == -1 ? kAccAdd : 0);
    const int last = (n == -1) ? kSkipOutput : 0;
    if (!c->cfg.lossless) {
      a.flags = first;
      pass<T>(c, a, A_R1, batch, true, s, cnt);
      a.flags = 0;
      pass<T>(c, a, A_C2, batch, false, s, cnt);
      a.flags = acc | last;
      pass<T>(c, a, A_R3, batch, true, s, cnt);
    } else {
      a.flags = first | acc | last;
      pass<T>(c, a, A_R1L, batch, true, s, cnt);
    }
    if (n > -1) {
      a.flags = 0;
      pass<T>(c, a, A_C4, batch, false, s, cnt);
      pass<T>(c, a, A_R5, batch, true, s, cnt);
      pass<T>(c, a, A_C6, batch, false, s, cnt);
    }
  }
  return cnt;
}

// The launch sequence of H_a (dir 0) or H_a^* (dir 1) for the context's
// dimension and precision, enqueued on s; returns the kernel count.
long long seq_any(qpat_ctx* c, int dir, int batch, cudaStream_t s) {
  const bool ll = c->cfg.lossless != 0;
  if (c->dim == 3) {
    if (c->prec == QPAT_FP32)
      return dir == 0 ? seq3_forward<float>(c->p3f, batch, ll, s) : seq3_adjoint<float>(c->p3f, batch, ll, s);
    return dir == 0 ? seq3_forward<double>(c->p3d, batch, ll, s) : seq3_adjoint<double>(c->p3d, batch, ll, s);
  }
  if (c->prec == QPAT_FP32) return dir == 0 ? seq_forward<float>(c, batch, s) : seq_adjoint<float>(c, batch, s);
  return dir == 0 ? seq_forward<double>(c, batch, s) : seq_adjoint<double>(c, batch, s);
}

// Run H_a (dir 0) or H_a^* (dir 1) on the caller's buffers.  The launch
// sequence is captured once per (direction, batch) into a CUDA graph on a
// private stream and replayed on the context's stream; only a one-thread
// kernel that writes the buffer pointers into the device struct a.io
// precedes each replay.  With graphs disabled, or while a pass is being
// profiled, the sequence is launched directly.
template <typename T>
qpat_status run_prop(qpat_ctx* c, int dir, int batch, const T* p0, T* data, const T* w, T* p0adj) {
  IoPtrs<T>* io = const_cast<IoPtrs<T>*>(c->dim == 3 ? args3<T>(c).io : args<T>(c).io);
  launch_set_io<T>(io, p0, data, w, p0adj, nullptr, c->stream);
  QCK(cudaGetLastError());
  const bool direct = c->cfg.no_graphs || c->prof_phase >= 0;
  if (direct) {
    c->launches += seq_any(c, dir, batch, c->stream);
    QCK(cudaGetLastError());
    return QPAT_OK;
  }
  const int key = dir * 1000000 + batch;
  auto it = c->graphs.find(key);
  if (it == c->graphs.end()) {
    if (!c->cap_stream) QCK(cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking));
    QCK(cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeThreadLocal));
    const long long n = seq_any(c, dir, batch, c->cap_stream);
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamEndCapture(c->cap_stream, &g);
    if (e != cudaSuccess) return cuda_fail(c, e, "graph capture");
    cudaGraphExec_t ex = nullptr;
    e = cudaGraphInstantiate(&ex, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return cuda_fail(c, e, "graph instantiation");
    it = c->graphs.emplace(key, std::make_pair(ex, n)).first;
  }
  QCK(cudaGraphLaunch(it->second.first, c->stream));
  c->launches += it->second.second;
  return QPAT_OK;
}

// Checkpointed forward (store) or resumed forward, launched directly.
template <typename T>
qpat_status run_ckpt(qpat_ctx* c, int batch, const T* p0, T* data, T* ckpt, int K, int resume_m) {
  PropArgs<T>& a = args<T>(c);
  IoPtrs<T>* io = const_cast<IoPtrs<T>*>(a.io);
  launch_set_io<T>(io, p0, data, nullptr, nullptr, ckpt, c->stream);
  c->launches += seq_forward<T>(c, batch, c->stream, K, resume_m < 0, resume_m);
  QCK(cudaGetLastError());
  return QPAT_OK;
}

qpat_status check_batch(qpat_ctx* c, int batch) {
  if (!c) return QPAT_EINVAL;
  if (batch < 1 || batch > c->maxb)
    return fail(c, QPAT_EINVAL, "batch " + std::to_string(batch) + " outside 1.." + std::to_string(c->maxb));
  return QPAT_OK;
}

qpat_status solve_da(qpat_ctx* c, int batch, const double* mu, const double* rhs, double* x) {
  cudaError_t e = cudaSuccess;
  const int used = pcg_solve(c->da, mu, batch, rhs, x, c->pcg, c->cfg.pcg_max_iter, c->cfg.pcg_tol, c->stream, &e);
  c->last_pcg_iters = used;
  if (e != cudaSuccess) return cuda_fail(c, e, "diffusion solve");
  if (used < 0) return fail(c, QPAT_ENOCONV, "diffusion solve reached its iteration cap");
  return QPAT_OK;
}

qpat_status fluence(qpat_ctx* c, int batch, const double* mu, unsigned illum, double* phi) {
  QCK(da_rhs_from_sides(c->da, illum, batch, c->d_rhs, c->stream));
  return solve_da(c, batch, mu, c->d_rhs, phi);
}

}  // namespace

extern "C" {

qpat_status qpat_create(const qpat_config* cfg, const qpat_medium* med, const double* sensor_xy, int ns,
                        qpat_precision prec, void* stream, qpat_ctx** out) {
  if (!out) return QPAT_EINVAL;
  *out = nullptr;
  if (!cfg || !med || !med->c || !med->rho || !med->kappa || !sensor_xy || ns < 1) return QPAT_EINVAL;
  qpat_ctx* c = new qpat_ctx();
  c->cfg = *cfg;
  c->prec = prec;
  c->stream = (cudaStream_t)stream;
  auto bad = [&](qpat_status st, const std::string& m) {
    fprintf(stderr, "qpat_create: %s\n", m.c_str());
    qpat_destroy(c);
    return st;
  };
  if (prec != QPAT_FP32 && prec != QPAT_FP64) return bad(QPAT_EINVAL, "unknown precision");
  if (cfg->n[0] < 1 || cfg->n[1] < 1 || cfg->pml < 0) return bad(QPAT_EINVAL, "bad grid size");
  if (!(cfg->dx > 0) || !(cfg->dt > 0)) return bad(QPAT_EINVAL, "dx and dt must be positive");
  if (cfg->nt < 2) return bad(QPAT_EINVAL, "nt must be at least 2");
  c->n0 = cfg->n[0];
  c->n1 = cfg->n[1];
  c->dim = cfg->n2 > 0 ? 3 : 2;
  c->n2 = c->dim == 3 ? cfg->n2 : 1;
  c->pml = cfg->pml;
  c->nx = c->n0 + 2 * c->pml;
  c->ny = c->n1 + 2 * c->pml;
  c->nz = c->dim == 3 ? c->n2 + 2 * c->pml : 1;
  if (c->nx % 2 || c->ny % 2 || (c->dim == 3 && c->nz % 2)) return bad(QPAT_EINVAL, "FFT grid extents must be even");
  if (c->nx < 8 || c->ny < 8 || (c->dim == 3 && c->nz < 8))
    return bad(QPAT_EINVAL, "FFT grid extents must be at least 8");
  c->nxh = c->nx / 2 + 1;
  c->pitch = (c->nxh + 3) / 4 * 4;
  c->N = (long long)c->n0 * c->n1 * c->n2;
  c->G = (long long)c->nx * c->ny * c->nz;
  c->ns = ns;
  c->nt = cfg->nt;
  c->dx = cfg->dx;
  c->dt = cfg->dt;
  c->maxb = cfg->max_batch > 0 ? cfg->max_batch : 1;
  if (!(c->cfg.pml_alpha > 0)) c->cfg.pml_alpha = 2.0;
  if (!(c->cfg.gamma_d > 0)) c->cfg.gamma_d = c->dim == 3 ? 0.25 : 1.0 / M_PI;
  if (c->cfg.pcg_max_iter <= 0) c->cfg.pcg_max_iter = 20000;
  if (!(c->cfg.pcg_tol > 0)) c->cfg.pcg_tol = 1e-13;
  if (!c->cfg.lossless) {
    if (!med->alpha0_db) return bad(QPAT_EINVAL, "alpha0_db is required unless lossless");
    if (!(cfg->y > 1.0 && cfg->y < 3.0) || fabs(cfg->y - 2.0) < 1e-12)
      return bad(QPAT_EINVAL, "power-law exponent y must lie in (1, 3) and differ from 2");
  }
  double cmax = 0.0;
  for (long long g = 0; g < c->G; ++g) {
    const double v = med->c[g], r = med->rho[g];
    if (!(v > 0) || !(r > 0)) return bad(QPAT_EINVAL, "c and rho must be positive and finite");
    if (!c->cfg.lossless && !(med->alpha0_db[g] >= 0)) return bad(QPAT_EINVAL, "alpha0 must be >= 0");
    cmax = std::max(cmax, v);
  }
  for (long long g = 0; g < c->N; ++g)
    if (!(med->kappa[g] > 0)) return bad(QPAT_EINVAL, "kappa must be positive and finite");
  c->c_max = cmax;
  c->c_ref = cfg->c_ref > 0 ? cfg->c_ref : cmax;
  if (cmax * c->dt / c->dx > 2.0 / (M_PI * sqrt((double)c->dim)))
    return bad(QPAT_EUNSTABLE, "c_max dt / dx exceeds 2 / (pi sqrt d)");

  cudaError_t e;
#define QCKC(expr)                                                                  \
  do {                                                                              \
    e = (expr);                                                                     \
    if (e != cudaSuccess) return bad(e == cudaErrorMemoryAllocation ? QPAT_ENOMEM : QPAT_ECUDA, \
                                     std::string(#expr) + ": " + cudaGetErrorString(e)); \
  } while (0)
  QCKC(dalloc(c, &c->d_err, sizeof(int)));
  QCKC(cudaMemset(c->d_err, 0, sizeof(int)));
  QCKC(cudaMallocHost(&c->h_err, sizeof(int)));
  c->host_allocs.push_back(c->h_err);
  qpat_status st;
  if (c->dim == 3)
    st = (prec == QPAT_FP32) ? build_context3<float>(c, med, sensor_xy) : build_context3<double>(c, med, sensor_xy);
  else
    st = (prec == QPAT_FP32) ? build_context<float>(c, med, sensor_xy) : build_context<double>(c, med, sensor_xy);
  if (st != QPAT_OK) return bad(st, c->err);

  // diffusion solve
  const int B = c->maxb;
  const long long N = c->N;
  c->da.n0 = c->n0;
  c->da.n1 = c->n1;
  c->da.n2 = c->n2;
  c->da.dim = c->dim;
  c->da.N = (int)N;
  c->da.h = c->dx;
  c->da.hd = c->dim == 3 ? c->dx * c->dx * c->dx : c->dx * c->dx;
  c->da.gamma = c->cfg.gamma_d;
  double *diag0, *cxf, *cyf, *czf, *bside, *dkappa;
  QCKC(dalloc(c, &diag0, N * sizeof(double)));
  QCKC(dalloc(c, &cxf, N * sizeof(double)));
  QCKC(dalloc(c, &cyf, N * sizeof(double)));
  QCKC(dalloc(c, &czf, N * sizeof(double)));
  QCKC(dalloc(c, &bside, 2 * c->dim * N * sizeof(double)));
  QCKC(dalloc(c, &dkappa, N * sizeof(double)));
  QCKC(cudaMemcpy(dkappa, med->kappa, N * sizeof(double), cudaMemcpyHostToDevice));
  c->d_kappa = dkappa;
  QCKC(da_setup(c->da, diag0, cxf, cyf, czf, bside, dkappa, c->stream));
  PCGWork& w = c->pcg;
  for (double** p : {&w.x, &w.r, &w.z, &w.p, &w.q, &w.dinv, &w.b}) QCKC(dalloc(c, p, B * N * sizeof(double)));
  QCKC(dalloc(c, &w.mu, B * N * sizeof(double)));
  QCKC(dalloc(c, &w.partial, (size_t)B * kPCGBlocks * 4 * sizeof(double)));
  QCKC(dalloc(c, &w.scal, (size_t)B * 8 * sizeof(double)));
  w.use_graphs = !c->cfg.no_graphs;
  if (!c->cfg.da_jacobi) {
    c->mg.reset(new MGHierarchy());
    QCKC(mg_setup(*c->mg, c->da, dkappa, B, dalloc_cb, c, c->stream));
    // a grid with an odd extent has no coarse level: diagonal preconditioning
    w.mg = c->mg->nlev > 1 ? c->mg.get() : nullptr;
  }
  QCKC(cudaMallocHost(&w.hostscal, (size_t)B * 8 * sizeof(double)));
  c->host_allocs.push_back(w.hostscal);
  QCKC(dalloc(c, &c->d_phi, B * N * sizeof(double)));
  QCKC(dalloc(c, &c->d_rhs, B * N * sizeof(double)));
  QCKC(dalloc(c, &c->d_tmp, B * N * sizeof(double)));
  QCKC(dalloc(c, &c->d_dot_partial, (size_t)B * kPartials * 4 * sizeof(double)));
  QCKC(dalloc(c, &c->d_dot_out, (size_t)B * sizeof(double)));
  QCKC(cudaMallocHost(&c->h_dot_out, (size_t)B * sizeof(double)));
  c->host_allocs.push_back(c->h_dot_out);
  QCKC(cudaStreamSynchronize(c->stream));
#undef QCKC
  *out = c;
  return QPAT_OK;
}

qpat_status qpat_destroy(qpat_ctx* c) {
  if (!c) return QPAT_OK;
  cudaStreamSynchronize(c->stream);
  for (auto& kv : c->graphs) cudaGraphExecDestroy(kv.second.first);
  if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
  if (c->pcg.chunk) cudaGraphExecDestroy(c->pcg.chunk);
  if (c->pcg.cap) cudaStreamDestroy(c->pcg.cap);
  for (void* p : c->dev_allocs) cudaFree(p);
  for (void* p : c->host_allocs) cudaFreeHost(p);
  for (cudaEvent_t e : c->prof_events) cudaEventDestroy(e);
  delete c;
  return QPAT_OK;
}

qpat_status qpat_set_stream(qpat_ctx* c, void* stream) {
  if (!c) return QPAT_EINVAL;
  c->stream = (cudaStream_t)stream;
  return QPAT_OK;
}

const char* qpat_last_error(const qpat_ctx* c) { return c ? c->err.c_str() : "null context"; }

qpat_status qpat_get_sizes(const qpat_ctx* c, long long out[6]) {
  if (!c || !out) return QPAT_EINVAL;
  out[0] = c->nx;
  out[1] = c->ny;
  out[2] = c->N;
  out[3] = c->ns;
  out[4] = c->nt;
  out[5] = c->maxb;
  return QPAT_OK;
}

qpat_status qpat_sync(qpat_ctx* c) {
  if (!c) return QPAT_EINVAL;
  QCK(cudaMemcpyAsync(c->h_err, c->d_err, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  QCK(cudaStreamSynchronize(c->stream));
  if (*c->h_err) {
    QCK(cudaMemsetAsync(c->d_err, 0, sizeof(int), c->stream));
    QCK(cudaStreamSynchronize(c->stream));
    if (*c->h_err & 1) return fail(c, QPAT_ENONFINITE, "non-finite value in the acoustic fields");
    if (*c->h_err & 2) return fail(c, QPAT_ETIMEOUT, "a bounded wait for a bulk copy gave up");
  }
  return QPAT_OK;
}

qpat_status qpat_acoustic_forward(qpat_ctx* c, int batch, const void* p0, void* data) {
  qpat_status st = check_batch(c, batch);
  if (st != QPAT_OK) return st;
  if (!p0 || !data) return fail(c, QPAT_EINVAL, "null buffer");
  return c->prec == QPAT_FP32 ? run_prop<float>(c, 0, batch, (const float*)p0, (float*)data, nullptr, nullptr)
                              : run_prop<double>(c, 0, batch, (const double*)p0, (double*)data, nullptr, nullptr);
}

qpat_status qpat_acoustic_adjoint(qpat_ctx* c, int batch, const void* data, void* p0_adj) {
  qpat_status st = check_batch(c, batch);
  if (st != QPAT_OK) return st;
  if (!p0_adj || !data) return fail(c, QPAT_EINVAL, "null buffer");
  return c->prec == QPAT_FP32
             ? run_prop<float>(c, 1, batch, nullptr, nullptr, (const float*)data, (float*)p0_adj)
             : run_prop<double>(c, 1, batch, nullptr, nullptr, (const double*)data, (double*)p0_adj);
}

qpat_status qpat_da_solve(qpat_ctx* c, int batch, const double* mu, unsigned illum, double* phi) {
  qpat_status st = check_batch(c, batch);
  if (st != QPAT_OK) return st;
  if (!mu || !phi) return fail(c, QPAT_EINVAL, "null buffer");
  if (illum == 0 || illum >= (1u << (2 * c->dim)))
    return fail(c, QPAT_EINVAL, "illumination mask must select sides 0 .. 2d-1");
  return fluence(c, batch, mu, illum, phi);
}

qpat_status qpat_forward(qpat_ctx* c, int batch, const double* mu, unsigned illum, void* data, double* phi0_out) {
  qpat_status st = qpat_da_solve(c, batch, mu, illum, c ? c->d_phi : nullptr);
  if (st != QPAT_OK) return st;
  if (!data) return fail(c, QPAT_EINVAL, "null buffer");
  const int N = (int)c->N;
  // heating h = mu o phi (eq. h), p0 = h (Gamma = 1)
  if (c->prec == QPAT_FP32) QCK(da_heating_T<float>(batch, N, mu, c->d_phi, nullptr, nullptr, (float*)c->tw_p0, c->stream));
  else QCK(da_heating_T<double>(batch, N, mu, c->d_phi, nullptr, nullptr, (double*)c->tw_p0, c->stream));
  if (phi0_out)
    QCK(cudaMemcpyAsync(phi0_out, c->d_phi, (size_t)batch * N * sizeof(double), cudaMemcpyDeviceToDevice, c->stream));
  return qpat_acoustic_forward(c, batch, c->tw_p0, data);
}

}  // extern "C"

namespace {
// J_o dmu into the context's heating buffer: dh = dmu o phi0 + mu o dphi with
// A(mu) dphi = -h^2 dmu o phi0 (eq. dh_des).
qpat_status jvp_heating(qpat_ctx* c, int batch, const double* mu, const double* phi0, const double* dmu,
                        unsigned illum) {
  const int N = (int)c->N;
  qpat_status st;
  if (!phi0) {
    st = qpat_da_solve(c, batch, mu, illum, c->d_phi);
    if (st != QPAT_OK) return st;
    phi0 = c->d_phi;
  }
  QCK(da_hadamard(batch, N, -c->da.hd, dmu, phi0, c->d_rhs, c->stream));
  st = solve_da(c, batch, mu, c->d_rhs, c->d_tmp);
  if (st != QPAT_OK) return st;
  if (c->prec == QPAT_FP32) QCK(da_heating_T<float>(batch, N, dmu, phi0, mu, c->d_tmp, (float*)c->tw_p0, c->stream));
  else QCK(da_heating_T<double>(batch, N, dmu, phi0, mu, c->d_tmp, (double*)c->tw_p0, c->stream));
  return QPAT_OK;
}
}  // namespace

extern "C" {

qpat_status qpat_jvp(qpat_ctx* c, int batch, const double* mu, const double* phi0, const double* dmu, unsigned illum,
                     void* dP) {
  qpat_status st = check_batch(c, batch);
  if (st != QPAT_OK) return st;
  if (!mu || !dmu || !dP) return fail(c, QPAT_EINVAL, "null buffer");
  st = jvp_heating(c, batch, mu, phi0, dmu, illum);
  if (st != QPAT_OK) return st;
  return qpat_acoustic_forward(c, batch, c->tw_p0, dP);
}

qpat_status qpat_vjp(qpat_ctx* c, int batch, const double* mu, const double* phi0, const void* w, unsigned illum,
                     double* g) {
  qpat_status st = check_batch(c, batch);
  if (st != QPAT_OK) return st;
  if (!mu || !w || !g) return fail(c, QPAT_EINVAL, "null buffer");
  const int N = (int)c->N;
  st = qpat_acoustic_adjoint(c, batch, w, c->tw_hbar);
  if (st != QPAT_OK) return st;
  if (!phi0) {
    st = qpat_da_solve(c, batch, mu, illum, c->d_phi);
    if (st != QPAT_OK) return st;
    phi0 = c->d_phi;
  }
  // A H~ = -h^2 mu o hbar (eq. system_adjoint); g = phi0 o (hbar + H~) (eq. prodtproj)
  const double sc = -c->da.hd;
  if (c->prec == QPAT_FP32) QCK(da_adjoint_rhs<float>(batch, N, sc, mu, (const float*)c->tw_hbar, c->d_rhs, c->stream));
  else QCK(da_adjoint_rhs<double>(batch, N, sc, mu, (const double*)c->tw_hbar, c->d_rhs, c->stream));
  st = solve_da(c, batch, mu, c->d_rhs, c->d_tmp);
  if (st != QPAT_OK) return st;
  if (c->prec == QPAT_FP32) QCK(da_adjoint_out<float>(batch, N, phi0, (const float*)c->tw_hbar, c->d_tmp, g, c->stream));
  else QCK(da_adjoint_out<double>(batch, N, phi0, (const double*)c->tw_hbar, c->d_tmp, g, c->stream));
  return QPAT_OK;
}

// kappa derivatives (Lemma 1, delta-kappa rows) ---------------------------------

qpat_status qpat_set_kappa(qpat_ctx* c, const double* kappa) {
  if (!c) return QPAT_EINVAL;
  if (!kappa) return fail(c, QPAT_EINVAL, "null buffer");
  QCK(cudaMemcpyAsync(c->d_kappa, kappa, (size_t)c->N * sizeof(double), cudaMemcpyDeviceToDevice, c->stream));
  QCK(da_setup(c->da, const_cast<double*>(c->da.diag0), const_cast<double*>(c->da.cxf),
               const_cast<double*>(c->da.cyf), const_cast<double*>(c->da.czf), const_cast<double*>(c->da.bside),
               c->d_kappa, c->stream));
  if (c->mg) {
    c->mg->lev[0].A = c->da;
    QCK(mg_rekappa(*c->mg, c->stream));
  }
  QCK(cudaStreamSynchronize(c->stream));
  return QPAT_OK;
}

qpat_status qpat_jvp_kappa(qpat_ctx* c, int batch, const double* mu, const double* phi0, const double* dkappa,
                           unsigned illum, void* dP) {
  qpat_status st = check_batch(c, batch);
  if (st != QPAT_OK) return st;
  if (!mu || !dkappa || !dP) return fail(c, QPAT_EINVAL, "null buffer");
  const int N = (int)c->N;
  if (!phi0) {
    st = qpat_da_solve(c, batch, mu, illum, c->d_phi);
    if (st != QPAT_OK) return st;
    phi0 = c->d_phi;
  }
  // A dphi = delta-b - delta-A phi0 (eq. dPhi), dh = mu o dphi (eq. fr)
  QCK(da_kappa_source(c->da, c->d_kappa, batch, phi0, dkappa, illum, c->d_rhs, c->stream));
  st = solve_da(c, batch, mu, c->d_rhs, c->d_tmp);
  if (st != QPAT_OK) return st;
  if (c->prec == QPAT_FP32) QCK(da_heating_T<float>(batch, N, mu, c->d_tmp, nullptr, nullptr, (float*)c->tw_p0, c->stream));
  else QCK(da_heating_T<double>(batch, N, mu, c->d_tmp, nullptr, nullptr, (double*)c->tw_p0, c->stream));
  return qpat_acoustic_forward(c, batch, c->tw_p0, dP);
}

qpat_status qpat_vjp_kappa(qpat_ctx* c, int batch, const double* mu, const double* phi0, const void* w,
                           unsigned illum, double* g) {
  qpat_status st = check_batch(c, batch);
  if (st != QPAT_OK) return st;
  if (!mu || !w || !g) return fail(c, QPAT_EINVAL, "null buffer");
  const int N = (int)c->N;
  st = qpat_acoustic_adjoint(c, batch, w, c->tw_hbar);
  if (st != QPAT_OK) return st;
  if (!phi0) {
    st = qpat_da_solve(c, batch, mu, illum, c->d_phi);
    if (st != QPAT_OK) return st;
    phi0 = c->d_phi;
  }
  // psi = A^-1 (mu o hbar); g = <delta-b - delta-A phi0, psi> per cell
  if (c->prec == QPAT_FP32) QCK(da_adjoint_rhs<float>(batch, N, 1.0, mu, (const float*)c->tw_hbar, c->d_rhs, c->stream));
  else QCK(da_adjoint_rhs<double>(batch, N, 1.0, mu, (const double*)c->tw_hbar, c->d_rhs, c->stream));
  st = solve_da(c, batch, mu, c->d_rhs, c->d_tmp);
  if (st != QPAT_OK) return st;
  QCK(da_kappa_grad(c->da, c->d_kappa, batch, phi0, c->d_tmp, illum, 1.0, g, c->stream));
  return QPAT_OK;
}

}  // extern "C"

// Optical halves of the composite maps for one problem, with caller buffers,
// so that a caller holding several illuminations can batch their acoustic
// propagations (declared in qpat_internal.h).
namespace qpat {

int optics_forward(qpat_ctx* c, const double* mu, unsigned illum, double* phi, void* h) {
  qpat_status st = qpat_da_solve(c, 1, mu, illum, phi);
  if (st != QPAT_OK) return st;
  const int N = (int)c->N;
  if (c->prec == QPAT_FP32) QCK(da_heating_T<float>(1, N, mu, phi, nullptr, nullptr, (float*)h, c->stream));
  else QCK(da_heating_T<double>(1, N, mu, phi, nullptr, nullptr, (double*)h, c->stream));
  return QPAT_OK;
}

int optics_jvp2(qpat_ctx* c, const double* mu, const double* phi0, const double* dmu, const double* dkappa,
                unsigned illum, void* dh) {
  const int N = (int)c->N;
  // right-hand side of A dphi: -h^d dmu o phi0 (delta-mu) + delta-b - delta-A phi0 (delta-kappa)
  if (dkappa) QCK(da_kappa_source(c->da, c->d_kappa, 1, phi0, dkappa, illum, c->d_rhs, c->stream));
  else QCK(cudaMemsetAsync(c->d_rhs, 0, (size_t)N * sizeof(double), c->stream));
  if (dmu) {
    QCK(da_hadamard(1, N, -c->da.hd, dmu, phi0, c->d_tmp, c->stream));
    QCK(da_axpy(N, 1.0, c->d_tmp, c->d_rhs, c->stream));
  }
  qpat_status st = solve_da(c, 1, mu, c->d_rhs, c->d_tmp);
  if (st != QPAT_OK) return st;
  // dh = dmu o phi0 + mu o dphi
  const double* a1 = dmu ? dmu : mu;
  const double* b1 = dmu ? phi0 : c->d_tmp;
  const double* a2 = dmu ? mu : nullptr;
  if (c->prec == QPAT_FP32) QCK(da_heating_T<float>(1, N, a1, b1, a2, c->d_tmp, (float*)dh, c->stream));
  else QCK(da_heating_T<double>(1, N, a1, b1, a2, c->d_tmp, (double*)dh, c->stream));
  return QPAT_OK;
}

int optics_vjp2(qpat_ctx* c, const double* mu, const double* phi0, const void* hbar, unsigned illum, double* g_mu,
                double* g_kappa) {
  const int N = (int)c->N;
  const double sc = -c->da.hd;
  // A H~ = -h^d mu o hbar; psi = A^-1 (mu o hbar) = -H~ / h^d
  if (c->prec == QPAT_FP32) QCK(da_adjoint_rhs<float>(1, N, sc, mu, (const float*)hbar, c->d_rhs, c->stream));
  else QCK(da_adjoint_rhs<double>(1, N, sc, mu, (const double*)hbar, c->d_rhs, c->stream));
  qpat_status st = solve_da(c, 1, mu, c->d_rhs, c->d_tmp);
  if (st != QPAT_OK) return st;
  if (g_mu) {
    if (c->prec == QPAT_FP32) QCK(da_adjoint_out<float>(1, N, phi0, (const float*)hbar, c->d_tmp, g_mu, c->stream));
    else QCK(da_adjoint_out<double>(1, N, phi0, (const double*)hbar, c->d_tmp, g_mu, c->stream));
  }
  if (g_kappa) QCK(da_kappa_grad(c->da, c->d_kappa, 1, phi0, c->d_tmp, illum, -1.0 / c->da.hd, g_kappa, c->stream));
  return QPAT_OK;
}

}  // namespace qpat

extern "C" {

qpat_status qpat_dot(qpat_ctx* c, int batch, long long len, const void* a, const void* b, double* out) {
  qpat_status st = check_batch(c, batch);
  if (st != QPAT_OK) return st;
  if (!a || !b || !out || len < 0) return fail(c, QPAT_EINVAL, "bad dot arguments");
  if (c->prec == QPAT_FP32)
    QCK(dot_compensated<float>(batch, len, (const float*)a, (const float*)b, c->d_dot_partial, c->d_dot_out, c->stream));
  else
    QCK(dot_compensated<double>(batch, len, (const double*)a, (const double*)b, c->d_dot_partial, c->d_dot_out,
                                c->stream));
  QCK(cudaMemcpyAsync(c->h_dot_out, c->d_dot_out, batch * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  QCK(cudaStreamSynchronize(c->stream));
  for (int i = 0; i < batch; ++i) out[i] = c->h_dot_out[i];
  return QPAT_OK;
}

qpat_status qpat_ckpt_bytes(const qpat_ctx* c, int batch, int K, long long* bytes) {
  if (!c || !bytes || K < 1 || batch < 1) return QPAT_EINVAL;
  const long long M = (c->nt - 1) / K;
  const long long per = c->prec == QPAT_FP32 ? ckpt_elems<float>(c->pf) * 4 : ckpt_elems<double>(c->pd) * 8;
  *bytes = M * batch * per;
  return QPAT_OK;
}

qpat_status qpat_acoustic_forward_ckpt(qpat_ctx* c, int batch, const void* p0, void* data, int K, void* ckpt) {
  qpat_status st = check_batch(c, batch);
  if (st != QPAT_OK) return st;
  if (!p0 || !data || !ckpt || K < 1) return fail(c, QPAT_EINVAL, "bad checkpoint arguments");
  if (c->dim != 2) return fail(c, QPAT_EINVAL, "checkpointing is implemented for 2D grids");
  return c->prec == QPAT_FP32 ? run_ckpt<float>(c, batch, (const float*)p0, (float*)data, (float*)ckpt, K, -1)
                              : run_ckpt<double>(c, batch, (const double*)p0, (double*)data, (double*)ckpt, K, -1);
}

qpat_status qpat_acoustic_resume(qpat_ctx* c, int batch, const void* ckpt, int K, int m, void* data) {
  qpat_status st = check_batch(c, batch);
  if (st != QPAT_OK) return st;
  if (c->dim != 2) return fail(c, QPAT_EINVAL, "checkpointing is implemented for 2D grids");
  if (!data || !ckpt || K < 1 || m < 0 || m >= (c->nt - 1) / K)
    return fail(c, QPAT_EINVAL, "bad resume arguments (checkpoint index out of range)");
  return c->prec == QPAT_FP32
             ? run_ckpt<float>(c, batch, nullptr, (float*)data, (float*)const_cast<void*>(ckpt), K, m)
             : run_ckpt<double>(c, batch, nullptr, (double*)data, (double*)const_cast<void*>(ckpt), K, m);
}


}  // extern "C"

// ---------------------------------------------------------------------------
// Groups: several contexts (e.g. different grids) propagated concurrently in
// one CUDA graph, each context's time loop a parallel branch.
// ---------------------------------------------------------------------------
struct qpat_group {
  std::vector<qpat_ctx*> ctxs;
  cudaStream_t cap = nullptr;
  cudaEvent_t fork = nullptr;
  std::vector<cudaEvent_t> join;
  std::map<std::vector<int>, std::pair<cudaGraphExec_t, long long>> graphs;
  qpat_group_shape shape{1, 144, 576, 1};
};

namespace {

template <typename T>
void set_io_for(qpat_ctx* c, int dir, const void* in, void* out, cudaStream_t s) {
  IoPtrs<T>* io = const_cast<IoPtrs<T>*>(c->dim == 3 ? args3<T>(c).io : args<T>(c).io);
  if (dir == 0) launch_set_io<T>(io, (const T*)in, (T*)out, nullptr, nullptr, nullptr, s);
  else launch_set_io<T>(io, nullptr, nullptr, (const T*)in, (T*)out, nullptr, s);
}

// ---- multi-problem launches (multi.h) --------------------------------------
struct MMember {
  qpat_ctx* c;
  int slot, batch, nt;
};

// The members a multi-problem sequence can serve: every member with work is a
// 2D FP32 context on a square grid whose extent has a slot, with the
// length-specialised passes selected, slots distinct, absorption on all or
// off on all.  Empty when any member does not qualify.
std::vector<MMember> multi_members(const qpat_group* g, const int* batches) {
  std::vector<MMember> mm;
  int used = 0, lossless = -1;
  for (size_t i = 0; i < g->ctxs.size(); ++i) {
    qpat_ctx* c = g->ctxs[i];
    if (batches[i] == 0) continue;
    const int slot = multi_slot_of(c->nx);
    if (c->prec != QPAT_FP32 || c->dim != 2 || c->nx != c->ny || slot < 0 || !c->pf.fast_rows ||
        !c->pf.fast_cols || (used >> slot) & 1 || (lossless >= 0 && lossless != (c->cfg.lossless != 0)))
      return {};
    used |= 1 << slot;
    lossless = c->cfg.lossless != 0;
    mm.push_back({c, slot, batches[i], c->nt});
  }
  if (mm.empty() || multi_prepare() != (int)cudaSuccess) return {};
  return mm;
}

// One multi-problem launch of `phase`: act(member, n, flags) says whether the
// member takes part and sets its time index and flags.  Returns the launches.
template <class Act>
long long multi_pass(const std::vector<MMember>& mm, const qpat_group_shape& sh, int phase, bool row, Act act,
                     cudaStream_t s) {
  MultiArgs m{};
  int tot = 0;
  for (int slot = 0; slot < kMultiSlots; ++slot) {
    m.first[slot] = tot;
    m.per[slot] = 1;
    for (const MMember& e : mm) {
      if (e.slot != slot) continue;
      int n = 0, flags = 0;
      if (!act(e, n, flags)) break;
      m.a[slot] = e.c->pf;
      m.a[slot].n = n;
      m.a[slot].flags = flags;
      const int per = row ? multi_row_tiles(slot, sh.row_block, e.c->ny) : multi_col_tiles(slot, sh.col_block, e.c->nxh);
      m.per[slot] = per;
      tot += per * e.batch;
    }
  }
  m.first[kMultiSlots] = tot;
  m.reverse = sh.largest_first != 0;
  if (tot == 0) return 0;
  if (row) launch_multi_row(m, phase, sh.row_block, tot, s);
  else launch_multi_col(m, phase, sh.col_block, tot, s);
  return 1;
}

// H_a of every member in one launch sequence: the members' loops are aligned
// on the time index n (Section 3.2.3 loop from n = -1); a member drops out of
// the launches once its own Nt is reached, and its last sample is gathered
// at the end (its state is no longer touched by then).
long long seq_multi_forward(const std::vector<MMember>& mm, const qpat_group_shape& sh, cudaStream_t s) {
  long long cnt = 0;
  int maxnt = 0;
  const bool lossless = mm[0].c->cfg.lossless != 0;
  for (const MMember& e : mm) {
    zero_state<float>(e.c, e.batch, s);
    maxnt = std::max(maxnt, e.nt);
  }
  auto all = [](int flags) {
    return [flags](const MMember&, int& n, int& f) { n = 0; f = flags; return true; };
  };
  if (!lossless) {
    cnt += multi_pass(mm, sh, F_R3, true, all(kSkipInput | kSource), s);    // step n = -1
    cnt += multi_pass(mm, sh, F_C3, false, all(0), s);
    for (int n = 0; n <= maxnt - 1; ++n) {
      cnt += multi_pass(mm, sh, F_R1, true, [n](const MMember& e, int& nn, int& f) {
        if (n > e.nt - 1) return false;
        nn = n;
        f = (n == e.nt - 1) ? kSkipOutput : 0;                             // p_(Nt-1), last pass
        return true;
      }, s);
      auto step = [n](int flags) {
        return [n, flags](const MMember& e, int& nn, int& f) {
          if (n > e.nt - 2) return false;
          nn = n;
          f = flags;
          return true;
        };
      };
      cnt += multi_pass(mm, sh, F_C1, false, step(0), s);
      cnt += multi_pass(mm, sh, F_R2, true, step(0), s);
      cnt += multi_pass(mm, sh, F_C2, false, step(0), s);
      cnt += multi_pass(mm, sh, F_R3, true, step(n == 0 ? kSource : 0), s);
      cnt += multi_pass(mm, sh, F_C3, false, step(0), s);
    }
  } else {
    cnt += multi_pass(mm, sh, F_R3L, true, all(kSkipInput | kSource), s);   // p_0
    for (int n = 0; n <= maxnt - 2; ++n) {
      auto step = [n](int flags) {
        return [n, flags](const MMember& e, int& nn, int& f) {
          if (n > e.nt - 2) return false;
          nn = n;
          f = flags;
          return true;
        };
      };
      cnt += multi_pass(mm, sh, F_C1, false, step(0), s);
      cnt += multi_pass(mm, sh, F_R2, true, step(0), s);
      cnt += multi_pass(mm, sh, F_C2, false, step(0), s);
      cnt += multi_pass(mm, sh, F_R3L, true, step(n == 0 ? kSource : 0), s);
    }
  }
  for (const MMember& e : mm) {
    PropArgs<float> a = e.c->pf;
    a.n = e.nt - 1;
    launch_gather<float>(a, e.batch, s);
    ++cnt;
  }
  return cnt;
}

// H_a^* of every member: the transposed steps in reverse, aligned so that
// every member reaches n = -1 in the same launch (Section 3.2.4).
long long seq_multi_adjoint(const std::vector<MMember>& mm, const qpat_group_shape& sh, cudaStream_t s) {
  long long cnt = 0;
  int maxnt = 0;
  const bool lossless = mm[0].c->cfg.lossless != 0;
  for (const MMember& e : mm) {
    zero_state<float>(e.c, e.batch, s);
    maxnt = std::max(maxnt, e.nt);
  }
  for (int n = maxnt - 2; n >= -1; --n) {
    // kind 0: first pass of the step, 1: the source-adjoint pass, 2: both
    // (lossless), 3: the others
    auto act = [n](int kind) {
      return [n, kind](const MMember& e, int& nn, int& f) {
        if (n > e.nt - 2) return false;
        nn = n + 1;                                                         // the sample p_(n+1)
        const int first = (n == e.nt - 2) ? kSkipInput : 0;
        const int acc = (n == 0) ? kAccWrite : (n == -1 ? kAccAdd : 0);
        const int last = (n == -1) ? kSkipOutput : 0;
        f = kind == 0 ? first : kind == 1 ? (acc | last) : kind == 2 ? (first | acc | last) : 0;
        return true;
      };
    };
    if (!lossless) {
      cnt += multi_pass(mm, sh, A_R1, true, act(0), s);
      cnt += multi_pass(mm, sh, A_C2, false, act(3), s);
      cnt += multi_pass(mm, sh, A_R3, true, act(1), s);
    } else {
      cnt += multi_pass(mm, sh, A_R1L, true, act(2), s);
    }
    if (n > -1) {
      cnt += multi_pass(mm, sh, A_C4, false, act(3), s);
      cnt += multi_pass(mm, sh, A_R5, true, act(3), s);
      cnt += multi_pass(mm, sh, A_C6, false, act(3), s);
    }
  }
  return cnt;
}

// The launch sequence of a group call on the capture stream: one multi-problem
// sequence when the shape asks for it and the members qualify, else each
// member's own sequence as a parallel branch.
long long seq_group(qpat_group* g, int dir, const int* batches, bool multi) {
  if (multi) {
    std::vector<MMember> mm = multi_members(g, batches);
    return dir == 0 ? seq_multi_forward(mm, g->shape, g->cap) : seq_multi_adjoint(mm, g->shape, g->cap);
  }
  long long kernels = 0;
  cudaEventRecord(g->fork, g->cap);
  for (size_t i = 0; i < g->ctxs.size(); ++i) {
    if (batches[i] == 0) continue;
    qpat_ctx* c = g->ctxs[i];
    cudaStreamWaitEvent(c->cap_stream, g->fork, 0);
    kernels += seq_any(c, dir, batches[i], c->cap_stream);
    cudaEventRecord(g->join[i], c->cap_stream);
    cudaStreamWaitEvent(g->cap, g->join[i], 0);
  }
  return kernels;
}

bool shape_valid(const qpat_group_shape& sh) {
  return (sh.multi == 0 || sh.multi == 1) && (sh.row_block == 144 || sh.row_block == 288) &&
         (sh.col_block == 288 || sh.col_block == 576) && (sh.largest_first == 0 || sh.largest_first == 1);
}

}  // namespace

extern "C" {

qpat_status qpat_group_create(int n, qpat_ctx* const* ctxs, qpat_group** out) {
  if (!out || n < 1 || !ctxs) return QPAT_EINVAL;
  *out = nullptr;
  qpat_group* g = new qpat_group();
  for (int i = 0; i < n; ++i) {
    if (!ctxs[i]) { delete g; return QPAT_EINVAL; }
    g->ctxs.push_back(ctxs[i]);
  }
  if (cudaStreamCreateWithFlags(&g->cap, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&g->fork, cudaEventDisableTiming) != cudaSuccess) {
    delete g;
    return QPAT_ECUDA;
  }
  g->join.resize(n);
  for (int i = 0; i < n; ++i) {
    if (cudaEventCreateWithFlags(&g->join[i], cudaEventDisableTiming) != cudaSuccess) return QPAT_ECUDA;
    if (!ctxs[i]->cap_stream && cudaStreamCreateWithFlags(&ctxs[i]->cap_stream, cudaStreamNonBlocking) != cudaSuccess)
      return QPAT_ECUDA;
  }
  *out = g;
  return QPAT_OK;
}

qpat_status qpat_group_destroy(qpat_group* g) {
  if (!g) return QPAT_OK;
  cudaStreamSynchronize(g->cap);
  for (auto& kv : g->graphs) cudaGraphExecDestroy(kv.second.first);
  for (cudaEvent_t e : g->join) cudaEventDestroy(e);
  if (g->fork) cudaEventDestroy(g->fork);
  if (g->cap) cudaStreamDestroy(g->cap);
  delete g;
  return QPAT_OK;
}

qpat_status qpat_group_propagate(qpat_group* g, int dir, const int* batches, const void* const* in, void* const* out,
                                 void* stream) {
  if (!g || !batches || !in || !out || (dir != 0 && dir != 1)) return QPAT_EINVAL;
  const int n = (int)g->ctxs.size();
  cudaStream_t s = (cudaStream_t)stream;
  std::vector<int> key{dir};
  for (int i = 0; i < n; ++i) {
    qpat_ctx* c = g->ctxs[i];
    if (batches[i] < 0 || batches[i] > c->maxb) return fail(c, QPAT_EINVAL, "group batch out of range");
    if (batches[i] > 0 && (!in[i] || !out[i])) return fail(c, QPAT_EINVAL, "null group buffer");
    if (c->prof_phase >= 0) return fail(c, QPAT_EINVAL, "profiling is not available in group calls");
    key.push_back(batches[i]);
  }
  for (int i = 0; i < n; ++i) {
    qpat_ctx* c = g->ctxs[i];
    c->stream = s;
    if (batches[i] == 0) continue;
    if (c->prec == QPAT_FP32) set_io_for<float>(c, dir, in[i], out[i], s);
    else set_io_for<double>(c, dir, in[i], out[i], s);
  }
  const bool multi = g->shape.multi && !multi_members(g, batches).empty();
  key.push_back(multi ? 1 : 0);
  if (multi) {
    key.push_back(g->shape.row_block);
    key.push_back(g->shape.col_block);
    key.push_back(g->shape.largest_first);
  }
  auto it = g->graphs.find(key);
  if (it == g->graphs.end()) {
    qpat_ctx* c0 = g->ctxs[0];
    cudaError_t e = cudaStreamBeginCapture(g->cap, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return cuda_fail(c0, e, "group capture");
    const long long kernels = seq_group(g, dir, batches, multi);
    cudaGraph_t graph = nullptr;
    e = cudaStreamEndCapture(g->cap, &graph);
    if (e != cudaSuccess) return cuda_fail(c0, e, "group capture end");
    cudaGraphExec_t ex = nullptr;
    e = cudaGraphInstantiate(&ex, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) return cuda_fail(c0, e, "group graph instantiation");
    it = g->graphs.emplace(key, std::make_pair(ex, kernels)).first;
  }
  cudaError_t e = cudaGraphLaunch(it->second.first, s);
  if (e != cudaSuccess) return cuda_fail(g->ctxs[0], e, "group graph launch");
  g->ctxs[0]->launches += it->second.second;
  return QPAT_OK;
}

qpat_status qpat_group_jvp(qpat_group* g, const int* batches, const double* const* mu, const double* const* phi0,
                           const double* const* dmu, unsigned illum, void* const* dP, void* stream) {
  if (!g || !batches || !mu || !dmu || !dP) return QPAT_EINVAL;
  const int n = (int)g->ctxs.size();
  std::vector<const void*> in(n, nullptr);
  for (int i = 0; i < n; ++i) {
    qpat_ctx* c = g->ctxs[i];
    c->stream = (cudaStream_t)stream;
    if (batches[i] == 0) continue;
    qpat_status st = check_batch(c, batches[i]);
    if (st != QPAT_OK) return st;
    st = jvp_heating(c, batches[i], mu[i], phi0 ? phi0[i] : nullptr, dmu[i], illum);
    if (st != QPAT_OK) return st;
    in[i] = c->tw_p0;
  }
  return qpat_group_propagate(g, 0, batches, in.data(), dP, stream);
}

qpat_status qpat_group_set_shape(qpat_group* g, const qpat_group_shape* shape) {
  if (!g || !shape || !shape_valid(*shape)) return QPAT_EINVAL;
  g->shape = *shape;
  return QPAT_OK;
}

qpat_status qpat_group_get_shape(const qpat_group* g, qpat_group_shape* shape, int* multi_ready,
                                 const int* batches) {
  if (!g || !shape) return QPAT_EINVAL;
  *shape = g->shape;
  if (multi_ready) *multi_ready = batches ? (int)!multi_members(g, batches).empty() : 0;
  return QPAT_OK;
}

qpat_status qpat_group_tune(qpat_group* g, const int* batches, int steps, void* stream, qpat_group_shape* best,
                            double* ms, int* ncand) {
  if (!g || !batches || steps < 2) return QPAT_EINVAL;
  const int n = (int)g->ctxs.size();
  qpat_ctx* c0 = g->ctxs[0];
  cudaStream_t s = (cudaStream_t)stream;
  for (int i = 0; i < n; ++i) {
    qpat_ctx* c = g->ctxs[i];
    if (batches[i] < 0 || batches[i] > c->maxb) return fail(c, QPAT_EINVAL, "group batch out of range");
    if (c->prof_phase >= 0) return fail(c, QPAT_EINVAL, "profiling is not available in group calls");
  }
  std::vector<qpat_group_shape> cand{{0, 144, 576, 1}};
  if (!multi_members(g, batches).empty())
    for (int rb : {144, 288})
      for (int cb : {288, 576})
        for (int lf : {1, 0}) cand.push_back({1, rb, cb, lf});
  // Tuning buffers: the kernels address the sensor series with each
  // context's full nt as the batch stride, so the series keep the full
  // [batch][nt][ns] shape while only the first `steps` samples are produced.
  struct Buf {
    std::vector<void*> p;
    ~Buf() {
      for (void* q : p) cudaFree(q);
    }
  } buf;
  std::vector<void*> in(n, nullptr), out(n, nullptr);
  std::vector<int> saved(n);
  for (int i = 0; i < n; ++i) {
    qpat_ctx* c = g->ctxs[i];
    saved[i] = c->nt;
    if (batches[i] == 0) continue;
    const size_t esz = c->prec == QPAT_FP32 ? 4 : 8;
    const size_t b_in = (size_t)batches[i] * c->N * esz, b_out = (size_t)batches[i] * c->nt * c->ns * esz;
    void *a = nullptr, *b = nullptr;
    if (cudaMalloc(&a, b_in) != cudaSuccess) return fail(c, QPAT_ENOMEM, "group tuning buffers");
    buf.p.push_back(a);
    if (cudaMalloc(&b, b_out) != cudaSuccess) return fail(c, QPAT_ENOMEM, "group tuning buffers");
    buf.p.push_back(b);
    QCK2(c, cudaMemsetAsync(a, 0, b_in, s));
    QCK2(c, cudaMemsetAsync(b, 0, b_out, s));
    in[i] = a;
    out[i] = b;
  }
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  QCK2(c0, cudaEventCreate(&e0));
  QCK2(c0, cudaEventCreate(&e1));
  const qpat_group_shape keep = g->shape;
  double best_ms = 1e300;
  int best_k = 0;
  qpat_status st = QPAT_OK;
  for (int i = 0; i < n; ++i) g->ctxs[i]->nt = std::max(2, std::min(steps, saved[i]));
  for (size_t k = 0; k < cand.size() && st == QPAT_OK; ++k) {
    g->shape = cand[k];
    const bool multi = cand[k].multi != 0;
    cudaGraphExec_t ex[2] = {nullptr, nullptr};
    for (int dir = 0; dir < 2 && st == QPAT_OK; ++dir) {
      cudaGraph_t graph = nullptr;
      cudaError_t e = cudaStreamBeginCapture(g->cap, cudaStreamCaptureModeThreadLocal);
      if (e == cudaSuccess) {
        seq_group(g, dir, batches, multi);
        e = cudaStreamEndCapture(g->cap, &graph);
      }
      if (e == cudaSuccess) e = cudaGraphInstantiate(&ex[dir], graph, 0);
      if (graph) cudaGraphDestroy(graph);
      if (e != cudaSuccess) st = cuda_fail(c0, e, "group tuning graph");
    }
    float t = 0.f;
    for (int rep = 0; rep < 2 && st == QPAT_OK; ++rep) {   // the first repetition warms up
      cudaEventRecord(e0, s);
      for (int dir = 0; dir < 2; ++dir) {
        for (int i = 0; i < n; ++i) {
          qpat_ctx* c = g->ctxs[i];
          c->stream = s;
          if (batches[i] == 0) continue;
          if (c->prec == QPAT_FP32) set_io_for<float>(c, dir, dir == 0 ? in[i] : out[i], dir == 0 ? out[i] : in[i], s);
          else set_io_for<double>(c, dir, dir == 0 ? in[i] : out[i], dir == 0 ? out[i] : in[i], s);
        }
        cudaGraphLaunch(ex[dir], s);
      }
      cudaEventRecord(e1, s);
      cudaError_t e = cudaEventSynchronize(e1);
      if (e != cudaSuccess) st = cuda_fail(c0, e, "group tuning run");
      else cudaEventElapsedTime(&t, e0, e1);
    }
    for (cudaGraphExec_t x : ex)
      if (x) cudaGraphExecDestroy(x);
    if (ms && k < 16) ms[k] = t;
    if (st == QPAT_OK && t < best_ms) {
      best_ms = t;
      best_k = (int)k;
    }
  }
  for (int i = 0; i < n; ++i) g->ctxs[i]->nt = saved[i];
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  g->shape = st == QPAT_OK ? cand[best_k] : keep;
  if (best) *best = g->shape;
  if (ncand) *ncand = (int)cand.size();
  return st;
}

qpat_status qpat_autotune(qpat_ctx* c, int batch, int steps, int* choice) {
  qpat_status st = check_batch(c, batch);
  if (st != QPAT_OK) return st;
  const int elt = c->prec == QPAT_FP32 ? 4 : 8;
  const bool rows_ok = c->dim == 2 && !c->cfg.generic_fft && fast_rows_supported(c->nx, elt);
  const bool cols_ok = c->dim == 2 && !c->cfg.generic_fft && fast_cols_supported(c->ny, elt);
  const int nt_saved = c->nt;
  const int nt_try = std::max(2, std::min(steps, nt_saved));
  const size_t esz = elt;
  // The kernels address the sensor series with the context's full nt as
  // the batch stride, so the tuning buffer has the full [batch][nt][ns]
  // shape even though only the first nt_try samples are produced.
  void *p0 = nullptr, *data = nullptr;
  const size_t data_bytes = (size_t)batch * nt_saved * c->ns * esz;
  QCK(cudaMalloc(&p0, (size_t)batch * c->N * esz));
  QCK(cudaMalloc(&data, data_bytes));
  QCK(cudaMemsetAsync(p0, 0, (size_t)batch * c->N * esz, c->stream));
  QCK(cudaMemsetAsync(data, 0, data_bytes, c->stream));
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  float best = 1e30f;
  int best_choice = 0;
  c->nt = nt_try;
  for (int cand = 0; cand < 4; ++cand) {
    const int fr = cand & 1, fc = (cand >> 1) & 1;
    if ((fr && !rows_ok) || (fc && !cols_ok)) continue;
    c->pf.fast_rows = c->pd.fast_rows = fr;
    c->pf.fast_cols = c->pd.fast_cols = fc;
    float total = 0.f;
    for (int rep = 0; rep < 2; ++rep) {   // first repetition warms up
      if (c->prec == QPAT_FP32) set_io_for<float>(c, 0, p0, data, c->stream);
      else set_io_for<double>(c, 0, p0, data, c->stream);
      cudaEventRecord(e0, c->stream);
      seq_any(c, 0, batch, c->stream);
      if (c->prec == QPAT_FP32) set_io_for<float>(c, 1, data, p0, c->stream);
      else set_io_for<double>(c, 1, data, p0, c->stream);
      seq_any(c, 1, batch, c->stream);
      cudaEventRecord(e1, c->stream);
      cudaEventSynchronize(e1);
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      if (rep == 1) total = ms;
    }
    if (total < best) { best = total; best_choice = cand; }
  }
  c->nt = nt_saved;
  c->pf.fast_rows = c->pd.fast_rows = best_choice & 1;
  c->pf.fast_cols = c->pd.fast_cols = (best_choice >> 1) & 1;
  for (auto& kv : c->graphs) cudaGraphExecDestroy(kv.second.first);
  c->graphs.clear();
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(p0);
  cudaFree(data);
  QCK(cudaGetLastError());
  if (choice) *choice = best_choice;
  return QPAT_OK;
}

qpat_status qpat_set_medium_checkpoints(qpat_ctx* c, int K) {
  if (!c || K < 0) return QPAT_EINVAL;
  c->medium_k = K;
  return QPAT_OK;
}

qpat_status qpat_get_stats(const qpat_ctx* c, long long out[3]) {
  if (!c || !out) return QPAT_EINVAL;
  out[0] = c->launches;
  out[1] = (long long)c->prof_used / 2;
  out[2] = c->last_pcg_iters;
  return QPAT_OK;
}

qpat_status qpat_profile(qpat_ctx* c, int phase) {
  if (!c) return QPAT_EINVAL;
  c->prof_phase = phase;
  c->prof_used = 0;
  return QPAT_OK;
}

qpat_status qpat_profile_read(qpat_ctx* c, double* total_ms, long long* count) {
  if (!c || !total_ms || !count) return QPAT_EINVAL;
  QCK(cudaStreamSynchronize(c->stream));
  double tot = 0.0;
  for (size_t k = 0; k + 1 < c->prof_used; k += 2) {
    float ms = 0.f;
    QCK(cudaEventElapsedTime(&ms, c->prof_events[k], c->prof_events[k + 1]));
    tot += ms;
  }
  *total_ms = tot;
  *count = (long long)c->prof_used / 2;
  c->prof_used = 0;
  return QPAT_OK;
}

}  // extern "C"
