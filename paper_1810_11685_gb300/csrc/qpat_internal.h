// Internal declarations shared by the library's translation units.
#pragma once
#include <cuda_runtime.h>
#include <string>
#include <vector>

#include "fft_smem.cuh"

struct qpat_ctx;

namespace qpat {

// Flags of one propagation kernel launch.
enum : int {
  kSkipInput = 1,    // the incoming spectral slots are zero (first step)
  kSource = 2,       // additive source active at this step (eq. s1, n = -1, 0)
  kAccWrite = 4,     // adjoint: write the source adjoint into p0_adj
  kAccAdd = 8,       // adjoint: add the source adjoint into p0_adj
  kSkipOutput = 16,  // no outgoing spectral slots needed (last step)
};

// Propagation phases.  F_*: forward step (Section 3.2.3), A_*: transposed
// step (Section 3.2.4).  R = row pass (x FFTs + pointwise), C = column pass
// (y FFTs + spectral operator).
enum Phase : int {
  F_R1 = 0,   // pressure from rho and the fractional-Laplacian terms (num-p)
  F_R2 = 1,   // velocity update (num-vel)
  F_R3 = 2,   // density update + source (num-rho); lossless: also pressure
  F_R3L = 3,
  F_C1 = 10,  // d/dr^+ of p, and sensor gather (num-m)
  F_C2 = 11,  // d/dr^- of v
  F_C3 = 12,  // Y_dis, Y_abs
  A_R1 = 20,  // adjoint of num-m and of the pressure update (lossy)
  A_R1L = 21, // same, lossless, fused with the transposed density update
  A_R3 = 22,  // transposed density update (+ source adjoint)
  A_R5 = 23,  // transposed velocity update
  A_C2 = 30,  // Y_dis^T, Y_abs^T
  A_C4 = 31,  // (d/dr^-)^T
  A_C6 = 32,  // -(d/dr^+)^T summed over axes
};

template <typename T>
struct IoPtrs {
  const T* p0;            // [B][N] interior source (forward)
  T* data;                // [B][nt][ns] (forward output)
  const T* w;             // [B][nt][ns] (adjoint input)
  T* p0adj;               // [B][N] (adjoint output)
  T* ckpt;                // forward-state checkpoints (optional)
};

template <typename T>
struct PropArgs {
  typedef typename V2<T>::t C;
  int nx, ny, nxh, pitch, pml, n0, n1, ns, nt;
  int cb;                 // columns per column-pass CTA
  FFTPlan px, py;
  const C* twx;
  const C* twy;
  // 1: the row (x) / column (y) passes run the length-specialised kernels
  int fast_rows, fast_cols;
  // medium diagonals on the full grid [ny][nx]
  const T* Cc;            // c^2
  const T* rho0;          // ambient density at nodes
  const T* dtrsx;         // dt / rho0 at (x + dx/2)
  const T* dtrsy;         // dt / rho0 at (y + dx/2)
  const T* tau;
  const T* eta;
  // PML diagonals A_i (per axis, nodes and staggered)
  const T* ax;
  const T* asx;
  const T* ay;
  const T* asy;
  T dt;
  // k-space symbols on the half spectrum [ny][nxh], each divided by nx*ny
  const T* kap;           // sinc(c_ref |k| dt / 2)
  const T* kp1;           // |k|^(y-1)
  const T* kp2;           // |k|^(y-2), 0 at k = 0
  const C* shxp;          // i kx exp(+i kx dx/2)  [nxh]
  const C* shxm;          // i kx exp(-i kx dx/2)  [nxh]
  const C* shyp;          // [ny]
  const C* shym;          // [ny]
  // sensors: gather form [ns][4], and scatter form (CSR over grid rows)
  const int* sidx;
  const T* sw;
  const int* rowptr;      // [ny + 1] range of grid points per row
  const int* pcol;        // [npts] column of each grid point
  const int* pent;        // [npts + 1] range of (sensor, weight) entries per point
  const int* esens;
  const T* ew;
  // workspace, batch strides in elements
  T* vx; T* vy; T* rx; T* ry;
  long long gstride;      // nx*ny
  C* spec;                // [B][2][ny][pitch]
  long long sstride;      // 2*ny*pitch
  T* pbuf;                // [B][ny][nx]
  // per call: the caller's buffers, read through a device-resident struct so
  // that a captured CUDA graph of the time loop serves every call
  const IoPtrs<T>* io;
  int n;                  // sample index this launch reads or writes
  int flags;
  int* err;               // device flags word (bit 0: non-finite; bit 1: a bounded wait gave up)
};

template <typename T>
void launch_row(const PropArgs<T>& a, int phase, int batch, cudaStream_t s);
template <typename T>
void launch_col(const PropArgs<T>& a, int phase, int batch, cudaStream_t s);
template <typename T>
void launch_gather(const PropArgs<T>& a, int batch, cudaStream_t s);
template <typename T>
void launch_set_io(IoPtrs<T>* dst, const T* p0, T* data, const T* w, T* p0adj, T* ckpt, cudaStream_t s);
// Elements (of T) of one forward-state checkpoint of one problem: v_x, v_y,
// rho_x, rho_y and the sampling buffer (5 grids) plus the two spectral slots.
template <typename T>
__host__ __device__ long long ckpt_elems(const PropArgs<T>& a);
// store (to_ckpt = 1) or restore the state of all problems at checkpoint m
template <typename T>
void launch_ckpt_copy(const PropArgs<T>& a, int batch, int m, int to_ckpt, cudaStream_t s);
// length-specialised passes (fast_kernels.cuh), one translation unit per length
template <typename T, int L>
void launch_row_fast_len(const PropArgs<T>& a, int ph, int batch, cudaStream_t s);
template <typename T, int L>
void launch_col_fast_len(const PropArgs<T>& a, int ph, int batch, cudaStream_t s);
template <typename T, int L>
void prepare_fast_len();
// Whether FFT extent L has length-specialised row / column passes for
// elements of elt bytes (4: FP32, 8: FP64).
bool fast_rows_supported(int L, int elt);
bool fast_cols_supported(int L, int elt);
template <typename T>
size_t row_smem_bytes(int nx);
template <typename T>
size_t col_smem_bytes(int ny, int cb);
template <typename T>
int prop_init_attributes(int nx, int ny, int fast_rows, int fast_cols);

// Table construction (tables.cu)
template <typename T>
struct TableOut {
  typedef typename V2<T>::t C;
  T *Cc, *rho0, *dtrsx, *dtrsy, *tau, *eta;
  T *ax, *asx, *ay, *asy;
  T *kap, *kp1, *kp2;
  C *shxp, *shxm, *shyp, *shym;
  C *twx, *twy;
};
template <typename T>
cudaError_t build_tables(const TableOut<T>& o, const double* d_c, const double* d_rho, const double* d_alpha_db,
                         int nx, int ny, int nxh, int pml, double dx, double dt, double c_ref, double pml_alpha,
                         double y, int lossless, cudaStream_t s);

// FP64 helpers (da.cu)
struct DAArgs {
  int n0, n1, n2, N, dim;  // n2 = 1 in 2D
  double h, gamma;
  double hd;               // h^dim, volume weight of the absorption term
  const double* diag0;     // face + Robin terms [N]
  const double* cxf;       // coefficient to the +x neighbour [N]
  const double* cyf;       // coefficient to the +y neighbour [N]
  const double* czf;       // coefficient to the +z neighbour [N] (3D)
  const double* bside;     // [2 dim][N] right-hand side of a unit current on each side
};
cudaError_t da_setup(DAArgs& a, double* d_diag0, double* d_cxf, double* d_cyf, double* d_czf, double* d_bside,
                     const double* d_kappa, cudaStream_t s);

// One level of the multigrid preconditioner: the finite-volume operator
// rediscretised at spacing 2^l h (A), the absorption averaged to the level,
// and work vectors, all [B][N_l].
struct MGLevel {
  DAArgs A;
  double *mu, *x, *x2, *b;
  double* kappa;           // the level's kappa (the fine level: the context's)
};
constexpr int kMaxLevels = 16;
struct MGHierarchy {
  int nlev = 0;            // 0: Jacobi preconditioner
  MGLevel lev[kMaxLevels];
  int coarse_sweeps = 41;  // sweeps on the coarsest level (two before and two
                           // after the coarse correction on the others)
  double omega = 0.8;      // Jacobi damping
};

struct PCGWork {
  double *x, *r, *z, *p, *q, *dinv, *b;   // [B][N]
  double *partial;                         // [B][kPartials][4]
  double *scal;                            // [B][8]
  double *hostscal;                        // pinned [B][8]
  MGHierarchy* mg;                         // null: Jacobi preconditioner
  double* mu;                              // [B][N] copy of the absorption of the current solve
  // CUDA graph of kPCGChunk iterations (fixed pointers: mu is staged in `mu`)
  bool use_graphs;
  cudaStream_t cap;
  cudaGraphExec_t chunk;
  int chunk_batch;
};
constexpr int kPCGChunk = 4;
// Build the coarse levels of `fine` (kappa on the fine grid) for up to
// max_batch problems; allocations go through `alloc` (owned by the caller).
typedef cudaError_t (*DevAlloc)(void* owner, void** p, size_t bytes);
cudaError_t mg_setup(MGHierarchy& h, const DAArgs& fine, const double* d_kappa, int max_batch, DevAlloc alloc,
                     void* owner, cudaStream_t s);
// Solve A(mu_b) x_b = rhs_b for a batch; x holds the result.  Returns the
// number of iterations used, or -1 if the cap was reached.
int pcg_solve(const DAArgs& a, const double* mu, int batch, const double* rhs, double* x, PCGWork& w,
              int max_iter, double tol, cudaStream_t s, cudaError_t* err);
cudaError_t da_rhs_from_sides(const DAArgs& a, unsigned mask, int batch, double* rhs, cudaStream_t s);
// Rebuild every coarse level's operator from the fine level's kappa, in the
// same buffers (captured graphs stay valid).
cudaError_t mg_rekappa(MGHierarchy& h, cudaStream_t s);
// delta-b - delta-A phi of the system for the kappa perturbation dkappa_b
// (illumination mask), [B][N] (Lemma 1, delta-kappa rows).
cudaError_t da_kappa_source(const DAArgs& a, const double* kappa, int batch, const double* phi, const double* dkappa,
                            unsigned mask, double* out, cudaStream_t s);
// Its transpose read against psi_b: the kappa gradient <delta-b - delta-A phi,
// psi> per cell, [B][N].
cudaError_t da_kappa_grad(const DAArgs& a, const double* kappa, int batch, const double* phi, const double* psi,
                          unsigned mask, double scale, double* out, cudaStream_t s);
// y += alpha x
cudaError_t da_axpy(long long n, double alpha, const double* x, double* y, cudaStream_t s);
// out_b = alpha * (u_b o v_b)   (all [B][N] FP64)
cudaError_t da_hadamard(int batch, int N, double alpha, const double* u, const double* v, double* out,
                        cudaStream_t s);
// dh = dmu o phi + mu o dphi, written in T
template <typename T>
cudaError_t da_heating_T(int batch, int N, const double* a1, const double* b1, const double* a2,
                         const double* b2, T* out, cudaStream_t s);
// g = phi o (hbar + ht) with hbar in T
template <typename T>
cudaError_t da_adjoint_out(int batch, int N, const double* phi, const T* hbar, const double* ht, double* g,
                           cudaStream_t s);
template <typename T>
cudaError_t T_to_double(long long n, const T* in, double* out, cudaStream_t s);
// out = -h^d * mu o T-valued hbar
template <typename T>
cudaError_t da_adjoint_rhs(int batch, int N, double scale, const double* mu, const T* hbar, double* out,
                           cudaStream_t s);
template <typename T>
cudaError_t dot_compensated(int batch, long long len, const T* a, const T* b, double* d_partial, double* d_out,
                            cudaStream_t s);
constexpr int kPartials = 256;

// What code outside api.cu needs to know about a context (the reconstruction
// loop in ld.cu is a client of the public entry points).
struct CtxView {
  int prec, dim, n0, n1, n2, nt, ns, maxb;
  long long N;
  double dx;
  cudaStream_t stream;
};
bool ctx_view(const struct ::qpat_ctx* c, CtxView* v);
// Record msg as the context's last error and return st.
int ctx_fail(struct ::qpat_ctx* c, int st, const char* msg);
// Optical halves of the composite maps for one problem (return qpat_status):
// optics_forward: phi = fluence of mu, h = mu o phi (prec [N]);
int optics_forward(struct ::qpat_ctx* c, const double* mu, unsigned illum, double* phi, void* h);
// dh = J_o (dmu, dkappa): either may be NULL (Lemma 1, eq. fr)
int optics_jvp2(struct ::qpat_ctx* c, const double* mu, const double* phi0, const double* dmu,
                const double* dkappa, unsigned illum, void* dh);
// g_mu, g_kappa = J_o^*(hbar) in mu and in kappa: either may be NULL (eq. opt_adjoint)
int optics_vjp2(struct ::qpat_ctx* c, const double* mu, const double* phi0, const void* hbar, unsigned illum,
                double* g_mu, double* g_kappa);
// CTAs per problem of the conjugate-gradient and multigrid kernels (eight per SM)
constexpr int kPCGBlocks = 1216;

}  // namespace qpat
