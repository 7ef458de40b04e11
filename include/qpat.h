/*
 * qpat.h -- C ABI of the GB300 (sm_103a) direct-QPAT propagation library.
 *
 * The library evaluates the discretised opto-acoustic forward map of
 * Javaherian & Holman, "Direct quantitative photoacoustic tomography for
 * realistic acoustic media":
 *
 *   P-hat = H_a H_o[mu]                    (Section 3.2.2, eq. com_des)
 *   dP-hat = H_a J_o[mu] dmu               (eq. J_des)
 *   dmu-bar = J_o^*[mu] H_a^*(w)           (adjoint map below eq. J_des)
 *
 * where H_o is the diffusion-approximation optical map (Section 2.1, eq. DA;
 * heating h = mu phi, eq. h; p0 = Gamma h with Gamma = 1) and H_a is the
 * k-space pseudo-spectral acoustic map of Section 3.2.3 (eqs. num-vel,
 * num-rho, num-p, num-m with the additive source of eq. s1), whose adjoint is
 * the exact discrete transpose (Section 3.2.4, Lemma 2, eq. t41).
 *
 * Conventions (all entry points):
 *  - Grids are 2D, or 3D when qpat_config.n2 > 0.  Arrays are row-major with x
 *    fastest: a full-grid field is [ny][nx] ([nz][ny][nx] in 3D), an interior
 *    field is [n[1]][n[0]] ([n2][n[1]][n[0]]).  The FFT grid is the
 *    interior plus `pml` nodes on every side (the PML is added outside the
 *    stated grid, Section 3.2.2).  Node j along an axis of N nodes sits at
 *    x = (j - (N - 1)/2) * dx.
 *  - Time series are [nt][ns] (sample n = 0 .. nt-1, sensor fastest);
 *    batched buffers add a leading batch index.
 *  - "prec" buffers hold double for QPAT_FP64 contexts and float for
 *    QPAT_FP32 contexts.  Optical vectors (mu, dmu, gradients, fluence) are
 *    always double.
 *  - Every device pointer is caller-owned CUDA device memory of the current
 *    device.  Work is enqueued on the context's stream and the call returns
 *    without waiting, except where a call says it synchronises.  Host
 *    pointers are only read during the call.
 *  - Errors are returned as qpat_status; the context keeps a message
 *    (qpat_last_error).  No entry point aborts the process.
 */
#ifndef QPAT_H
#define QPAT_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct qpat_ctx qpat_ctx;

typedef enum {
  QPAT_OK = 0,
  QPAT_EINVAL = 1,      /* bad argument (sizes, pointers, ranges) */
  QPAT_EUNSTABLE = 2,   /* time step violates the stability check */
  QPAT_ENONFINITE = 3,  /* a NaN/Inf appeared in the fields */
  QPAT_ENOCONV = 4,     /* diffusion solve hit its iteration cap */
  QPAT_ETIMEOUT = 5,    /* a bounded device wait gave up: a grid barrier of a cooperative solve,
                           or the wait for the bulk copies of a propagation pass */
  QPAT_ENOMEM = 6,      /* device allocation failed */
  QPAT_ECUDA = 7        /* any other CUDA runtime error */
} qpat_status;

typedef enum { QPAT_FP64 = 0, QPAT_FP32 = 1 } qpat_precision;

/* Problem description.  Values <= 0 in the optional fields select defaults. */
typedef struct {
  int n[2];            /* interior nodes along x, y (the optical grid) */
  int pml;             /* PML nodes added on each side; nx = n[0] + 2 pml must be even */
  double dx;           /* grid spacing [m] (isotropic) */
  double dt;           /* time step [s] */
  int nt;              /* recorded samples per series (>= 2) */
  double c_ref;        /* k-space reference speed [m/s]; <= 0: max(c) */
  double pml_alpha;    /* PML strength [Np per grid point]; <= 0: 2 */
  double y;            /* absorption power-law exponent (1 < y < 3, y != 2) */
  int lossless;        /* 1: no absorption/dispersion (alpha0 ignored) */
  int max_batch;       /* largest batch any call will use; <= 0: 1 */
  double gamma_d;      /* Robin factor of eq. DA; <= 0: 1/pi */
  int pcg_max_iter;    /* diffusion-solve iteration cap; <= 0: 20000 */
  double pcg_tol;      /* relative residual target; <= 0: 1e-13 */
  int generic_fft;     /* 1: use the generic shared-memory FFT passes even where a
                          length-specialised pass exists for the extent */
  int no_graphs;       /* 1: launch every pass directly instead of replaying a
                          CUDA graph of the time loop captured on first use */
  int n2;              /* interior nodes along z: > 0 makes the problem 3D (grids
                          [nz][ny][nx], sensors [ns][3], six illumination sides
                          4: z low, 5: z high, gamma_d default 1/4) */
  int da_jacobi;       /* 1: precondition the diffusion solve's conjugate gradients
                          with the diagonal only; 0: with one geometric multigrid
                          V-cycle (damped-Jacobi smoothing on grids halved while
                          every extent is even), which needs far fewer iterations */
} qpat_config;

/* Medium, host memory, FP64, read during qpat_create only.
 * c, rho, alpha0_db: full FFT grid [ny][nx] (PML region included).
 * alpha0_db in dB MHz^-y cm^-1 (eq. Twelve uses it in Np (rad/s)^-y m^-1);
 * may be NULL when lossless.  kappa: optical diffusion [m] on the interior
 * grid [n1][n0] (fixed, not an unknown). */
typedef struct {
  const double* c;
  const double* rho;
  const double* alpha0_db;
  const double* kappa;
} qpat_medium;

/* Create a context on the current device.
 * sensor_xy: host [ns][2] sensor positions [m] (bilinear interpolation of the
 * node grid, eq. num-m).  stream: a cudaStream_t (NULL = legacy default).
 * Allocates and fills all device tables (FP64-computed k-space symbols, PML
 * diagonals, medium coefficients, FFT twiddles) and the workspace for
 * max_batch problems.  Synchronises the stream before returning.
 * Errors: EINVAL (sizes, odd grid, an FFT extent with a prime factor above 7,
 * sensors outside the grid, nt < 2), EUNSTABLE (c_max dt / dx above
 * 2 / (pi sqrt 2), the pseudo-spectral leapfrog limit, which the k-space
 * correction only relaxes), ENOMEM, ECUDA.  On error *out is NULL. */
qpat_status qpat_create(const qpat_config* cfg, const qpat_medium* med,
                        const double* sensor_xy, int ns, qpat_precision prec,
                        void* stream, qpat_ctx** out);

/* Free every device allocation of the context (synchronises its stream). */
qpat_status qpat_destroy(qpat_ctx* ctx);

/* Change the stream later calls enqueue on. */
qpat_status qpat_set_stream(qpat_ctx* ctx, void* stream);

/* Message describing the last error of this context ("" if none). */
const char* qpat_last_error(const qpat_ctx* ctx);

/* Sizes: out[0] = nx, out[1] = ny (FFT grid), out[2] = interior N,
 * out[3] = ns, out[4] = nt, out[5] = max_batch. */
qpat_status qpat_get_sizes(const qpat_ctx* ctx, long long out[6]);

/* Wait for the context's stream and report device-side failures found by
 * the kernels since the last check (ENONFINITE; ETIMEOUT when a pass's
 * bounded wait for its bulk copies gave up).  Clears the flags. */
qpat_status qpat_sync(qpat_ctx* ctx);

/* H_a (Section 3.2.3): batch of initial pressures -> sensor series.
 * p0:   device prec [batch][N] interior initial pressure (0 in the PML).
 * data: device prec [batch][nt][ns] output.  1 <= batch <= max_batch. */
qpat_status qpat_acoustic_forward(qpat_ctx* ctx, int batch, const void* p0, void* data);

/* H_a^* (Lemma 2, eq. t41, computed as the exact transpose of H_a).
 * data: device prec [batch][nt][ns]; p0_adj: device prec [batch][N] output. */
qpat_status qpat_acoustic_adjoint(qpat_ctx* ctx, int batch, const void* data, void* p0_adj);

/* Diffusion solve (eq. DA, finite-volume form): A(mu) phi = G(illum).
 * mu: device double [batch][N] absorption [1/m]; illum: bit s set = unit
 * inward current on side s (0: x low, 1: x high, 2: y low, 3: y high);
 * phi: device double [batch][N] output.  Synchronises (iteration control);
 * ENOCONV if the cap is reached before pcg_tol. */
qpat_status qpat_da_solve(qpat_ctx* ctx, int batch, const double* mu, unsigned illum,
                          double* phi);

/* Composite forward P-hat = H_a(mu o phi) (eq. com_des).
 * mu: device double [batch][N]; data: device prec [batch][nt][ns];
 * phi0_out: optional device double [batch][N] receiving the fluence. */
qpat_status qpat_forward(qpat_ctx* ctx, int batch, const double* mu, unsigned illum,
                         void* data, double* phi0_out);

/* Jacobian-vector product dP-hat = H_a(dmu o phi0 + mu o dphi),
 * A(mu) dphi = -h^2 dmu o phi0 (eq. dh_des, J_des).
 * phi0: optional device double [batch][N] fluence of mu (NULL: solved here).
 * dmu: device double [batch][N]; dP: device prec [batch][nt][ns]. */
qpat_status qpat_jvp(qpat_ctx* ctx, int batch, const double* mu, const double* phi0,
                     const double* dmu, unsigned illum, void* dP);

/* Vector-Jacobian product g = phi0 o (hbar + H~), hbar = H_a^*(w),
 * A(mu) H~ = -h^2 mu o hbar (Lemma 1 mu row; eqs. system_adjoint, prodtproj).
 * w: device prec [batch][nt][ns]; g: device double [batch][N] output. */
qpat_status qpat_vjp(qpat_ctx* ctx, int batch, const double* mu, const double* phi0,
                     const void* w, unsigned illum, double* g);

/* Derivatives in kappa (Lemma 1, delta-kappa rows), on the finite-volume
 * system: A(kappa, mu) phi = b(kappa) with harmonic-mean face coefficients and
 * Robin terms, differentiated face by face.
 * qpat_set_kappa: replace the context's kappa (device double [N], > 0; read
 *   during the call) and rebuild the diffusion operator and its multigrid
 *   levels in place.  Synchronises.
 * qpat_jvp_kappa: dP-hat = H_a(mu o dphi), A dphi = delta-b - delta-A phi0
 *   (eqs. fr, dPhi with delta-mu = 0); dkappa: device double [batch][N].
 * qpat_vjp_kappa: g = <delta-b - delta-A phi0, psi> per cell with
 *   A psi = mu o H_a^*(w) (the discrete counterpart of the grad phi0 . grad h~
 *   row of eq. opt_adjoint with its boundary term); g: device double
 *   [batch][N].  phi0 as in qpat_jvp (NULL: solved here). */
qpat_status qpat_set_kappa(qpat_ctx* ctx, const double* kappa);
qpat_status qpat_jvp_kappa(qpat_ctx* ctx, int batch, const double* mu, const double* phi0,
                           const double* dkappa, unsigned illum, void* dP);
qpat_status qpat_vjp_kappa(qpat_ctx* ctx, int batch, const double* mu, const double* phi0,
                           const void* w, unsigned illum, double* g);

/* Forward-state checkpointing of H_a.  The mu-gradient (qpat_vjp) needs no
 * forward fields -- the transposed step T^* of Section 3.2.4 does not depend
 * on the forward state -- so these calls serve callers that need the fields
 * themselves (e.g. derivatives in c or rho) and let tests confirm that a
 * forward resumed from any checkpoint reproduces the stored series exactly.
 * A checkpoint holds, per problem, v_x, v_y, rho_x, rho_y, the sampling
 * buffer and the two spectral work slots after loop iteration n with
 * (n + 1) % K == 0 (Section 3.2.3 loop), m = (n + 1)/K - 1, 0 <= m < (nt-1)/K.
 * qpat_ckpt_bytes: size of the checkpoint buffer for batch and K.
 * qpat_acoustic_forward_ckpt: H_a as qpat_acoustic_forward, also filling
 *   ckpt (device, caller-owned, qpat_ckpt_bytes bytes).
 * qpat_acoustic_resume: restore checkpoint m and continue the loop, writing
 *   samples (m + 1) K .. nt - 1 of data (other samples untouched). */
qpat_status qpat_ckpt_bytes(const qpat_ctx* ctx, int batch, int K, long long* bytes);
qpat_status qpat_acoustic_forward_ckpt(qpat_ctx* ctx, int batch, const void* p0, void* data, int K,
                                       void* ckpt);
qpat_status qpat_acoustic_resume(qpat_ctx* ctx, int batch, const void* ckpt, int K, int m, void* data);

/* Derivatives of H_a in the medium: the sound speed c and the ambient
 * density rho, both on the full FFT grid [ny][nx] (PML included), for one
 * problem.  The paper's Discussion names the sound speed as the next
 * unknown of a joint reconstruction; the derivative is taken of the
 * discretised map (as H_a^* is, Section 3.2.4): c enters through C = c^2 of
 * eq. num-p, tau and eta of eq. Twelve and the source of eq. s1; rho through
 * rho-bar at the nodes (eqs. num-rho, num-p) and at the staggered points
 * (eq. num-vel, the mean of two nodes).  c_ref and dt stay fixed.
 * Needs a 2D context (else EINVAL).  The sweeps run in the context's
 * precision; the directions, the weights, the outputs and the gradient sums
 * over the time steps are FP64 in both.  FP64 device buffers whatever the
 * context precision: p0 [n1][n0] interior initial pressure; dc, drho
 * [ny][nx] (either may be NULL: zero); dP and w [nt][ns]; g_c, g_rho
 * [ny][nx] (either may be NULL: not returned).  Workspace is allocated per
 * call: the tangent needs 27 real grid fields of the context precision, one
 * FP64 and 8 complex; the gradient up to 24 real of the context precision,
 * 7 to 9 FP64 and 8 complex, plus a tape of 5 (lossless) or 7 real grid
 * fields per stored time step.  The gradient keeps the tape of every step
 * while that history fits in 2 GiB; beyond, it stores the loop state (5 real grid fields) every K steps
 * during the forward sweep and recomputes each segment's tape from its
 * checkpoint before the segment's transposed steps (K tape slots; K near
 * sqrt(5 nt / fields), or as set by qpat_set_medium_checkpoints).  The
 * result is the same bit for bit for every K.  Both calls synchronise the
 * stream.
 * qpat_jvp_medium: dP = J_c dc + J_rho drho at p0.
 * qpat_vjp_medium: g_c = J_c^T w and g_rho = J_rho^T w at p0.
 * Errors: EINVAL, ENOMEM, ECUDA. */
qpat_status qpat_jvp_medium(qpat_ctx* ctx, const double* p0, const double* dc, const double* drho, double* dP);
qpat_status qpat_vjp_medium(qpat_ctx* ctx, const double* p0, const double* w, double* g_c, double* g_rho);
/* Checkpoint interval of qpat_vjp_medium on this context: K > 0 forces
 * checkpoints every K steps (K >= nt: the whole history), 0 restores the
 * automatic choice.  EINVAL for K < 0. */
qpat_status qpat_set_medium_checkpoints(qpat_ctx* ctx, int K);

/* Groups: propagate several contexts (e.g. uneven grids of one Newton
 * inner loop) concurrently in one CUDA graph, each context's time loop a
 * parallel branch.  Contexts must live on one device and outlive the group.
 * Group calls enqueue on `stream` and make it each member's stream.
 * qpat_group_propagate: dir 0 = H_a (in: p0, out: data), dir 1 = H_a^* (in:
 *   data, out: p0_adj), per member i with batches[i] problems (0 = skip);
 *   the graph is captured on the first call with a given batches tuple.
 * qpat_group_jvp: qpat_jvp for every member (diffusion solves per member,
 *   synchronising), then one graph launch for all acoustic forwards. */
typedef struct qpat_group qpat_group;
qpat_status qpat_group_create(int n, qpat_ctx* const* ctxs, qpat_group** out);
qpat_status qpat_group_destroy(qpat_group* group);
qpat_status qpat_group_propagate(qpat_group* group, int dir, const int* batches, const void* const* in,
                                 void* const* out, void* stream);
qpat_status qpat_group_jvp(qpat_group* group, const int* batches, const double* const* mu,
                           const double* const* phi0, const double* const* dmu, unsigned illum,
                           void* const* dP, void* stream);

/* Launch shape of group calls.
 * multi = 1: every pass kind of a time step runs as ONE launch for all
 *   members: its work list spans (member, problem, tile) items over the
 *   members' uneven grids, one item per CTA, running the same
 *   length-specialised pass bodies as the members' own launches (results are
 *   bit for bit the same).  The members' loops are aligned on the time index;
 *   a member drops out of the launches when its Nt ends.  Applies when every
 *   member with work is a 2D QPAT_FP32 context on a square grid of FFT extent
 *   288, 432 or 576 (each extent at most once), with the specialised passes
 *   selected (generic_fft = 0), all lossy or all lossless; otherwise the call
 *   falls back to multi = 0.
 * multi = 0: each member's own launch sequence is a parallel branch of one
 *   CUDA graph.
 * row_block: threads per row-pass CTA, 144 or 288 (row pairs per CTA:
 *   row_block / 48 at extent 288, row_block / 72 at 432 and 576).
 * col_block: threads per column-pass CTA, 288 or 576 (adjacent columns per
 *   CTA: col_block / 48 or col_block / 72).
 * largest_first: 1 hands the work items of the largest extent to the first
 *   CTAs.  Default {1, 144, 576, 1}. */
typedef struct {
  int multi;
  int row_block;
  int col_block;
  int largest_first;
} qpat_group_shape;

/* Set the shape of later group calls (EINVAL for values outside the lists). */
qpat_status qpat_group_set_shape(qpat_group* group, const qpat_group_shape* shape);

/* The present shape; *multi_ready (optional) = 1 when the members with work
 * in `batches` (per member, may be NULL) qualify for multi-problem launches. */
qpat_status qpat_group_get_shape(const qpat_group* group, qpat_group_shape* shape, int* multi_ready,
                                 const int* batches);

/* Autotuner of the group's launch shape: times a `steps`-step forward +
 * adjoint of batches[i] problems per member (a CUDA graph per direction,
 * second of two runs, CUDA events on `stream`) for multi = 0 and for every
 * multi-problem shape (row_block x col_block x largest_first) when the
 * members qualify, keeps the fastest as the group's shape and returns it in
 * *best.  ms (optional, up to 16 entries) receives each candidate's time in
 * candidate order (multi = 0 first, then row_block 144/288 x col_block
 * 288/576 x largest_first 1/0); *ncand (optional) their count.  The members'
 * loops are shortened to `steps` during the call.  Allocates and frees
 * temporary input and output buffers; synchronises. */
qpat_status qpat_group_tune(qpat_group* group, const int* batches, int steps, void* stream,
                            qpat_group_shape* best, double* ms, int* ncand);

/* Autotuner: time a `steps`-step forward + adjoint of `batch` problems with
 * every supported choice of pass kernels (specialised or generic row passes,
 * specialised or generic column passes) and keep the fastest for this
 * context; *choice = bit 0 rows specialised, bit 1 columns specialised.
 * Synchronises; allocates and frees temporary buffers. */
qpat_status qpat_autotune(qpat_ctx* ctx, int batch, int steps, int* choice);

/* FP64 inner products <a_b, c_b> of two device prec vectors [batch][len]
 * with compensated (Neumaier) accumulation; out: host double [batch].
 * Synchronises. */
qpat_status qpat_dot(qpat_ctx* ctx, int batch, long long len, const void* a, const void* b,
                     double* out);

/* Reconstruction of mu, or of kappa and mu together, by the inexact-Newton
 * lagged-diffusivity method with TV priorconditioning (Section 5.2.1,
 * Algorithms 4 and 5), by the inexact Newton method with the primal-dual
 * interior-point TV (Section 5.2.2, Algorithm 6: method = 1), or by the
 * gradient-based benchmark of Section 5.1 (method = 2, below).
 *  - Algorithm 3 (method 2): linear scaling Xbar = X / mean(X0) per block
 *    (eq. linscale); augmented Lagrangian F_A (eq. FAm) with the TV difference
 *    operator D of eq. dd; W by the shrinkage of eq. thre, then Xbar by at
 *    most j_max L-BFGS iterations (Algorithm 1, the last lbfgs_m pairs,
 *    initial inverse Hessian (s^T y / y^T y) I, the identity before any pair)
 *    with the direction projected onto the box [lower, upper] (eq.
 *    LBFGSsearch, read as landing on the bound) and a backtracking line
 *    search from alpha = 1 by tau (Algorithm 2) until both Wolfe conditions
 *    of eq. wo hold (the curvature condition read as d^T grad F(Xbar +
 *    alpha d) >= c2 d^T grad F(Xbar)); if none of ls_max trials meets both,
 *    the largest that met sufficient decrease, and if none did, the inner
 *    loop ends; then U_w += D Xbar - W and U_p,q += H_q - P_q.  Stops after
 *    k_max iterations or when ||grad F_A|| <= tol_out (< 0: 1e-2); the inner
 *    loop also stops when ||grad F_A|| <= tol_in.  Pairs with y^T s <= 0 are
 *    not kept; a projected direction that is not one of descent is replaced
 *    by the projected -grad and the history cleared.  eps_hist: the misfit
 *    after each ADMM iteration (eps^0 first); inner_hist: the L-BFGS
 *    iterations of each; info->inner_total their sum.
 *  - Algorithm 6 replaces the single PCG of a linearisation by sub-subproblems
 *    k' on the update d: Algorithm 4 on H dd = -(g + H d) with the
 *    preconditioner D^T C (I - C chi (D d)^T) D + gamma I (read face by face:
 *    face l weighs c_l (1 - c_l chi_l (D d)_l), c_l = ((D d)_l^2 + beta)^(-1/2)),
 *    d += dd, and the dual step of eq. dw per face with the step length rule
 *    (chi stays in [-1, 1]); they stop at kp_max or when the last r^T z of a
 *    PCG loop falls by no more than tol_med against the previous one.  Xbar += d.
 *    inner_hist then counts the PCG iterations of all sub-subproblems.
 *  - kappa == NULL: the unknown is mu, kappa stays the context's.  Otherwise
 *    the unknown is [kappa, mu] (eq. scaling): kappa is a device double [N],
 *    kappa0 on entry and the reconstruction on return; the derivatives in
 *    kappa are those of qpat_jvp_kappa / qpat_vjp_kappa, M_gamma and D are
 *    block diagonal (eq. dd), and the context's kappa is replaced
 *    (qpat_set_kappa) at every linearisation point, so it holds the
 *    reconstructed kappa on return.
 *  - Unknown Xbar = log(X / X0) per block (eq. logscale); misfit
 *    eps = 1/2 sum_q ||H_q[mu] - P_q||^2 over the illuminations q (eq. varr).
 *  - Outer iteration k (Algorithm 5): gradient g = sum_q mu o J_q^*(H_q - P_q)
 *    (eq. gr); M_gamma = D^T C D + gamma I frozen at Xbar^k (eqs. m, m1:
 *    D has +a/-a per interior face, C = ((D Xbar)^2 + beta)^(-1/2));
 *    Algorithm 4 (PCG, start 0) on H d = -g with H d = sum_q mu o J_q^* J_q
 *    (mu o d) (eq. apj) and preconditioner M_gamma; Xbar += d (alpha = 1).
 *    Stops when k = k_max or 1 - eps^k / eps^(k-1) <= tol_out.
 *  - M_gamma z = r is solved exactly along constants (M 1 = 0, so
 *    M_gamma 1 = gamma 1) and by conjugate gradients on the mean-free part
 *    (diagonal preconditioner, mean removed), to a relative residual tv_tol.
 * The acoustic halves of the nq illuminations run as one batch, so the
 * context's max_batch must be at least nq.
 * nq illuminations illum[q] (host, side masks as in qpat_da_solve); data:
 * device prec [nq][nt][ns] measured series P_q; mu: device double [N], mu0 on
 * entry (the initial guess, also the scale of Xbar), the reconstruction on
 * return.  eps_hist (host double [k_max + 1]) and inner_hist (host int
 * [k_max]) are optional: eps^0, eps^1, ... and the PCG iterations per outer
 * iteration.  info (optional) receives the counts below.
 * Allocates and frees its workspace (about (20 + nq) N doubles, 2 nq nt ns
 * and 2 nq N prec values, and the face weights); synchronises (the Krylov
 * scalars are read on the host every iteration).  mu0 must be positive (log scaling); this is
 * not checked.  Errors: EINVAL (nq < 1 or > max_batch, bad masks), ENOCONV
 * (a diffusion solve), ETIMEOUT (a grid-barrier wait of the cooperative
 * M_gamma solve gave up, see qpat_barrier_check), ENOMEM, ECUDA. */
typedef struct {
  int k_max;         /* outer linearisations; <= 0: 10 */
  int i_max;         /* PCG iterations per linearisation; <= 0: 30 */
  int i_m;           /* window of the inner stopping rule; <= 0: 5 */
  double tol_in;     /* Tol_in; < 0: 0 */
  double tol_out;    /* Tol_out; < 0: 1e-3 */
  double gamma;      /* <= 0: 1e-6 */
  double beta;       /* <= 0: 2e-5 */
  double tv_edge;    /* a: face length (2D) / area (3D) in the length unit of beta;
                        <= 0: dx in mm (2D), (dx in mm)^2 (3D) */
  int tv_max_iter;   /* CG iterations per M_gamma solve; <= 0: 20000 */
  double tv_tol;     /* relative residual of the M_gamma solve; <= 0: 1e-12 */
  int method;        /* 0: lagged diffusivity (Algorithm 5); 1: primal-dual interior point
                        (Algorithm 6); 2: the gradient-based benchmark, ADMM with L-BFGS
                        (Algorithms 1-3) */
  int kp_max;        /* Algorithm 6: sub-subproblems per linearisation; <= 0: 20 */
  double tol_med;    /* Algorithm 6: Tol_med, taken as given (Section 6: 1e-3) */
  /* method 2 (defaults: the values of Section 6) */
  int lbfgs_m;       /* (s, y) pairs kept by Algorithm 1; <= 0: 5 */
  int j_max;         /* L-BFGS iterations per ADMM iteration; <= 0: 10 */
  int ls_max;        /* trial steps of Algorithm 2; <= 0: 20 */
  double c1, c2;     /* Wolfe constants of eq. wo; <= 0: 1e-4, 0.9 */
  double tau;        /* backtracking factor; <= 0: 0.25 */
  double rho;        /* rho of eq. FAm; <= 0: 1 */
  double nu;         /* shrinkage threshold of eq. thre; <= 0: 1e-3 */
  double lower, upper;  /* box on Xbar (eq. cons); upper <= lower: [1e-3, 1e3] */
} qpat_ld_params;

typedef struct {
  int outer;              /* linearisations performed */
  int inner_total;        /* PCG iterations, all outer iterations */
  int sub_total;          /* Algorithm 6: sub-subproblems, all outer iterations */
  long long tv_iters;     /* CG iterations of all M_gamma solves */
  long long products;     /* applications of J_q or J_q^* (one propagation each) */
  double eps_first;       /* eps at mu0 */
  double eps_last;        /* eps at the returned mu */
  double seconds[3];      /* host wall time in the acoustic propagations, the optical
                             (diffusion) halves, and the M_gamma solves */
} qpat_ld_info;

qpat_status qpat_ld_solve(qpat_ctx* ctx, int nq, const unsigned* illum, const void* data, double* mu,
                          double* kappa, const qpat_ld_params* prm, qpat_ld_info* info, double* eps_hist,
                          int* inner_hist);

/* M_gamma u of the TV priorconditioner at Xbar (the operator qpat_ld_solve
 * builds; exposed for testing and for callers that run their own Krylov
 * loop).  xbar, u, out: device double [N].  Synchronises. */
qpat_status qpat_tv_apply(qpat_ctx* ctx, const double* xbar, double edge, double beta, double gamma,
                          const double* u, double* out);

/* Instrumentation (no counterpart in the paper).
 * qpat_get_stats: out[0] = propagation kernels launched by this context so
 * far, out[1] = launches currently held by the phase profiler, out[2] =
 * iterations of the last diffusion solve (-1: it hit the cap).
 * qpat_profile: from now on bracket every launch of pass `phase` (an
 * internal pass id, see paper_1810_11685_gb300/binding.py PHASES; -1 turns
 * profiling off) with CUDA events on the context's stream.
 * qpat_profile_read: synchronise, return the summed device time [ms] and the
 * number of profiled launches, and reset the profiler. */
qpat_status qpat_get_stats(const qpat_ctx* ctx, long long out[3]);
qpat_status qpat_profile(qpat_ctx* ctx, int phase);
qpat_status qpat_profile_read(qpat_ctx* ctx, double* total_ms, long long* count);

/* Check of the bounded grid barrier that cooperative launches of this library
 * use (the M_gamma solve of qpat_ld_solve): a cooperative grid of `blocks`
 * CTAs runs `rounds` rounds of barriers; the first `absent` CTAs return
 * before the first barrier, so with absent > 0 every wait of the others
 * gives up after limit_s seconds of device time (at most 10) and the call
 * returns QPAT_ETIMEOUT, the status a solver reports when a barrier wait
 * gives up; with absent = 0 it returns QPAT_OK once every round has let
 * exactly the whole grid through.  *status receives the same code.  blocks
 * must fit on the device at once (else EINVAL).  Allocates 32 bytes of
 * device memory; synchronises `stream`.  The paper has no counterpart: this
 * is instrumentation for the failure path. */
qpat_status qpat_barrier_check(int blocks, int rounds, int absent, double limit_s, void* stream, int* status);

/* Inner products <a_b, c_b> exactly as qpat_dot computes them, for callers
 * that may not allocate device memory where they call it (a frozen memory
 * pool, a host framework that owns all device allocations, an inner solver
 * loop where cudaMalloc would synchronise the device) and hold no context.
 * The paper has no counterpart: this is an interface convenience.
 * prec: QPAT_FP32 or QPAT_FP64 element type of a and b (device, [batch][len]);
 * out: device double [batch]; stream: cudaStream_t (NULL = legacy default).
 * a, b, out and stream must all belong to the current device: the scratch
 * address and the launch are those of the current device.
 * Allocates nothing: the scratch is a fixed 512 KiB device array inside the
 * library, so batch is limited to 1..64 (EINVAL beyond, message in
 * qpat_noalloc_last_error).  The first call on each device looks up that
 * array's address with the device current; make it before any stream
 * capture.  Calls share the array: overlapping calls race and must be
 * ordered by the caller.  Enqueue-only; returns without waiting. */
qpat_status qpat_dot_noalloc(int prec, int batch, long long len, const void* a, const void* b,
                             double* out, void* stream);
/* Message of the last failing qpat_dot_noalloc call on this host thread. */
const char* qpat_noalloc_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* QPAT_H */
