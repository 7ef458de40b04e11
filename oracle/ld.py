"""FP64 oracle of the inexact-Newton lagged-diffusivity (LD) reconstruction.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

The unknown is the absorption mu on the interior grid with kappa fixed
(``Problem``), or both kappa and mu (``JointProblem``, the simultaneous
reconstruction of Section 6, using the kappa derivatives of ``optics``).
Written out from Sections 4 and 5:

* logarithmic scaling Xbar = log(mu / mu0) (eq. logscale), so that
  d mu / d Xbar = diag(mu);
* data misfit eps = 1/2 sum_q ||H_q[mu] - P_q||^2 (eq. varr);
* gradient  grad eps = sum_q diag(mu) J_q^* (H_q[mu] - P_q) (eq. gr);
* Gauss-Newton Hessian  H d = sum_q diag(mu) J_q^* J_q diag(mu) d (eq. apj);
* TV prior (eqs. tvm, dd, jm, m, m1): one row of D per interior face l
  between cells j1, j2 with entries +a, -a (a = the face length in 2D, the
  face area in 3D, here measured in mm as in Section 6), C = diag(((D Xbar)^2
  + beta)^(-1/2)), M[Xbar] = D^T C D, and M_gamma = M + gamma I;
* Algorithm 4 (PCG on the priorconditioned normal equation, eq. pre) with
  M_gamma^k = M_gamma[Xbar^k] lagged at the subproblem's start point, and its
  stopping rule (i_max; after i_m iterations the relative reduction of r^T z
  over the last i_m iterations against Tol_in);
* Algorithm 5 (outer loop, step alpha = 1, stop when the relative decrease of
  eps falls to Tol_out, or after k_max linearisations);
* Algorithm 6 (PD-IPM): per linearisation, sub-subproblems on the update d
  with a dual variable chi per face (eqs. du, dw, pre1 with lambda = 0) and
  the step length rule for chi (eq. sstep).

Library primitives: scipy's sparse direct solve for M_gamma z = r, and the
composite maps of ``oracle.qpat``.
"""
from __future__ import annotations

import dataclasses
from typing import Callable, List, Sequence

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import acoustic, optics


@dataclasses.dataclass
class LDParams:
    """Parameters of Algorithms 4 and 5 (Section 6 values for the 2D phantom
    as defaults: i_max = 30, i_m = 5, Tol_in = 0, gamma = 1e-6, beta = 2e-5,
    Tol_out = 1e-3)."""
    k_max: int = 10
    i_max: int = 30
    i_m: int = 5
    tol_in: float = 0.0
    tol_out: float = 1e-3
    gamma: float = 1e-6
    beta: float = 2e-5
    edge: float = 0.1          # a: face length (2D) / area (3D) of an interior face


# ---- TV prior ----------------------------------------------------------------
def tv_difference(shape, edge):
    """D: one row per interior face, +edge at the lower cell and -edge at the
    upper cell of the face (cells x fastest), faces of axis x first."""
    dim = len(shape)
    N = int(np.prod(shape))
    idx = np.arange(N).reshape(shape)
    rows, cols, vals = [], [], []
    r0 = 0
    for i in range(dim):
        a = dim - 1 - i
        lo = [slice(None)] * dim
        hi = [slice(None)] * dim
        lo[a] = slice(0, shape[a] - 1)
        hi[a] = slice(1, shape[a])
        ia, ib = idx[tuple(lo)].ravel(), idx[tuple(hi)].ravel()
        r = r0 + np.arange(ia.size)
        rows += [r, r]
        cols += [ia, ib]
        vals += [np.full(ia.size, edge), np.full(ia.size, -edge)]
        r0 += ia.size
    return sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))), shape=(r0, N))


def tv_functional(xbar, edge, beta):
    """J_beta[Xbar] = sum_l sqrt((D Xbar)_l^2 + beta): the smoothed TV whose
    gradient is M[Xbar] Xbar (eq. jm)."""
    D = tv_difference(xbar.shape, edge)
    g = D @ xbar.ravel()
    return float(np.sum(np.sqrt(g * g + beta)))


def tv_matrix(xbar, edge, beta):
    """M[Xbar] = D^T C[Xbar] D (eqs. m, m1)."""
    D = tv_difference(xbar.shape, edge)
    g = D @ xbar.ravel()
    C = sp.diags(1.0 / np.sqrt(g * g + beta))
    return (D.T @ C @ D).tocsr()


def m_gamma(xbar, edge, beta, gamma):
    M = tv_matrix(xbar, edge, beta)
    return (M + gamma * sp.identity(M.shape[0], format="csr")).tocsc()


# ---- data misfit, gradient and Gauss-Newton Hessian -----------------------------
class JointProblem:
    """The simultaneous reconstruction of kappa and mu (Sections 5 and 6):
    Xbar = [kappa-bar, mu-bar] (eq. scaling), each log-scaled against its
    initial guess (eq. logscale), so d X / d Xbar = diag(kappa, mu); J_q
    acts on both blocks (Lemma 1, eq. fr), and D is block diagonal (eq. dd)."""

    def __init__(self, S, illums: Sequence[int], P, mu0, kappa0):
        self.S = S
        self.illums = list(illums)
        self.P = [np.asarray(p, dtype=np.float64) for p in P]
        self.mu0 = np.asarray(mu0, dtype=np.float64)
        self.kappa0 = np.asarray(kappa0, dtype=np.float64)
        self.shape = (2,) + self.mu0.shape

    def coeffs(self, xbar):
        """(kappa, mu) at Xbar."""
        return self.kappa0 * np.exp(xbar[0]), self.mu0 * np.exp(xbar[1])

    def forward(self, kappa, mu, q):
        return acoustic.forward(self.S, optics.heating(mu, kappa, self.S.dx, self.illums[q]))

    def residuals(self, xbar):
        kappa, mu = self.coeffs(xbar)
        return [self.forward(kappa, mu, q) - self.P[q] for q in range(len(self.illums))]

    def misfit(self, xbar):
        return 0.5 * sum(float(np.sum(r * r)) for r in self.residuals(xbar))

    def _JT(self, kappa, mu, q, W):
        hbar = acoustic.adjoint(self.S, W)
        gk = optics.vjp_kappa(mu, kappa, self.S.dx, self.illums[q], hbar)
        gm = optics.vjp(mu, kappa, self.S.dx, self.illums[q], hbar)
        return np.stack([kappa * gk, mu * gm])

    def gradient(self, xbar, res=None):
        """eq. gr with d X / d Xbar = diag(kappa, mu)."""
        kappa, mu = self.coeffs(xbar)
        res = self.residuals(xbar) if res is None else res
        return sum(self._JT(kappa, mu, q, res[q]) for q in range(len(self.illums)))

    def gn_product(self, xbar, d):
        """eq. apj on both blocks."""
        kappa, mu = self.coeffs(xbar)
        out = np.zeros(self.shape)
        for q, m in enumerate(self.illums):
            dh = (optics.jvp_kappa(mu, kappa, self.S.dx, m, kappa * d[0])
                  + optics.jvp(mu, kappa, self.S.dx, m, mu * d[1]))
            out += self._JT(kappa, mu, q, acoustic.forward(self.S, dh))
        return out


class Problem:
    """Direct-QPAT misfit over illuminations ``illums`` (side masks) for the
    data ``P`` [nq][Nt][Ns], with the FP64 oracle maps."""

    def __init__(self, S, kappa, illums: Sequence[int], P, mu0):
        self.S, self.kappa = S, np.asarray(kappa, dtype=np.float64)
        self.illums = list(illums)
        self.P = [np.asarray(p, dtype=np.float64) for p in P]
        self.mu0 = np.asarray(mu0, dtype=np.float64)

    def mu(self, xbar):
        return self.mu0 * np.exp(xbar)

    def forward(self, mu, q):
        h = optics.heating(mu, self.kappa, self.S.dx, self.illums[q])
        return acoustic.forward(self.S, h)

    def J(self, mu, q, dmu):
        dh = optics.jvp(mu, self.kappa, self.S.dx, self.illums[q], dmu)
        return acoustic.forward(self.S, dh)

    def JT(self, mu, q, W):
        hbar = acoustic.adjoint(self.S, W)
        return optics.vjp(mu, self.kappa, self.S.dx, self.illums[q], hbar)

    def residuals(self, xbar):
        mu = self.mu(xbar)
        return [self.forward(mu, q) - self.P[q] for q in range(len(self.illums))]

    def misfit(self, xbar):
        """eps (eq. varr)."""
        return 0.5 * sum(float(np.sum(r * r)) for r in self.residuals(xbar))

    def gradient(self, xbar, res=None):
        """grad eps = sum_q diag(mu) J_q^* (H_q - P_q) (eq. gr)."""
        mu = self.mu(xbar)
        res = self.residuals(xbar) if res is None else res
        return sum(mu * self.JT(mu, q, res[q]) for q in range(len(self.illums)))

    def gn_product(self, xbar, d):
        """H d = sum_q diag(mu) J_q^* J_q diag(mu) d (eq. apj)."""
        mu = self.mu(xbar)
        return sum(mu * self.JT(mu, q, self.J(mu, q, mu * d)) for q in range(len(self.illums)))


# ---- Algorithm 4 ---------------------------------------------------------------
def pcg(apply_H: Callable, rhs, solve_M: Callable, i_max, i_m, tol_in):
    """Algorithm 4: PCG for H d = rhs preconditioned by M (solve_M(r) = M^-1 r),
    starting from d = 0.  Stops when i reaches i_max, or when i >= i_m and
    1 - (r_i^T z_i) / (r_{i-i_m}^T z_{i-i_m}) <= tol_in, or when r_i^T z_i = 0
    (the exact solution has been reached; the step would divide 0 by 0).
    Returns (d, i, the sequence r_i^T z_i)."""
    x = np.zeros_like(rhs)
    r = rhs.copy()
    z = solve_M(r)
    d = z.copy()
    rz = [float(r.ravel() @ z.ravel())]
    i = 0
    while i < i_max and rz[i] != 0.0 and (i < i_m or 1.0 - rz[i] / rz[i - i_m] > tol_in):
        Hd = apply_H(d)
        alpha = rz[i] / float(d.ravel() @ Hd.ravel())
        x = x + alpha * d
        r = r - alpha * Hd
        z = solve_M(r)
        rz.append(float(r.ravel() @ z.ravel()))
        beta = rz[i + 1] / rz[i]
        d = z + beta * d
        i += 1
    return x, i, rz


# ---- Algorithm 5 ---------------------------------------------------------------
def ld_newton(prob, prm: LDParams):
    """Algorithm 5: returns (mu*, Xbar*, eps history, inner iterations per
    outer iteration) for a ``Problem`` (mu only), or ((kappa*, mu*), Xbar*,
    ...) for a ``JointProblem``, where M_gamma acts block by block.  eps
    history holds eps^0, eps^1, ...: the misfit at each linearisation point,
    the last at the returned coefficients."""
    joint = isinstance(prob, JointProblem)
    shape = prob.shape if joint else prob.mu0.shape
    xbar = np.zeros(shape)
    eps_hist: List[float] = []
    inner: List[int] = []
    k = 0
    while True:
        res = prob.residuals(xbar)
        eps = 0.5 * sum(float(np.sum(r * r)) for r in res)
        eps_hist.append(eps)
        if k > 0 and not (1.0 - eps_hist[k] / eps_hist[k - 1] > prm.tol_out):
            break
        if k >= prm.k_max:
            break
        g = prob.gradient(xbar, res)
        if joint:
            lus = [spla.splu(m_gamma(xbar[b], prm.edge, prm.beta, prm.gamma)) for b in range(2)]
            n = xbar[0].size

            def solve_M(r):
                return np.concatenate([lus[0].solve(r[:n]), lus[1].solve(r[n:])])
        else:
            lu = spla.splu(m_gamma(xbar, prm.edge, prm.beta, prm.gamma))

            def solve_M(r):
                return lu.solve(r)
        d, i, _ = pcg(lambda v: prob.gn_product(xbar, v.reshape(shape)).ravel(), -g.ravel(),
                      solve_M, prm.i_max, prm.i_m, prm.tol_in)
        inner.append(i)
        xbar = xbar + d.reshape(shape)
        k += 1
    return (prob.coeffs(xbar) if joint else prob.mu(xbar)), xbar, eps_hist, inner


# ---- Algorithm 6: inexact Newton with the primal-dual interior-point TV ----------
@dataclasses.dataclass
class PDParams(LDParams):
    """Algorithm 6 parameters (Section 6, 2D phantom: k'_max = 20,
    Tol_med = 1e-3, beta = gamma = 1e-6; the PCG as in LD)."""
    kp_max: int = 20
    tol_med: float = 1e-3


def pd_weights(d, chi, edge, beta):
    """Per-face weights of M~ = D^T C (I - C chi (D d)^T) D (section
    PD-IPM, with the outer product read face by face: the factor for face l
    is c_l (1 - c_l chi_l (D d)_l), c_l = ((D d)_l^2 + beta)^(-1/2))."""
    D = tv_difference(d.shape, edge)
    g = D @ d.ravel()
    c = 1.0 / np.sqrt(g * g + beta)
    return D, g, c, c * (1.0 - c * chi * g)


def pd_matrix(d, chi, edge, beta, gamma):
    """M~_gamma = D^T diag(c (1 - c chi Dd)) D + gamma I."""
    D, g, c, wf = pd_weights(d, chi, edge, beta)
    M = (D.T @ sp.diags(wf) @ D).tocsr()
    return (M + gamma * sp.identity(M.shape[0], format="csr")).tocsc()


def pd_dual_step(d, dd, chi, edge, beta):
    """eq. dw face by face: dchi = c (1 - c chi Dd) D dd - chi + c D d (c at
    d), and the step length rule: s = min(1, phi*) with phi* the largest phi
    keeping |chi + phi dchi| <= 1 on every face.  Returns chi + s dchi."""
    D, g, c, wf = pd_weights(d, chi, edge, beta)
    dchi = wf * (D @ dd.ravel()) - chi + c * g
    phi = np.inf
    pos, neg = dchi > 0, dchi < 0
    if np.any(pos):
        phi = min(phi, float(np.min((1.0 - chi[pos]) / dchi[pos])))
    if np.any(neg):
        phi = min(phi, float(np.min((-1.0 - chi[neg]) / dchi[neg])))
    return chi + min(1.0, phi) * dchi


def pdipm_newton(prob, prm: PDParams):
    """Algorithm 6 for a ``Problem`` or a ``JointProblem`` (D, chi and M~
    block by block).  Returns (coefficients, Xbar*, eps history, PCG
    iterations of every sub-subproblem per outer iteration).

    Each sub-subproblem k' solves eq. pre1 by Algorithm 4 with
    grad eps~_k' = grad eps + H d_k' (the right-hand side of eq. du with
    lambda = 0), updates d (alpha_k' = 1) and chi (eq. dw with the step length
    rule).  r_k',* is the last r^T z of that PCG loop; the sub-subproblems stop
    at k'_max or when 1 - r_k',* / r_k'-1,* <= Tol_med."""
    joint = isinstance(prob, JointProblem)
    shape = prob.shape if joint else prob.mu0.shape
    blocks = 2 if joint else 1
    bshape = shape[1:] if joint else shape
    xbar = np.zeros(shape)
    eps_hist: List[float] = []
    inner: List[List[int]] = []
    k = 0
    while True:
        res = prob.residuals(xbar)
        eps_hist.append(0.5 * sum(float(np.sum(r * r)) for r in res))
        if k > 0 and not (1.0 - eps_hist[k] / eps_hist[k - 1] > prm.tol_out):
            break
        if k >= prm.k_max:
            break
        g = prob.gradient(xbar, res).ravel()

        def H(v):
            return prob.gn_product(xbar, v.reshape(shape)).ravel()

        n = int(np.prod(bshape))
        nf = tv_difference(bshape, prm.edge).shape[0]
        d = np.zeros(blocks * n)
        chi = [np.zeros(nf) for _ in range(blocks)]
        its, r_prev = [], None
        for kp in range(prm.kp_max):
            lus = [spla.splu(pd_matrix(d[b * n:(b + 1) * n].reshape(bshape), chi[b], prm.edge, prm.beta, prm.gamma))
                   for b in range(blocks)]

            def solve_M(r):
                return np.concatenate([lus[b].solve(r[b * n:(b + 1) * n]) for b in range(blocks)])

            dd, i, rz = pcg(H, -(g + H(d)), solve_M, prm.i_max, prm.i_m, prm.tol_in)
            its.append(i)
            for b in range(blocks):
                chi[b] = pd_dual_step(d[b * n:(b + 1) * n].reshape(bshape), dd[b * n:(b + 1) * n].reshape(bshape),
                                      chi[b], prm.edge, prm.beta)
            d = d + dd
            r_star = rz[-1]
            if r_prev is not None and not (1.0 - r_star / r_prev > prm.tol_med):
                break
            r_prev = r_star
        inner.append(its)
        xbar = xbar + d.reshape(shape)
        k += 1
    return (prob.coeffs(xbar) if joint else prob.mu(xbar)), xbar, eps_hist, inner
