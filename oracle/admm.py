"""FP64 oracle of the gradient-based benchmark method: TV regularisation by
ADMM with L-BFGS search directions (Section 5.1 and Section 4.2).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Written out from the paper, in its notation:

* linear scaling Xbar = X / mean(X^0) per coefficient block (eq. linscale), so
  that d X / d Xbar = mean(X^0) per block;
* the augmented Lagrangian (eq. FAm)
      F_A(W, Xbar) = rho (1/2 ||D Xbar - W + U_w||^2 + nu ||W||_1)
                     + sum_q 1/2 ||H_q[X(Xbar)] - P_q + U_{p,q}||^2
  with D the TV difference operator of eq. dd (one row per interior face,
  +a / -a at its two cells), and its gradient in Xbar
      rho D^T (D Xbar - W + U_w) + sum_q dX/dXbar J_q^* (H_q - P_q + U_{p,q});
* Algorithm 3 (ADMM): W by the shrinkage formula of eq. thre, Xbar by the
  bound-constrained minimisation of F_A at fixed W (Algorithms 1 and 2), then
  the multiplier updates U_w += D Xbar - W and U_{p,q} += H_q - P_q, while
  ||grad_Xbar F_A|| > Tol_out;
* Algorithm 1 (L-BFGS two-loop recursion over the last m pairs s = Xbar_k -
  Xbar_{k-1}, y = grad_k - grad_{k-1}, rho_i = 1 / y_i^T s_i, initial inverse
  Hessian (s^T y / y^T y) I of the latest pair);
* the projection of eq. LBFGSsearch onto the box [Xbar_l, Xbar_u];
* Algorithm 2 (backtracking from alpha = 1 by the factor tau until the Wolfe
  conditions of eq. wo hold within the bounds of eq. cons).

Readings of points the paper leaves open (the same in the CUDA path):
* eq. LBFGSsearch prints "-Xbar_l" and "-Xbar_u" for the clipped cases; read
  as the direction that lands on the bound, d = Xbar_l - Xbar_k (resp.
  Xbar_u - Xbar_k) in that component, i.e. Xbar_k + d projected onto the box;
* the curvature condition of eq. wo carries a stray d_k: read as
  d^T grad F(Xbar + alpha d) >= c2 d^T grad F(Xbar);
* Algorithm 1 needs an initial inverse Hessian before any pair exists: the
  identity; pairs with y^T s <= 0 are not stored; a direction that is not
  one of descent after the projection is replaced by the projected -grad,
  and the history is cleared;
* Algorithm 2 has no iteration cap: at most ls_max trials; if none meets both
  Wolfe conditions, the largest trial step that met the sufficient-decrease
  condition is taken, and if none did, the inner minimisation stops;
* the inner minimisation (line al3l2) runs at most j_max L-BFGS iterations,
  stopping early when ||grad F_A|| <= tol_in; its history starts empty at
  every outer iteration (F_A changes with W and the multipliers);
* Algorithm 3 starts from Xbar^0 = X^0 / mean(X^0), W^0 = 0 and zero
  multipliers, and runs at most k_max outer iterations.
"""
from __future__ import annotations

import dataclasses
from typing import List, Sequence

import numpy as np

from . import acoustic, optics
from .ld import tv_difference


@dataclasses.dataclass
class ADMMParams:
    """Parameters of Algorithms 1-3 (Section 6: m = 5, c1 = 1e-4, c2 = 0.9,
    tau = 0.25, rho = 1, nu = 1e-3, Tol_out = 1e-2)."""
    k_max: int = 10
    j_max: int = 10
    m: int = 5
    c1: float = 1e-4
    c2: float = 0.9
    tau: float = 0.25
    ls_max: int = 20
    rho: float = 1.0
    nu: float = 1e-3
    tol_out: float = 1e-2
    tol_in: float = 0.0
    lower: float = 1e-3
    upper: float = 1e3
    edge: float = 0.1


def shrink(v, nu):
    """eq. thre: max(|v| - nu, 0) sgn(v), the minimiser of 1/2 (v - w)^2 + nu |w|."""
    return np.maximum(np.abs(v) - nu, 0.0) * np.sign(v)


def lbfgs_direction(g, S: List[np.ndarray], Y: List[np.ndarray]):
    """Algorithm 1: d = -H g from the pairs (S[i], Y[i]), oldest first."""
    q = g.copy()
    k = len(S)
    alpha = [0.0] * k
    rho = [1.0 / float(np.vdot(Y[i], S[i])) for i in range(k)]
    for i in range(k - 1, -1, -1):
        alpha[i] = rho[i] * float(np.vdot(S[i], q))
        q = q - alpha[i] * Y[i]
    h0 = float(np.vdot(S[-1], Y[-1])) / float(np.vdot(Y[-1], Y[-1])) if k else 1.0
    r = h0 * q
    for i in range(k):
        beta = rho[i] * float(np.vdot(Y[i], r))
        r = r + S[i] * (alpha[i] - beta)
    return -r


def project_direction(x, d, lower, upper):
    """eq. LBFGSsearch as read: the direction from x to the projection of x + d
    onto the box [lower, upper]."""
    return np.clip(x + d, lower, upper) - x


class Problem:
    """F_A for the joint unknown Xbar = [kappa-bar, mu-bar] (kappa0 given) or
    mu-bar alone (kappa0 None, kappa fixed at the setup's value)."""

    def __init__(self, S, kappa, illums: Sequence[int], P, mu0, kappa0=None, edge=0.1):
        self.S = S
        self.kappa = np.asarray(kappa, dtype=np.float64)
        self.illums = list(illums)
        self.P = [np.asarray(p, dtype=np.float64) for p in P]
        self.mu0 = np.asarray(mu0, dtype=np.float64)
        self.joint = kappa0 is not None
        self.kappa0 = None if kappa0 is None else np.asarray(kappa0, dtype=np.float64)
        self.scale = [float(np.mean(self.kappa0)), float(np.mean(self.mu0))] if self.joint else \
            [float(np.mean(self.mu0))]
        self.shape = ((2,) if self.joint else (1,)) + self.mu0.shape
        self.D = tv_difference(self.mu0.shape, edge)

    def x0(self):
        """Xbar^0 = X^0 / mean(X^0) per block (eq. linscale)."""
        blocks = [self.kappa0, self.mu0] if self.joint else [self.mu0]
        return np.stack([b / s for b, s in zip(blocks, self.scale)])

    def coeffs(self, xbar):
        """(kappa, mu) at Xbar."""
        if self.joint:
            return xbar[0] * self.scale[0], xbar[1] * self.scale[1]
        return self.kappa, xbar[0] * self.scale[0]

    def series(self, xbar):
        kappa, mu = self.coeffs(xbar)
        return [acoustic.forward(self.S, optics.heating(mu, kappa, self.S.dx, m)) for m in self.illums]

    def Dx(self, xbar):
        return np.stack([self.D @ b.ravel() for b in xbar])

    def DT(self, w):
        return np.stack([(self.D.T @ b).reshape(self.mu0.shape) for b in w])

    def value(self, xbar, W, Uw, Up, prm: ADMMParams, H=None):
        """F_A (eq. FAm)."""
        H = self.series(xbar) if H is None else H
        t = self.Dx(xbar) - W + Uw
        tv = prm.rho * (0.5 * float(np.sum(t * t)) + prm.nu * float(np.sum(np.abs(W))))
        return tv + 0.5 * sum(float(np.sum((h - p + u) ** 2)) for h, p, u in zip(H, self.P, Up))

    def gradient(self, xbar, W, Uw, Up, prm: ADMMParams, H=None):
        """grad_Xbar F_A: rho D^T (D Xbar - W + U_w) + sum_q dX/dXbar J_q^*(H_q - P_q + U_{p,q})."""
        H = self.series(xbar) if H is None else H
        kappa, mu = self.coeffs(xbar)
        g = prm.rho * self.DT(self.Dx(xbar) - W + Uw)
        for q, m in enumerate(self.illums):
            hbar = acoustic.adjoint(self.S, H[q] - self.P[q] + Up[q])
            gm = optics.vjp(mu, kappa, self.S.dx, m, hbar)
            if self.joint:
                gk = optics.vjp_kappa(mu, kappa, self.S.dx, m, hbar)
                g = g + np.stack([self.scale[0] * gk, self.scale[1] * gm])
            else:
                g = g + self.scale[0] * gm[None]
        return g


def line_search(f_and_g, x, f0, g0, d, prm: ADMMParams):
    """Algorithm 2: alpha = 1, 1 tau, 1 tau^2, ... until the Wolfe conditions
    (eq. wo, curvature as read) hold; x + alpha d stays in the box for every
    alpha in (0, 1] because x and x + d do.  Returns (alpha, f, g) or None."""
    gd = float(np.vdot(g0, d))
    alpha = 1.0
    armijo_only = None
    for _ in range(prm.ls_max):
        f, g = f_and_g(x + alpha * d)
        if f <= f0 + prm.c1 * alpha * gd:
            if float(np.vdot(g, d)) >= prm.c2 * gd:
                return alpha, f, g
            if armijo_only is None:
                armijo_only = (alpha, f, g)
        alpha *= prm.tau
    return armijo_only


def lbfgs_minimise(f_and_g, x, prm: ADMMParams):
    """Line al3l2 of Algorithm 3: at most j_max L-BFGS iterations (Algorithms
    1 and 2) on the box.  Returns (x, f, g, iterations)."""
    f, g = f_and_g(x)
    S: List[np.ndarray] = []
    Y: List[np.ndarray] = []
    it = 0
    while it < prm.j_max and float(np.linalg.norm(g)) > prm.tol_in:
        d = project_direction(x, lbfgs_direction(g, S, Y), prm.lower, prm.upper)
        if float(np.vdot(g, d)) >= 0.0:
            S.clear()
            Y.clear()
            d = project_direction(x, -g, prm.lower, prm.upper)
            if float(np.vdot(g, d)) >= 0.0:
                break
        step = line_search(f_and_g, x, f, g, d, prm)
        if step is None:
            break
        alpha, fn, gn = step
        s, y = alpha * d, gn - g
        if float(np.vdot(y, s)) > 0.0:
            S.append(s)
            Y.append(y)
            if len(S) > prm.m:
                S.pop(0)
                Y.pop(0)
        x, f, g = x + alpha * d, fn, gn
        it += 1
    return x, f, g, it


def admm(prob: Problem, prm: ADMMParams):
    """Algorithm 3.  Returns (Xbar, history dict: misfit eps per outer
    iteration, ||grad F_A||, inner iterations)."""
    x = prob.x0()
    W = np.zeros_like(prob.Dx(x))
    Uw = np.zeros_like(W)
    Up = [np.zeros_like(p) for p in prob.P]
    H = prob.series(x)
    hist = {"eps": [0.5 * sum(float(np.sum((h - p) ** 2)) for h, p in zip(H, prob.P))],
            "grad_norm": [float(np.linalg.norm(prob.gradient(x, W, Uw, Up, prm, H)))], "inner": []}
    k = 0
    while k < prm.k_max and hist["grad_norm"][-1] > prm.tol_out:
        W = shrink(prob.Dx(x) + Uw, prm.nu)

        def f_and_g(xx, W=W):
            Hx = prob.series(xx)
            return prob.value(xx, W, Uw, Up, prm, Hx), prob.gradient(xx, W, Uw, Up, prm, Hx)
        x, _, _, it = lbfgs_minimise(f_and_g, x, prm)
        H = prob.series(x)
        Uw = Uw + prob.Dx(x) - W
        Up = [u + h - p for u, h, p in zip(Up, H, prob.P)]
        hist["eps"].append(0.5 * sum(float(np.sum((h - p) ** 2)) for h, p in zip(H, prob.P)))
        hist["grad_norm"].append(float(np.linalg.norm(prob.gradient(x, W, Uw, Up, prm, H))))
        hist["inner"].append(it)
        k += 1
    return x, hist
