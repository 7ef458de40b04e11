"""FP64 oracle of the derivatives of the acoustic data in the medium: the
sound speed c and the ambient density rho.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

The paper's Discussion names a joint reconstruction of the optical
coefficients and the sound speed as the next step; its Jacobian needs the
derivative of H_a in c (and rho).  As for H_a^* (Section 3.2.4, Lemma 2) the
derivative is taken of the discretised map itself, step by step through the
loop of ``acoustic.forward_full`` (eqs. num-vel, num-rho, num-p, num-m with
the source s1):

* c enters through C = c^2 in num-p, through tau = -2 alpha0 c^(y-1) and
  eta = 2 alpha0 c^y tan(pi y / 2) (eq. Twelve), and through the source
  dt s_i = P0 / (2 d C) of s1;
* rho enters through rho-bar at the nodes (num-rho and the absorption term of
  num-p) and through the staggered rho-bar_i (num-vel), the mean of the two
  neighbouring nodes.

Readings: c_ref (the k-space correction and the PML scale) and dt are held
fixed: they are parameters of the discretisation, and c_ref = max(c) is not
differentiable.  Both derivatives are taken on the full FFT grid, PML
included, since the medium extends into the layer.

* ``jvp_medium``: the tangent-linear loop, dP-hat = J_c dc + J_rho drho.
* ``vjp_medium``: its exact transpose, run backwards over the stored forward
  states (every step is kept: this oracle is for small grids).
"""
from __future__ import annotations

import numpy as np

from .acoustic import Setup, spectral, spectral_T


def _coefficient_slopes(S: Setup, y):
    """d tau / dc and d eta / dc from eq. Twelve: tau ~ c^(y-1), eta ~ c^y."""
    c = np.sqrt(S.C)
    return c, (y - 1.0) * S.tau / c, y * S.eta / c


def _stag(S: Setup, f, i):
    """Mean of the two nodes around the staggered point r + dr_i / 2."""
    a = S.axis(i)
    return 0.5 * (f + np.roll(f, -1, axis=a))


def _stag_T(S: Setup, g, i):
    """Transpose of ``_stag``."""
    a = S.axis(i)
    return 0.5 * (g + np.roll(g, 1, axis=a))


def jvp_medium(S: Setup, y, P0, dc, drho, nt=None):
    """Derivative of ``acoustic.forward_full(S, P0)`` along (dc, drho), both
    full-grid fields; returns the sensor series (Nt, Ns)."""
    nt = S.nt if nt is None else nt
    d, dt = S.dim, S.dt
    c, dtau_dc, deta_dc = _coefficient_slopes(S, y)
    dC = 2.0 * c * dc
    dtau, deta = dtau_dc * dc, deta_dc * dc
    drs = [_stag(S, drho, i) for i in range(d)]
    v = [np.zeros(S.shape) for _ in range(d)]
    rho = [np.zeros(S.shape) for _ in range(d)]
    dv = [np.zeros(S.shape) for _ in range(d)]
    drh = [np.zeros(S.shape) for _ in range(d)]
    p = np.zeros(S.shape)
    dp = np.zeros(S.shape)
    q = P0 / (2.0 * d * S.C)
    dq = -q * dC / S.C
    out = np.zeros((nt, S.M.shape[0]))
    for n in range(-1, nt - 1):
        # num-vel: v_i = A (A v_i - dt / rho_i grad_i p)
        for i in range(d):
            g, dg = spectral(p, S.D_plus[i]), spectral(dp, S.D_plus[i])
            rs = S.rho0_stag[i]
            v[i] = S.A_stag[i] * (S.A_stag[i] * v[i] - dt / rs * g)
            dv[i] = S.A_stag[i] * (S.A_stag[i] * dv[i] - dt / rs * dg + dt * drs[i] / (rs * rs) * g)
        # num-rho: rho_i = A (A rho_i - dt rho div_i) + dt s_i
        div, ddiv = [], []
        for i in range(d):
            di, ddi = spectral(v[i], S.D_minus[i]), spectral(dv[i], S.D_minus[i])
            div.append(di)
            ddiv.append(ddi)
            rho[i] = S.A_node[i] * (S.A_node[i] * rho[i] - dt * S.rho0 * di)
            drh[i] = S.A_node[i] * (S.A_node[i] * drh[i] - dt * (drho * di + S.rho0 * ddi))
            if n in (-1, 0):
                rho[i] = rho[i] + q
                drh[i] = drh[i] + dq
        # num-p: p = C X with X = sum rho (lossless) or the absorbing form
        r, dr = sum(rho), sum(drh)
        if S.lossless:
            X, dX = r, dr
        else:
            u = sum(S.A_node[i] * S.rho0 * div[i] for i in range(d))
            du = sum(S.A_node[i] * (drho * div[i] + S.rho0 * ddiv[i]) for i in range(d))
            Yr, Yu = spectral(r, S.Y_dis), spectral(u, S.Y_abs)
            X = r - S.eta * Yr + S.tau * Yu
            dX = dr - deta * Yr - S.eta * spectral(dr, S.Y_dis) + dtau * Yu + S.tau * spectral(du, S.Y_abs)
        p = S.C * X
        dp = dC * X + S.C * dX
        # num-m
        out[n + 1] = S.M @ dp.ravel()
    return out


def vjp_medium(S: Setup, y, P0, W, nt=None):
    """Transpose of ``jvp_medium``: the gradients (g_c, g_rho) on the full
    grid of <W, forward_full(S, P0)> in c and rho."""
    nt = S.nt if nt is None else nt
    d, dt = S.dim, S.dt
    # forward pass, keeping what each step's derivative needs
    v = [np.zeros(S.shape) for _ in range(d)]
    rho = [np.zeros(S.shape) for _ in range(d)]
    p = np.zeros(S.shape)
    q = P0 / (2.0 * d * S.C)
    tape = {}
    for n in range(-1, nt - 1):
        p_in = p
        for i in range(d):
            v[i] = S.A_stag[i] * (S.A_stag[i] * v[i] - dt / S.rho0_stag[i] * spectral(p, S.D_plus[i]))
        div = [spectral(v[i], S.D_minus[i]) for i in range(d)]
        for i in range(d):
            rho[i] = S.A_node[i] * (S.A_node[i] * rho[i] - dt * S.rho0 * div[i])
            if n in (-1, 0):
                rho[i] = rho[i] + q
        r = sum(rho)
        if S.lossless:
            X, Yr, Yu = r, None, None
        else:
            u = sum(S.A_node[i] * S.rho0 * div[i] for i in range(d))
            Yr, Yu = spectral(r, S.Y_dis), spectral(u, S.Y_abs)
            X = r - S.eta * Yr + S.tau * Yu
        p = S.C * X
        tape[n] = (p_in, div, X, Yr, Yu)

    # reverse sweep: the adjoint of acoustic.adjoint_full plus the medium terms
    gC, gtau, geta, grho = (np.zeros(S.shape) for _ in range(4))
    grs = [np.zeros(S.shape) for _ in range(d)]
    vb = [np.zeros(S.shape) for _ in range(d)]
    rb = [np.zeros(S.shape) for _ in range(d)]
    pb = np.zeros(S.shape)
    qb = np.zeros(S.shape)
    MT = S.M.T.tocsr()
    for n in range(nt - 2, -2, -1):
        p_in, div, X, Yr, Yu = tape.pop(n)
        pb = pb + (MT @ W[n + 1]).reshape(S.shape)
        # num-p
        gC += pb * X
        Cp = S.C * pb
        if S.lossless:
            rpart, ub = Cp, None
        else:
            geta -= Cp * Yr
            gtau += Cp * Yu
            rpart = Cp - spectral_T(S.eta * Cp, S.Y_dis)
            ub = spectral_T(S.tau * Cp, S.Y_abs)
        rtot = [rb[i] + rpart for i in range(d)]
        # num-rho (and the absorption term's u = sum A rho div)
        db = []
        for i in range(d):
            g = -dt * S.rho0 * S.A_node[i] * rtot[i]
            grho -= dt * S.A_node[i] * div[i] * rtot[i]
            if ub is not None:
                g = g + S.rho0 * S.A_node[i] * ub
                grho += S.A_node[i] * div[i] * ub
            db.append(g)
            rb[i] = S.A_node[i] * S.A_node[i] * rtot[i]
        if n in (-1, 0):
            qb = qb + sum(rtot)
        # num-vel
        vtot = [vb[i] + spectral_T(db[i], S.D_minus[i]) for i in range(d)]
        pb = np.zeros(S.shape)
        for i in range(d):
            rs = S.rho0_stag[i]
            grs[i] += vtot[i] * S.A_stag[i] * dt / (rs * rs) * spectral(p_in, S.D_plus[i])
            vb[i] = S.A_stag[i] * S.A_stag[i] * vtot[i]
            pb = pb - spectral_T(S.A_stag[i] * dt / rs * vtot[i], S.D_plus[i])
    # source s1: q = P0 / (2 d C)  =>  dq / dC = -q / C
    gC -= qb * q / S.C
    c, dtau_dc, deta_dc = _coefficient_slopes(S, y)
    g_c = 2.0 * c * gC + dtau_dc * gtau + deta_dc * geta
    for i in range(d):
        grho += _stag_T(S, grs[i], i)
    return g_c, grho
