"""FP64 oracle of the optical map (diffusion approximation) and its derivatives.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

The paper discretises eq. DA with P1 finite elements (Section 3.1).  The
workloads here put the optical unknowns on the acoustic interior grid, so
this oracle uses the cell-centred finite-volume analogue, written out term by
term:

* -div(kappa grad phi) + mu phi = 0 in Omega (eq. DA, first line): each
  interior face between cells a and b carries the flux
  kappa_f h^(d-2) (phi_a - phi_b) with the harmonic mean kappa_f;
  the absorption term is mu phi h^d (volume weight h^d);
* Robin condition phi + kappa/(2 gamma_d) d phi/dn = I/gamma_d (eq. DA, second
  line), gamma_2 = 1/pi, gamma_3 = 1/4: the outward flux density is
  2 gamma phi_b - 2 I at the boundary face value phi_b, which is eliminated
  through the half-cell gradient.  That adds 2 gamma kappa h^(d-1)/(gamma h +
  kappa) to the diagonal and 2 kappa I h^(d-1)/(gamma h + kappa) to the
  right-hand side for each boundary face of a cell;
* heating h = mu phi and p0 = Gamma h with Gamma = 1 (eq. h and the p0
  definition).

The derivative and adjoint in mu follow Lemma 1 restricted to delta kappa = 0:
A delta-Phi = -h^d (delta-mu o Phi0), delta-H = delta-mu o Phi0 + mu o delta-Phi
(eq. dh_des), and the adjoint A H~ = -h^d (mu o H), J_o^*(H) = Phi0 o (H + H~)
(mu row of eq. prodtproj with S_j = h^d and the node-to-element map equal
to the identity on a cell grid).  The solves use a sparse direct
factorisation from scipy.
"""
from __future__ import annotations

import math

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla


def gamma_d(dim):
    """Dimension factor of the Robin condition (Section 2.1)."""
    return 1.0 / math.pi if dim == 2 else 0.25


def _harmonic(a, b):
    return 2.0 * a * b / (a + b)


def boundary_current(shape, sides_mask):
    """I on every boundary face: a list over sides s = 2*i + (0 low, 1 high) of
    physical axis i, each an array over the face's cells (1 where the side's
    bit is set in ``sides_mask``, else 0)."""
    dim = len(shape)
    out = []
    for i in range(dim):
        a = dim - 1 - i
        face_shape = tuple(n for k, n in enumerate(shape) if k != a)
        for hi in (0, 1):
            s = 2 * i + hi
            out.append(np.full(face_shape, 1.0 if (sides_mask >> s) & 1 else 0.0))
    return out


def assemble(mu, kappa, h, currents, gamma=None):
    """Sparse system A Phi = G of the finite-volume DA (x fastest).

    ``currents``: per side s (see ``boundary_current``) an array of I values on
    that side's boundary faces."""
    mu = np.asarray(mu, dtype=np.float64)
    kappa = np.asarray(kappa, dtype=np.float64)
    shape = mu.shape
    dim = mu.ndim
    gam = gamma_d(dim) if gamma is None else gamma
    N = mu.size
    idx = np.arange(N).reshape(shape)
    diag = (mu * h ** dim).ravel().copy()
    rhs = np.zeros(N)
    rows, cols, vals = [], [], []
    for i in range(dim):
        a = dim - 1 - i
        lo = [slice(None)] * dim
        hi = [slice(None)] * dim
        lo[a] = slice(0, shape[a] - 1)
        hi[a] = slice(1, shape[a])
        ka, kb = kappa[tuple(lo)], kappa[tuple(hi)]
        t = (_harmonic(ka, kb) * h ** (dim - 2)).ravel()
        ia, ib = idx[tuple(lo)].ravel(), idx[tuple(hi)].ravel()
        np.add.at(diag, ia, t)
        np.add.at(diag, ib, t)
        rows += [ia, ib]
        cols += [ib, ia]
        vals += [-t, -t]
        for side in (0, 1):
            sl = [slice(None)] * dim
            sl[a] = 0 if side == 0 else shape[a] - 1
            kc = kappa[tuple(sl)]
            cells = idx[tuple(sl)].ravel()
            coef = (2.0 * gam * kc * h ** (dim - 1) / (gam * h + kc)).ravel()
            np.add.at(diag, cells, coef)
            I = np.asarray(currents[2 * i + side], dtype=np.float64)
            np.add.at(rhs, cells, (2.0 * kc * I * h ** (dim - 1) / (gam * h + kc)).ravel())
    rows.append(np.arange(N))
    cols.append(np.arange(N))
    vals.append(diag)
    A = sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                      shape=(N, N))
    return A, rhs


def solve(A, b):
    return spla.spsolve(A.tocsc(), b)


def fluence(mu, kappa, h, sides_mask):
    """Phi for illumination ``sides_mask`` (bit s: side s carries I = 1)."""
    A, b = assemble(mu, kappa, h, boundary_current(mu.shape, sides_mask))
    return solve(A, b).reshape(mu.shape)


def heating(mu, kappa, h, sides_mask):
    """H_o[mu] = mu o Phi (eq. forward_out with the identity node-to-element map)."""
    return mu * fluence(mu, kappa, h, sides_mask)


def jvp(mu, kappa, h, sides_mask, dmu, phi0=None):
    """J_o dmu = dmu o Phi0 + mu o dPhi, A dPhi = -h^d dmu o Phi0 (eq. dh_des)."""
    dim = mu.ndim
    A, b = assemble(mu, kappa, h, boundary_current(mu.shape, sides_mask))
    if phi0 is None:
        phi0 = solve(A, b).reshape(mu.shape)
    dphi = solve(A, -(h ** dim) * (dmu * phi0).ravel()).reshape(mu.shape)
    return dmu * phi0 + mu * dphi


def vjp(mu, kappa, h, sides_mask, hbar, phi0=None):
    """J_o^T hbar = Phi0 o (hbar + H~), A H~ = -h^d mu o hbar (eq. system_adjoint,
    prodtproj)."""
    dim = mu.ndim
    A, b = assemble(mu, kappa, h, boundary_current(mu.shape, sides_mask))
    if phi0 is None:
        phi0 = solve(A, b).reshape(mu.shape)
    ht = solve(A, -(h ** dim) * (mu * hbar).ravel()).reshape(mu.shape)
    return phi0 * (hbar + ht)


# ---- derivatives in kappa (Lemma 1, delta-kappa rows) -------------------------
def _dharmonic_da(a, b):
    """d/da of the harmonic mean 2ab/(a+b)."""
    return 2.0 * b * b / (a + b) ** 2


def kappa_source(mu, kappa, h, sides_mask, phi0, dkappa, gamma=None):
    """delta-b - delta-A Phi0 for the perturbation dkappa of the cell values
    of kappa: the right-hand side of A delta-Phi in the discrete counterpart of
    eq. dPhi.  Written out face by face like ``assemble``: an interior face
    between cells a, b carries t = kappa_f h^(d-2) with the harmonic mean
    kappa_f, so delta-t = h^(d-2) (d kappa_f/d kappa_a dkappa_a + d kappa_f /
    d kappa_b dkappa_b) and delta-A Phi0 gains delta-t (Phi_a - Phi_b) at a
    and the opposite at b; a boundary face of cell c adds
    2 gamma kappa_c h^(d-1)/(gamma h + kappa_c) to the diagonal and
    2 kappa_c I h^(d-1)/(gamma h + kappa_c) to the right-hand side, both
    differentiated in kappa_c."""
    mu = np.asarray(mu, dtype=np.float64)
    kappa = np.asarray(kappa, dtype=np.float64)
    shape = mu.shape
    dim = mu.ndim
    gam = gamma_d(dim) if gamma is None else gamma
    out = np.zeros(shape)
    currents = boundary_current(shape, sides_mask)
    for i in range(dim):
        a = dim - 1 - i
        lo = [slice(None)] * dim
        hi = [slice(None)] * dim
        lo[a] = slice(0, shape[a] - 1)
        hi[a] = slice(1, shape[a])
        lo, hi = tuple(lo), tuple(hi)
        ka, kb = kappa[lo], kappa[hi]
        dt = (_dharmonic_da(ka, kb) * dkappa[lo] + _dharmonic_da(kb, ka) * dkappa[hi]) * h ** (dim - 2)
        flux = dt * (phi0[lo] - phi0[hi])
        out[lo] -= flux
        out[hi] += flux
        for side in (0, 1):
            sl = [slice(None)] * dim
            sl[a] = 0 if side == 0 else shape[a] - 1
            sl = tuple(sl)
            kc = kappa[sl]
            q = gam * h / (gam * h + kc) ** 2 * h ** (dim - 1)    # d/dkappa of kappa h^(d-1)/(gamma h + kappa)
            I = np.asarray(currents[2 * i + side], dtype=np.float64)
            out[sl] += 2.0 * q * dkappa[sl] * (I - gam * phi0[sl])
    return out


def jvp_kappa(mu, kappa, h, sides_mask, dkappa, phi0=None):
    """J_o dkappa = mu o delta-Phi with A delta-Phi = delta-b - delta-A Phi0
    (Lemma 1, eqs. fr and dPhi, delta-mu = 0)."""
    A, b = assemble(mu, kappa, h, boundary_current(mu.shape, sides_mask))
    if phi0 is None:
        phi0 = solve(A, b).reshape(mu.shape)
    rhs = kappa_source(mu, kappa, h, sides_mask, phi0, np.asarray(dkappa, dtype=np.float64))
    return mu * solve(A, rhs.ravel()).reshape(mu.shape)


def vjp_kappa(mu, kappa, h, sides_mask, hbar, phi0=None):
    """J_o^T hbar in kappa: with psi = A^-1 (mu o hbar) (A is symmetric),
    <J_o dkappa, hbar> = <delta-b - delta-A Phi0, psi>, read off cell by cell
    (the discrete counterpart of the grad-phi0 . grad-h~ row of eq.
    opt_adjoint with its boundary term)."""
    mu = np.asarray(mu, dtype=np.float64)
    kappa = np.asarray(kappa, dtype=np.float64)
    shape = mu.shape
    dim = mu.ndim
    gam = gamma_d(dim)
    A, b = assemble(mu, kappa, h, boundary_current(shape, sides_mask))
    if phi0 is None:
        phi0 = solve(A, b).reshape(shape)
    psi = solve(A, (mu * hbar).ravel()).reshape(shape)
    g = np.zeros(shape)
    currents = boundary_current(shape, sides_mask)
    for i in range(dim):
        a = dim - 1 - i
        lo = [slice(None)] * dim
        hi = [slice(None)] * dim
        lo[a] = slice(0, shape[a] - 1)
        hi[a] = slice(1, shape[a])
        lo, hi = tuple(lo), tuple(hi)
        ka, kb = kappa[lo], kappa[hi]
        w = -(phi0[lo] - phi0[hi]) * (psi[lo] - psi[hi]) * h ** (dim - 2)
        g[lo] += _dharmonic_da(ka, kb) * w
        g[hi] += _dharmonic_da(kb, ka) * w
        for side in (0, 1):
            sl = [slice(None)] * dim
            sl[a] = 0 if side == 0 else shape[a] - 1
            sl = tuple(sl)
            kc = kappa[sl]
            q = gam * h / (gam * h + kc) ** 2 * h ** (dim - 1)
            I = np.asarray(currents[2 * i + side], dtype=np.float64)
            g[sl] += 2.0 * q * (I - gam * phi0[sl]) * psi[sl]
    return g
