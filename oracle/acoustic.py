"""FP64 oracle of the acoustic operator H_a and its adjoint H_a^*.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Follows Section 3.2 of the paper step by step, in its notation:

* staggered grid: v_i lives at r + dr_i/2 and t - dt/2, the acoustic
  density is split per axis rho_i (Section 3.2.1);
* medium diagonals c-bar, rho-bar, staggered rho-bar_i, tau-bar, eta-bar with
  tau = -2 alpha0 c^(y-1), eta = 2 alpha0 c^y tan(pi y / 2) (eq. Twelve);
* fractional Laplacians Y_abs = F^-1 k^(y-2) F, Y_dis = F^-1 k^(y-1) F and the
  k-space staggered gradient of eq. grr with kappa = sinc(c_ref k dt / 2);
* PML diagonals A_i = exp(-alpha_i dt / 2) (eq. dis-pml), applied twice per
  update, on a layer added outside the stated grid;
* additive source s1 split over n = -1, 0;
* the four-step loop num-vel, num-rho, num-p, num-m from n = -1 to Nt - 2.

The adjoint is the exact matrix transpose of that loop (the paper's
discretise-then-adjoint principle, Lemma 2 and eq. t1/t41): each
sub-operation of one step is transposed and the steps are run in reverse
order.  Arrays are C-ordered with x fastest: physical axis i (0 = x) is array
axis ``dim - 1 - i``.

Readings of points the paper leaves open:
sinc is the unnormalised sin(x)/x of |k|; c_ref = max(c); the PML profile is
alpha_max (c_ref/dx) (xi/P)^4 Np/s with xi the distance into the layer in
grid units (staggered points at half-integer xi); the Y_abs symbol is 0 at
k = 0; the smoothing operator S is the identity; the staggered ambient
density is the mean of the two neighbouring nodes (periodic); sensors are
bilinear / trilinear on the node grid.
"""
from __future__ import annotations

import dataclasses
import math
from typing import Callable, List, Optional

import numpy as np
import scipy.sparse as sp


def db_to_neper(alpha_db, y):
    """alpha0 in dB MHz^-y cm^-1 -> Np (rad/s)^-y m^-1.

    dB -> Np divides by 20 log10(e); cm^-1 -> m^-1 multiplies by 100; the
    MHz^-y frequency unit becomes (2 pi 1e6 rad/s)^-y."""
    return np.asarray(alpha_db, dtype=np.float64) * 100.0 / (20.0 * math.log10(math.e)) \
        / (2.0 * math.pi * 1e6) ** y


def absorption_coefficients(c, alpha_np, y):
    """eq. Twelve: tau = -2 alpha0 c^(y-1), eta = 2 alpha0 c^y tan(pi y/2)."""
    tau = -2.0 * alpha_np * c ** (y - 1.0)
    eta = 2.0 * alpha_np * c ** y * math.tan(math.pi * y / 2.0)
    return tau, eta


def max_supported_frequency(c_min, dx):
    """Highest frequency a k-space grid supports: two points per wavelength,
    f_max = c_min / (2 dx) (quoted for the paper's grids in Section 6)."""
    return c_min / (2.0 * dx)


def wavenumbers(n, dx):
    """Angular wavenumbers of an n-point DFT in FFT order.  For even n the
    Nyquist bin m = n/2 is taken as the negative frequency -pi/dx."""
    m = np.arange(n)
    m = np.where(m < n / 2.0, m, m - n)
    return 2.0 * math.pi * m / (n * dx)


def pml_profile(n, pml, dx, c_ref, dt, alpha_max=2.0, staggered=False):
    """Diagonal of A_i along one axis (eq. dis-pml), layer outside the interior.

    The absorption rises as the fourth power of the distance xi into the
    layer, reaching alpha_max nepers per grid point: alpha = alpha_max *
    (c_ref / dx) * (xi / P)^4.  Staggered points sit at j + 1/2."""
    s = np.arange(n, dtype=np.float64) + (0.5 if staggered else 0.0)
    if pml <= 0:
        return np.ones(n)
    lo, hi = float(pml), float(n - pml - 1)
    xi = np.where(s < lo, lo - s, np.where(s > hi, s - hi, 0.0))
    alpha = alpha_max * (c_ref / dx) * (xi / pml) ** 4
    return np.exp(-alpha * dt / 2.0)


def sensor_matrix(positions, shape, dx):
    """Sparse M (Ns x G): bilinear (2D) / trilinear (3D) interpolation of a
    node field at the sensor positions (eq. num-m, point detectors).

    Node j along physical axis i sits at (j - (N_i - 1)/2) dx."""
    positions = np.atleast_2d(np.asarray(positions, dtype=np.float64))
    dim = len(shape)
    ns = positions.shape[0]
    N = [shape[dim - 1 - i] for i in range(dim)]          # sizes per physical axis
    strides = [int(np.prod(shape[dim - i:])) if i > 0 else 1 for i in range(dim)]
    rows, cols, vals = [], [], []
    for s in range(ns):
        base, frac = [], []
        for i in range(dim):
            g = positions[s, i] / dx + (N[i] - 1) / 2.0
            j0 = int(math.floor(g))
            f = g - j0
            if j0 < 0 or j0 > N[i] - 1 or (j0 == N[i] - 1 and f > 0):
                raise ValueError(f"sensor {s} outside the grid")
            base.append(j0)
            frac.append(f)
        for corner in range(1 << dim):
            w = 1.0
            idx = 0
            for i in range(dim):
                b = (corner >> i) & 1
                w *= frac[i] if b else 1.0 - frac[i]
                idx += (base[i] + b) * strides[i]
            if w != 0.0:
                rows.append(s)
                cols.append(idx)
                vals.append(w)
    G = int(np.prod(shape))
    return sp.csr_matrix((vals, (rows, cols)), shape=(ns, G))


@dataclasses.dataclass
class Setup:
    """Everything the time loop needs, precomputed in FP64."""
    shape: tuple
    dim: int
    dx: float
    dt: float
    nt: int
    pml: int
    c_ref: float
    C: np.ndarray              # c-bar^2
    rho0: np.ndarray           # rho-bar at nodes
    rho0_stag: List[np.ndarray]  # rho-bar_i at r + dr_i/2
    tau: np.ndarray
    eta: np.ndarray
    lossless: bool
    A_node: List[np.ndarray]   # PML diagonal for rho_i (nodes)
    A_stag: List[np.ndarray]   # PML diagonal for v_i (staggered)
    D_plus: List[np.ndarray]   # symbols of d/dr_i^+ (eq. grr)
    D_minus: List[np.ndarray]  # symbols of d/dr_i^-
    Y_dis: np.ndarray          # symbol k^(y-1)
    Y_abs: np.ndarray          # symbol k^(y-2), 0 at k = 0
    M: sp.csr_matrix
    interior: tuple            # slices of the interior block

    def axis(self, i):
        """Array axis of physical axis i."""
        return self.dim - 1 - i


def make_setup(c, rho, alpha_db, y, dx, dt, nt, pml, sensor_pos, c_ref=None,
               pml_alpha=2.0, lossless=False):
    c = np.asarray(c, dtype=np.float64)
    rho = np.asarray(rho, dtype=np.float64)
    shape = c.shape
    dim = c.ndim
    if c_ref is None:
        c_ref = float(np.max(c))
    if lossless or alpha_db is None:
        lossless = True
        tau = np.zeros(shape)
        eta = np.zeros(shape)
    else:
        tau, eta = absorption_coefficients(c, db_to_neper(alpha_db, y), y)
    K = []
    for a in range(dim):
        k = wavenumbers(shape[a], dx)
        sh = [1] * dim
        sh[a] = shape[a]
        K.append(k.reshape(sh))
    kmag = np.sqrt(sum(k * k for k in K))
    kappa = np.sinc(c_ref * kmag * dt / 2.0 / math.pi)    # sin(x)/x with x = c_ref |k| dt / 2
    D_plus, D_minus, A_node, A_stag, rho_stag = [], [], [], [], []
    for i in range(dim):
        a = dim - 1 - i
        k = K[a]
        D_plus.append(1j * k * np.exp(1j * k * dx / 2.0) * kappa)
        D_minus.append(1j * k * np.exp(-1j * k * dx / 2.0) * kappa)
        sh = [1] * dim
        sh[a] = shape[a]
        A_node.append(np.broadcast_to(pml_profile(shape[a], pml, dx, c_ref, dt, pml_alpha, False).reshape(sh), shape))
        A_stag.append(np.broadcast_to(pml_profile(shape[a], pml, dx, c_ref, dt, pml_alpha, True).reshape(sh), shape))
        rho_stag.append(0.5 * (rho + np.roll(rho, -1, axis=a)))
    with np.errstate(divide="ignore", invalid="ignore"):
        Y_dis = np.where(kmag > 0, kmag ** (y - 1.0), 0.0) if not lossless else np.zeros(shape)
        Y_abs = np.where(kmag > 0, kmag ** (y - 2.0), 0.0) if not lossless else np.zeros(shape)
    interior = tuple(slice(pml, shape[a] - pml) for a in range(dim))
    M = sensor_matrix(sensor_pos, shape, dx)
    return Setup(shape=shape, dim=dim, dx=dx, dt=dt, nt=nt, pml=pml, c_ref=c_ref, C=c * c,
                 rho0=rho, rho0_stag=rho_stag, tau=tau, eta=eta, lossless=lossless,
                 A_node=A_node, A_stag=A_stag, D_plus=D_plus, D_minus=D_minus,
                 Y_dis=Y_dis, Y_abs=Y_abs, M=M, interior=interior)


def spectral(f, symbol):
    """F^-1 { symbol * F{f} } for a real field, real part kept."""
    return np.real(np.fft.ifftn(symbol * np.fft.fftn(f)))


def spectral_T(f, symbol):
    """Transpose of ``spectral(., symbol)`` as a real matrix: the conjugate symbol."""
    return np.real(np.fft.ifftn(np.conj(symbol) * np.fft.fftn(f)))


def embed(S: Setup, h):
    """Interior field -> full FFT grid, zero in the PML (p0 = 0 outside Omega)."""
    out = np.zeros(S.shape)
    out[S.interior] = h
    return out


def restrict(S: Setup, f):
    return np.array(f[S.interior])


def forward_full(S: Setup, P0, nt=None, callback: Optional[Callable] = None):
    """H_a on a full-grid P0: returns the sensor series P-hat, shape (Nt, Ns).

    Starts at n = -1 from zero fields and stops at n = Nt - 2; sample n + 1 is
    M p_(n+1) (eq. for_map_dis).  ``callback(n, v, rho, p)`` sees the state
    after each step (used by the invariant tests)."""
    nt = S.nt if nt is None else nt
    d, dt = S.dim, S.dt
    v = [np.zeros(S.shape) for _ in range(d)]
    rho = [np.zeros(S.shape) for _ in range(d)]
    p = np.zeros(S.shape)
    q = P0 / (2.0 * d * S.C)             # dt * s_i of eq. s1 (S = identity)
    data = np.zeros((nt, S.M.shape[0]))
    for n in range(-1, nt - 1):
        # 1. eq. num-vel
        for i in range(d):
            v[i] = S.A_stag[i] * (S.A_stag[i] * v[i] - dt / S.rho0_stag[i] * spectral(p, S.D_plus[i]))
        # 2. eq. num-rho, with the additive source at n = -1, 0
        div = []
        for i in range(d):
            di = spectral(v[i], S.D_minus[i])
            div.append(di)
            rho[i] = S.A_node[i] * (S.A_node[i] * rho[i] - dt * S.rho0 * di)
            if n in (-1, 0):
                rho[i] = rho[i] + q
        # 3. eq. num-p
        r = sum(rho)
        if S.lossless:
            p = S.C * r
        else:
            u = sum(S.A_node[i] * S.rho0 * div[i] for i in range(d))
            p = S.C * ((r - S.eta * spectral(r, S.Y_dis)) + S.tau * spectral(u, S.Y_abs))
        # 4. eq. num-m
        data[n + 1] = S.M @ p.ravel()
        if callback is not None:
            callback(n, v, rho, p)
    return data


def adjoint_full(S: Setup, W, nt=None):
    """H_a^* on a series W of shape (Nt, Ns): the exact transpose of
    ``forward_full``, returned on the full grid."""
    nt = S.nt if nt is None else nt
    d, dt = S.dim, S.dt
    vb = [np.zeros(S.shape) for _ in range(d)]
    rb = [np.zeros(S.shape) for _ in range(d)]
    pb = np.zeros(S.shape)
    qb = np.zeros(S.shape)
    MT = S.M.T.tocsr()
    for n in range(nt - 2, -2, -1):
        # transpose of step 4: the adjoint of p_(n+1) receives M^T W_(n+1)
        pb = pb + (MT @ W[n + 1]).reshape(S.shape)
        # transpose of step 3
        Cp = S.C * pb
        rtot = []
        if S.lossless:
            for i in range(d):
                rtot.append(rb[i] + Cp)
            ub = None
        else:
            # (I - eta Y_dis)^T C p-bar = C p-bar - Y_dis^T (eta C p-bar)
            rpart = Cp - spectral_T(S.eta * Cp, S.Y_dis)
            ub = spectral_T(S.tau * Cp, S.Y_abs)
            for i in range(d):
                rtot.append(rb[i] + rpart)
        # transpose of step 2 (and of the source injection)
        db = []
        for i in range(d):
            g = -dt * S.rho0 * S.A_node[i] * rtot[i]
            if ub is not None:
                g = g + S.rho0 * S.A_node[i] * ub
            db.append(g)
            rb[i] = S.A_node[i] * S.A_node[i] * rtot[i]
        if n in (-1, 0):
            qb = qb + sum(rtot)
        # transpose of step 1
        vtot = [vb[i] + spectral_T(db[i], S.D_minus[i]) for i in range(d)]
        pb = np.zeros(S.shape)
        for i in range(d):
            vb[i] = S.A_stag[i] * S.A_stag[i] * vtot[i]
            pb = pb - spectral_T(S.A_stag[i] * dt / S.rho0_stag[i] * vtot[i], S.D_plus[i])
    # q = P0 / (2 d C)  =>  P0-bar = q-bar / (2 d C)
    return qb / (2.0 * d * S.C)


def forward(S: Setup, p0_interior, nt=None):
    """H_a: interior initial pressure (N) -> sensor series (Nt, Ns)."""
    return forward_full(S, embed(S, p0_interior), nt)


def adjoint(S: Setup, W, nt=None):
    """H_a^*: sensor series (Nt, Ns) -> interior field (N)."""
    return restrict(S, adjoint_full(S, W, nt))


def setup_from_workload(w, nt=None, c_ref=None):
    """Build a Setup from a ``phantoms.Workload`` (medium, sensors, dt)."""
    import phantoms
    c, rho, alpha = phantoms.acoustic_medium(w)
    dt = phantoms.time_step(w, c)
    return make_setup(c, rho, None if w.lossless else alpha, w.y, w.dx, dt,
                      w.nt if nt is None else nt, w.pml, phantoms.sensor_positions(w),
                      c_ref=c_ref, lossless=w.lossless)
