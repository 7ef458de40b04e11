"""FP64 oracle of the composite opto-acoustic maps.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

* forward  P-hat = H_a H_o[mu]                (eq. com_des)
* jvp      dP-hat = H_a J_o[mu] dmu           (eq. J_des)
* vjp      dmu-bar = J_o^*[mu] H_a^* (w)      (the adjoint map below J_des)
* jvp_kappa, vjp_kappa: the same in kappa (Lemma 1, delta-kappa rows)

with Gamma = 1 so p0 = h on the interior grid and 0 in the PML.
"""
from __future__ import annotations

from . import acoustic, optics


def forward(S, mu, kappa, sides_mask):
    h = optics.heating(mu, kappa, S.dx, sides_mask)
    return acoustic.forward(S, h)


def jvp(S, mu, kappa, sides_mask, dmu):
    dh = optics.jvp(mu, kappa, S.dx, sides_mask, dmu)
    return acoustic.forward(S, dh)


def vjp(S, mu, kappa, sides_mask, W):
    hbar = acoustic.adjoint(S, W)
    return optics.vjp(mu, kappa, S.dx, sides_mask, hbar)


def jvp_kappa(S, mu, kappa, sides_mask, dkappa):
    """dP-hat = H_a J_o dkappa (Lemma 1, delta-kappa rows)."""
    return acoustic.forward(S, optics.jvp_kappa(mu, kappa, S.dx, sides_mask, dkappa))


def vjp_kappa(S, mu, kappa, sides_mask, W):
    """dkappa-bar = J_o^* H_a^*(w) in kappa."""
    return optics.vjp_kappa(mu, kappa, S.dx, sides_mask, acoustic.adjoint(S, W))
