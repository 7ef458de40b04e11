"""FP64 oracle of the composite opto-acoustic maps.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

* forward  P-hat = H_a H_o[mu]                (eq. com_des)
* jvp      dP-hat = H_a J_o[mu] dmu           (eq. J_des)
* vjp      dmu-bar = J_o^*[mu] H_a^* (w)      (the adjoint map below J_des)

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
