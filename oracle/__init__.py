"""FP64 CPU oracle for the direct-QPAT propagation path.

TEST INFRASTRUCTURE ONLY.  This package is a plain, slow, literal restatement
of the paper's discretisation (Javaherian & Holman, "Direct quantitative
photoacoustic tomography for realistic acoustic media"), used to check the
CUDA path.  Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline
leg of ``bench.py`` may import it.  The product path never calls it and it
shares no code with the CUDA kernels: the two meet only at the seeded input
generators in ``phantoms.py``.

Modules
- ``acoustic``: k-space PSTD forward operator H_a (Section 3.2.3, eqs.
  num-vel, num-rho, num-p, num-m with the additive source s1) and its exact
  discrete transpose H_a^* (Section 3.2.4, Lemma 2).
- ``optics``: finite-difference diffusion approximation (Section 2.1, eq. DA)
  with its Frechet derivative and adjoint in mu (Lemma 1).
- ``qpat``: the composite maps H = H_a H_o, J and J^* (Section 3.2.2,
  eqs. com_des and J_des).
- ``medium``: the derivatives of H_a in the sound speed and the density, the
  tangent loop and its exact transpose (the Discussion's next unknown).
- ``ld``: the inexact-Newton lagged-diffusivity reconstruction of mu with the
  TV priorconditioner (Section 5.2.1, Algorithms 4 and 5; Section 5, eqs. gr,
  apj, tvm, m, m1), and the primal-dual interior-point variant (Algorithm 6).
- ``admm``: the gradient-based benchmark, TV by ADMM with L-BFGS search
  directions and a Wolfe backtracking line search (Section 5.1, Algorithms
  1-3, eqs. FAm, thre, LBFGSsearch, wo, linscale).

Every function is pinned by tests in ``tests/test_oracle_*.py`` against
closed forms, invariants, brute force or the paper's printed values; none is
marked "parity unpinned".
"""
