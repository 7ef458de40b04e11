"""Uneven-grid batches in one CUDA graph (qpat_group_*) and the autotuner:
group results equal the members' individual calls bit for bit, and the
members match the oracle; the c4 grid sizes (288^2, 432^2, 576^2 FFT grids)
run together and match the oracle over their first steps."""
import numpy as np
import pytest

import phantoms
from oracle import acoustic, qpat
from gpu_helpers import make_pair, rel_l2, to_gpu, to_np

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def members():
    return [phantoms.small(n=24, pml=8, nt=30, n_sensors=8, seed=1),     # 40
            phantoms.small(n=40, pml=8, nt=44, n_sensors=10, seed=2),    # 56
            phantoms.small(n=48, pml=8, nt=36, n_sensors=12, seed=3)]    # 64 (generic passes)


def test_group_equals_individual_calls():
    from paper_1810_11685_gb300.binding import Group
    ws = members()
    pairs = [make_pair(w, "fp32", max_batch=3) for w in ws]
    ctxs = [p[0] for p in pairs]
    g = Group(ctxs)
    p0s = [torch.stack([to_gpu(phantoms.smooth_p0(w, s), torch.float32) for s in range(b)])
           for w, b in zip(ws, (3, 2, 1))]
    outs = g.acoustic_forward(p0s)
    for c, p, o in zip(ctxs, p0s, outs):
        assert torch.equal(o, c.acoustic_forward(p))
    Ws = [to_gpu(phantoms.random_field((b, w.nt, w.n_sensors), 9), torch.float32) for w, b in zip(ws, (1, 3, 2))]
    adj = g.acoustic_adjoint(Ws)
    for c, W, o in zip(ctxs, Ws, adj):
        assert torch.equal(o, c.acoustic_adjoint(W))
    # a member may sit out a call
    outs2 = g.acoustic_forward([None, p0s[1], None])
    assert outs2[0] is None and torch.equal(outs2[1], outs[1])
    g.close()


def test_group_jvp_matches_oracle():
    from paper_1810_11685_gb300.binding import Group
    ws = members()
    pairs = [make_pair(w, "fp64", max_batch=2) for w in ws]
    g = Group([p[0] for p in pairs])
    mus = [to_gpu(phantoms.optical_absorption(w), torch.float64) for w in ws]
    dmus = [to_gpu(phantoms.random_field((2,) + w.interior_shape, 4), torch.float64) for w in ws]
    outs = g.jvp([torch.stack([m, m]) for m in mus], dmus, 0b0001)
    for (ctx, S), w, mu, dmu, o in zip(pairs, ws, mus, dmus, outs):
        for b in range(2):
            ref = qpat.jvp(S, to_np(mu), phantoms.optical_diffusion(w), 0b0001, to_np(dmu[b]))
            assert rel_l2(to_np(o[b]), ref) <= 1e-9
    g.close()


def test_autotune_keeps_results():
    w = phantoms.small(n=40, pml=8, nt=40, n_sensors=10, seed=4)
    ctx, S = make_pair(w, "fp32", max_batch=2)
    choice = ctx.autotune(batch=2, steps=20)
    assert set(choice) == {"fast_rows", "fast_cols"}
    p0 = phantoms.smooth_p0(w)
    got = to_np(ctx.acoustic_forward(to_gpu(p0, torch.float32)))[0]
    assert rel_l2(got, acoustic.forward(S, p0)) <= 2e-4


def test_c4_grids_together_first_steps():
    """The three grids of the Newton inner-loop mix (256^2, 384^2, 512^2
    interiors with 16/24/32-cell PMLs) in one group, 4 directions each,
    first 40 steps against the oracle."""
    from paper_1810_11685_gb300.binding import Group
    ws = [phantoms.dataclasses.replace(w, nt=40) for w in phantoms.c4_workloads()]
    pairs = [make_pair(w, "fp32", max_batch=4) for w in ws]
    g = Group([p[0] for p in pairs])
    p0s = [to_gpu(phantoms.random_field((4,) + w.interior_shape, 5), torch.float32) for w in ws]
    outs = g.acoustic_forward(p0s)
    for (ctx, S), p0, o in zip(pairs, p0s, outs):
        ref = acoustic.forward(S, to_np(p0[3]))
        assert rel_l2(to_np(o[3]), ref) <= 2e-4
    g.close()


SHAPES = [(rb, cb, lf) for rb in (144, 288) for cb in (288, 576) for lf in (1, 0)]


@pytest.fixture(scope="module")
def c4_full():
    """The Newton inner-loop mix at full size: 16 problems on each of the
    288^2, 432^2 and 576^2 FFT grids, each grid with its own Nt (1.5 domain
    crossings), white-noise initial pressures and adjoint series."""
    from paper_1810_11685_gb300.binding import Group, context_from_workload
    ws = phantoms.c4_workloads()
    ctxs = []
    for w in ws:
        c, _, _ = phantoms.acoustic_medium(w)
        ctxs.append(context_from_workload(w, precision="fp32", max_batch=16, nt=phantoms.c4_nt(w, c)))
    assert len({c.nt for c in ctxs}) == 3
    g = Group(ctxs)
    p0s = [to_gpu(phantoms.random_field((16,) + w.interior_shape, 5 + k), torch.float32)
           for k, w in enumerate(ws)]
    Ws = [to_gpu(phantoms.random_field((16, c.nt, c.ns), 9 + k), torch.float32) for k, c in enumerate(ctxs)]
    yield ws, ctxs, g, p0s, Ws
    g.close()


def test_c4_multi_launches_equal_member_graphs_bit_for_bit(c4_full):
    """One launch per pass kind for all 48 problems (every block-size and
    item-order shape) against each member's own launch sequence as a graph
    branch: forward and adjoint series identical bit for bit, at full Nt."""
    ws, ctxs, g, p0s, Ws = c4_full
    g.set_shape(multi=0)
    ref_f = [o.clone() for o in g.acoustic_forward(p0s)]
    ref_a = [o.clone() for o in g.acoustic_adjoint(Ws)]
    _, ready = g.shape([16, 16, 16])
    assert ready
    for k, (rb, cb, lf) in enumerate(SHAPES):
        g.set_shape(multi=1, row_block=rb, col_block=cb, largest_first=lf)
        for o, r in zip(g.acoustic_forward(p0s), ref_f):
            assert torch.equal(o, r), (rb, cb, lf)
        if k in (0, len(SHAPES) - 1):
            for o, r in zip(g.acoustic_adjoint(Ws), ref_a):
                assert torch.equal(o, r), (rb, cb, lf)


def test_c4_multi_uneven_nt_against_oracle():
    """Members with different Nt (20, 26, 32) in one multi-problem launch
    sequence: the jvp (diffusion solve, then the acoustic forward) and the
    adjoint of each grid against the oracle, three problems per grid."""
    from paper_1810_11685_gb300.binding import Group
    from oracle import optics
    from gpu_helpers import oracle_many
    ws = [phantoms.dataclasses.replace(w, nt=nt) for w, nt in zip(phantoms.c4_workloads(), (20, 26, 32))]
    ctxs = [make_pair(w, "fp32", max_batch=3)[0] for w in ws]
    g = Group(ctxs)
    g.set_shape(multi=1, row_block=144, col_block=576, largest_first=1)
    assert g.shape([3, 3, 3])[1]
    mus = [phantoms.optical_absorption(w) for w in ws]
    dmus = [phantoms.random_field((3,) + w.interior_shape, 4) for w in ws]
    outs = g.jvp([to_gpu(np.stack([m] * 3), torch.float64) for m in mus],
                 [to_gpu(d, torch.float64) for d in dmus], 0b0001)
    Ws = [phantoms.random_field((3, w.nt, w.n_sensors), 6) for w in ws]
    adj = g.acoustic_adjoint([to_gpu(W, torch.float32) for W in Ws])
    jobs = []
    for w, mu, dmu, W in zip(ws, mus, dmus, Ws):
        dh = optics.jvp(mu, phantoms.optical_diffusion(w), w.dx, 0b0001, dmu[2])
        jobs += [("forward", w, w.nt, dh), ("adjoint", w, w.nt, W[1])]
    ref = oracle_many(jobs)
    for k in range(3):
        assert rel_l2(to_np(outs[k][2]), ref[2 * k]) <= 2e-4
        assert rel_l2(to_np(adj[k][1]), ref[2 * k + 1]) <= 2e-4
    g.close()


def test_group_tune_picks_a_shape_and_keeps_results(c4_full):
    ws, ctxs, g, p0s, Ws = c4_full
    g.set_shape(multi=0)
    ref = [o.clone() for o in g.acoustic_forward(p0s)]
    best, cands = g.tune([16, 16, 16], steps=8)
    assert len(cands) == 1 + len(SHAPES) and all(ms > 0 for _, ms in cands)
    assert best == g.shape()[0] and min(cands, key=lambda c: c[1])[0] == best
    for o, r in zip(g.acoustic_forward(p0s), ref):
        assert torch.equal(o, r)
    assert [c.nt for c in ctxs] == [phantoms.c4_nt(w, phantoms.acoustic_medium(w)[0]) for w in ws]
