"""Parity of the atmosphere (inject mode TOPUP: the density profile of
App. B.1, Eq. densprofile, topped up every step, and gravity -T/h along r)
between the CUDA path and the FP64 oracle.

The number of particles topped up in a cell depends on the cell's plasma
weight after the move (integer sums), so the counts are compared exactly;
the topped-up particles themselves (ids, positions, momenta) by id, with the
tolerances of the other parity tests.
"""
import numpy as np
import pytest

import oracle as O
from paper_2609_17661_b300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

RTOL = 1e-5


def _by_id(p):
    o = np.argsort(p["id"])
    return {k: v[o] for k, v in p.items()}


def _relmax(a, b):
    return np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300)


def _field0(N):
    x = (np.arange(N) + 0.5) / N
    return 0.01 * np.sin(2 * np.pi * 3 * x) + 0.003 * np.cos(2 * np.pi * 7 * x + 1.0)


def _run_both(cfg, st, E, steps, step0=3):
    from paper_2609_17661_b300 import Line
    line = Line(cfg)
    line.set_state(st, E=E, step=step0)
    line.step(steps)
    S = O.Sim(cfg)
    o = W.to_oracle(st, cfg["n_cells"])
    S.set_particles(o["s"], o["u"], o["w"], o["sp"], o["id"])
    S.set_field(E)
    S.set_step(step0)
    S.step(steps)
    return line, S


def _compare(line, S, cfg, steps):
    N = cfg["n_cells"]
    F = W.fbits(N)
    dg, do = line.diag(), S.diag()
    for k in ("injected", "n_alive", "lost_north", "lost_south", "pairs_created", "scatters"):
        assert dg[k] == do[k], (k, dg[k], do[k])
    assert dg["injected_dropped"] == 0
    g = _by_id(line.particles())
    g["s"] = g["pos"].astype(np.float64) / float(1 << F)
    o = _by_id(S.particles())
    assert g["id"].tolist() == o["id"].tolist()
    assert np.array_equal(g["sp"].astype(np.int32), o["sp"])
    assert _relmax(g["u"].astype(np.float64), o["u"]) <= RTOL
    assert np.max(np.abs(g["s"] - o["s"])) <= steps * (2.0 ** -F + cfg["cfl"] * RTOL)
    Eg, _ = line.fields()
    Eo, _ = S.fields()
    assert _relmax(Eg, Eo) <= RTOL


@pytest.mark.parametrize("n_max_ppc", [0.0, 60.0])
def test_atmosphere_top_up_and_gravity_parity(n_max_ppc):
    """Five steps of a C1 line with drag, scattering and pairs, from a sparse
    random state: the first step fills the atmosphere's deficit (about 1,400
    particles), the next ones refill what the field and the thermal motion
    move; with the pair cap (n_max) on, the push that also sums the lepton
    density runs."""
    N = 1024
    cfg = W.config("C1", inject_mode=O.INJECT_TOPUP, drag_law=O.DRAG_TABLE, drag_scale=3e-3,
                   n_max_ppc=n_max_ppc, capacity=200000)
    st = W.load_random(cfg, 6000, u_scale=3.0, seed=11)
    line, S = _run_both(cfg, st, _field0(N), 5)
    assert S.diag()["injected"] > 1400
    _compare(line, S, cfg, 5)


def test_atmosphere_from_an_empty_line_matches_the_oracle_over_twelve_steps():
    """The atmosphere alone (no other particles, drag on): twelve steps of
    top-up, gravity and the field the atmosphere's own currents make."""
    N = 1024
    cfg = W.config("C1", inject_mode=O.INJECT_TOPUP, drag_law=O.DRAG_TABLE, drag_scale=3e-3, capacity=100000)
    st = W.empty_state(0)
    line, S = _run_both(cfg, st, np.zeros(N), 12, step0=0)
    _compare(line, S, cfg, 12)
    assert S.diag()["injected"] > 1700


def test_atmosphere_ignores_the_push_variant():
    """The streaming push (variant 0) and the per-thread push (variant 2, which
    runs the atmosphere's own instantiation) give the same results with the
    atmosphere's gravity and weight sums."""
    from paper_2609_17661_b300 import Line
    N = 1024
    cfg = W.config("C1", inject_mode=O.INJECT_TOPUP, drag_law=O.DRAG_TABLE, drag_scale=3e-3, capacity=100000)
    st = W.load_random(cfg, 3000, u_scale=3.0, seed=12)
    out = []
    for v in (0, 2):
        line = Line(cfg)
        line.set_variant(v)
        line.set_state(st, E=_field0(N), step=1)
        line.step(3)
        p = _by_id(line.particles())
        out.append((p, line.fields()[1], line.diag()["injected"]))
    (p0, J0, i0), (p1, J1, i1) = out
    assert i0 == i1
    for k in ("pos", "u", "id", "sp"):
        assert np.array_equal(p0[k], p1[k]), k
    assert np.array_equal(J0, J1)


def test_atmosphere_with_the_surrogate_drag_law_matches_the_oracle():
    """The atmosphere (top-up and gravity) with drag law SURROGATE: five
    steps of the C1 line from a sparse random state, against the oracle with
    the same BF16-exact network.  Counts (top-up, losses, pairs) exact; the
    momenta to 1e-5 of the line's scale plus 3 % of the drag's own change of
    u (the network's BF16 activations); E to 1e-5."""
    from oracle import surrogate as SU
    from paper_2609_17661_b300 import Line
    N = 1024
    # continuous drag everywhere (no scattering draws that the network's BF16
    # rate could tip), Newton without the limiter
    cfg = W.config("C1", inject_mode=O.INJECT_TOPUP, drag_law=O.DRAG_SURROGATE, drag_scale=3e-3, capacity=200000,
                   b_pair_threshold=1e30, mc_on=0, pairs_on=0, eta_min=0.0)
    theta = SU.bf16_tensor_layers(W.sur_init_params(21).astype(np.float64))
    st = W.load_random(cfg, 6000, u_scale=3000.0, seed=11)
    E = _field0(N)
    line = Line(cfg)
    line.sur_set_params(theta.astype(np.float32))
    line.set_state(st, E=E, step=3)
    line.step(5)
    o_ = W.to_oracle(st, N)
    runs = {}
    for law in (O.DRAG_SURROGATE, O.DRAG_OFF):
        S = O.Sim(dict(cfg, drag_law=law))
        if law == O.DRAG_SURROGATE:
            S.set_surrogate(theta)
        S.set_particles(o_["s"], o_["u"], o_["w"], o_["sp"], o_["id"])
        S.set_field(E)
        S.set_step(3)
        S.step(5)
        runs[law] = S
    S = runs[O.DRAG_SURROGATE]
    dg, do = line.diag(), S.diag()
    for k in ("injected", "n_alive", "lost_north", "lost_south", "newton_branch"):
        assert dg[k] == do[k], (k, dg[k], do[k])
    assert do["injected"] > 1400
    g = _by_id(line.particles())
    o = _by_id(S.particles())
    o0 = _by_id(runs[O.DRAG_OFF].particles())
    assert g["id"].tolist() == o["id"].tolist()
    drag_du = np.zeros(o["u"].size)
    common = np.isin(o["id"], o0["id"])
    drag_du[common] = np.abs(o["u"][common] - o0["u"][np.searchsorted(o0["id"], o["id"][common])])
    tol = 1e-5 * np.max(np.abs(o["u"])) + 0.03 * drag_du
    err = np.abs(g["u"].astype(np.float64) - o["u"])
    assert np.all(err <= tol), (float(np.max(err / tol)), int(np.sum(err > tol)))
    Eg, _ = line.fields()
    Eo, _ = S.fields()
    assert _relmax(Eg, Eo) <= RTOL


def test_top_up_parameters_are_checked():
    from paper_2609_17661_b300 import Line
    with pytest.raises(RuntimeError):
        Line(W.config("C1", inject_mode=O.INJECT_TOPUP, atmo_h=0.0))
