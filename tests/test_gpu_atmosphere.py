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


def test_top_up_is_refused_with_the_surrogate_drag_law():
    from paper_2609_17661_b300 import Line
    with pytest.raises(RuntimeError):
        Line(W.config("C1", inject_mode=O.INJECT_TOPUP, drag_law=W.DRAG_SURROGATE))
    with pytest.raises(RuntimeError):
        Line(W.config("C1", inject_mode=O.INJECT_TOPUP, atmo_h=0.0))
