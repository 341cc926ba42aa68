"""Discrete continuity on the device (Sec. 3: the deposit conserves charge,
so Gauss's law, once satisfied, stays satisfied).

After pic1d_gauss_mark the library keeps the cumulative current of every
cell and pic1d_diag reports max_i |rho_i - rho_ref_i - (Jcum_{i-1} - Jcum_i)|
over the interior nodes, in the integer units of the deposit.  These tests
step lines with pairs, scattering, supply, annihilation and losses, and check
(1) that residual is exactly 0 while the node charge itself changes, and
(2) the same residual recomputed here from pic1d_get_rho and each step's J.
"""
import numpy as np
import pytest

import oracle as O
from paper_2609_17661_b300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _crowded(cfg, seed):
    N = cfg["n_cells"]
    F = W.fbits(N)
    rng = np.random.default_rng(seed)
    parts = [W.load_random(cfg, 4000, u_scale=300.0, seed=seed + 1)]
    for c in range(N // 2 - 8, N // 2 + 8):
        for code, n in ((W.SP_ELEC, 60), (W.SP_POSI, 60 + int(rng.integers(-10, 10)))):
            st = W.empty_state(n)
            st["pos"][:] = ((c + rng.random(n)) * (1 << F)).astype(np.uint32)
            st["u"][:] = rng.normal(0.0, 0.05, n).astype(np.float32)
            st["w"][:] = rng.choice(np.array([0.5, 1.0, 1.5], np.float32), n)
            st["sp"][:] = code
            parts.append(st)
    parts.append(W.load_beam(cfg, 400, gamma_lo=30, gamma_hi=3e3, seed=seed))
    st = {k: np.concatenate([p[k] for p in parts]) for k in parts[0]}
    st["id"] = rng.permutation(len(st["pos"])).astype(np.uint64) * 3 + 1
    return st


CASES = {
    # pairs and scattering from a beam, surface supply at a rate, sort every 4
    "rate_pairs": lambda: (W.config("C1", inject_mode=O.INJECT_RATE, sort_every=4, capacity=400000), None),
    # the atmosphere's top-up with gravity, pair cap on
    "topup": lambda: (W.config("C1", inject_mode=O.INJECT_TOPUP, drag_law=O.DRAG_TABLE, drag_scale=3e-3,
                               n_max_ppc=60.0, capacity=400000), None),
    # annihilation at n_max every 2 steps on a crowded band
    "annihilation": lambda: (W.config("C1", n_cells=128, drag_law=O.DRAG_CLOSED, drag_scale=1e-3, n_max_ppc=60.0,
                                      annihilate_every=2, capacity=200000), "crowded"),
}


@pytest.mark.parametrize("case", sorted(CASES))
def test_continuity_residual_is_zero(case):
    from paper_2609_17661_b300 import Line
    cfg, kind = CASES[case]()
    N = cfg["n_cells"]
    line = Line(cfg)
    if kind == "crowded":
        st = _crowded(cfg, 5)
    else:
        st = W.load_drifting_plasma(cfg, seed=3)
        beam = W.load_beam(cfg, 2000, gamma_lo=30, gamma_hi=1e5, seed=4)
        st = {k: np.concatenate([st[k], beam[k]]) for k in st}
        st["id"] = np.arange(st["pos"].size, dtype=np.uint64) * 7 + 2
    line.set_state(st, step=0)
    d = line.diag()
    assert d["gauss_marked"] == 0 and d["gauss_residual_max"] == -1
    line.gauss_mark()
    rho_ref = line.rho()
    jcum = np.zeros(N, np.int64)
    for _ in range(12):
        line.step(1)
        jcum += line.fields()[1]
        d = line.diag()
        assert d["gauss_marked"] == 1
        assert d["gauss_residual_max"] == 0, (d["gauss_residual_max"], d["gauss_residual_node"])
    rho = line.rho()
    if case != "annihilation":
        # host recomputation from the node charges and the steps' currents
        r = rho[1:N] - rho_ref[1:N] - (jcum[:-1] - jcum[1:])
        assert np.all(r == 0)
    assert np.count_nonzero(rho != rho_ref) > N // 4        # the charge did move
    if case == "annihilation":
        assert d["annihilated"] > 0
    elif case == "rate_pairs":
        assert d["pairs_created"] > 0 and d["injected"] > 0 and d["lost_north"] + d["lost_south"] > 0
    else:
        assert d["injected"] > 0
    line.set_state(st, step=0)
    d = line.diag()
    assert d["gauss_marked"] == 0 and d["gauss_residual_max"] == -1


def test_continuity_residual_in_the_ensemble():
    """Lines of the ensemble keep the cumulative current in its own field
    update and annihilation passes: zero residual after a captured
    super-step plus directly launched steps."""
    from paper_2609_17661_b300 import Ensemble
    cfgs, states = [], []
    for k, (r, N, n, ae) in enumerate([(3.0, 512, 6000, 2), (8.0, 1024, 20000, 0)]):
        c = W.config("C1", r_eq=r, n_cells=N, drag_law=W.DRAG_SURROGATE, inject_mode=O.INJECT_TOPUP,
                     annihilate_every=ae, n_max_ppc=60.0 if ae else 0.0, drag_scale=0.05, seed=3 + k,
                     sort_every=20, capacity=400000)
        cfgs.append(c)
        states.append(W.load_pair_loaded(c, n, seed=70 + k) if ae == 0 else _crowded(c, 80 + k))
    ens = Ensemble(cfgs)
    ens.lines[0].sur_set_params(W.sur_init_params(31))
    for ln, st in zip(ens.lines, states):
        ln.set_state(st)
        ln.gauss_mark()
    ens.step(83)
    for k, ln in enumerate(ens.lines):
        d = ln.diag()
        assert d["gauss_marked"] == 1 and d["gauss_residual_max"] == 0, (k, d["gauss_residual_max"])
    assert ens.lines[0].diag()["annihilated"] > 0
    ens.close()
