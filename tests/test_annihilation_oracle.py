"""Pins of the oracle's annihilation at n_max (Sec. 3: pairs are annihilated
where the density reaches the skin-depth limit n_max).

The oracle sorts each cell's pair particles by their key and walks them; the
pins here recompute the expected result by brute force, in Python, with an
independent SplitMix64 written from its published definition (Steele, Lea
and Flood 2014), from the same line stepped without annihilation (the pass
acts at the end of the step, so that twin is the state it starts from):

* the weights left on every particle, the particles removed, and E;
* charge: both species lose the same weight, so the total charge is kept;
* the cap: a cell not limited by one species' weight ends at n_max or one
  unit above it (integer weights);
* the discrete Gauss law holds to rounding every step while annihilation,
  scattering, pairs and losses act;
* no pass below n_max, and passes only every annihilate_every steps.
"""
import math

import numpy as np
import pytest

import oracle as O
from paper_2609_17661_b300 import workloads as W

WQ = 4096
M64 = (1 << 64) - 1


def splitmix64(z):
    z = (z + 0x9E3779B97F4A7C15) & M64
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & M64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & M64
    return z ^ (z >> 31)


def key(pid, step):
    return splitmix64(int(pid) ^ splitmix64((int(step) ^ 0xA1111A7E) & M64))


def test_python_splitmix_and_key_match_the_definition():
    assert splitmix64(0) == 0xE220A8397B1DCDAF           # first output of the generator seeded with 0
    for pid, step in ((0, 1), (12345, 20), (2**63 + 7, 400)):
        assert O.annih_key(pid, step) == key(pid, step)


def _dense_pairs(cfg, seed=3, cells=range(56, 72), per_cell=60):
    """Electron-positron pairs (and a few atmospheric electrons and ions)
    crowded into a band of cells, weights 0.5, 1 or 1.5, slow."""
    rng = np.random.default_rng(seed)
    N = cfg["n_cells"]
    s, sp, w = [], [], []
    for c in cells:
        for code, n in ((W.SP_ELEC, per_cell), (W.SP_POSI, per_cell + rng.integers(-10, 10)),
                        (W.SP_ATMO, 8), (W.SP_ION, 8)):
            s.append(c + rng.random(n))
            sp.append(np.full(n, code))
            w.append(rng.choice([0.5, 1.0, 1.5], n))
    s = np.concatenate(s)
    n = s.size
    return dict(s=s, u=rng.normal(0.0, 0.05, n), w=np.concatenate(w),
                sp=np.concatenate(sp).astype(np.int32), id=rng.permutation(n).astype(np.uint64) * 3 + 11)


def _sim(cfg, st, step0):
    S = O.Sim(cfg)
    S.set_particles(st["s"], st["u"], st["w"], st["sp"], st["id"])
    S.set_step(step0)
    return S


def _cfg(**over):
    base = dict(n_cells=128, drag_law=O.DRAG_OFF, mc_on=0, pairs_on=0, n_max_ppc=80.0, annihilate_every=1)
    base.update(over)
    return W.config("C1", **base)


def _brute_force(p, E, cfg, step):
    """Annihilation of a state p (after the push) written out per cell."""
    N = cfg["n_cells"]
    nmax = math.floor(cfg["n_max_ppc"] * WQ)
    q_p = O.Sim(cfg).scalars()["q_p"]
    wint = np.rint(p["w"] * WQ).astype(np.int64)
    cell = np.floor(p["s"]).astype(np.int64)
    E = E.copy()
    lep = p["sp"] != W.SP_ION
    removed = 0
    limited = {}
    for c in range(N):
        inc = cell == c
        Wc = int(wint[inc & lep].sum())
        if Wc <= nmax:
            continue
        Wp = int(wint[inc & (p["sp"] == W.SP_POSI)].sum())
        We = int(wint[inc & (p["sp"] == W.SP_ELEC)].sum())
        A = min((Wc - nmax) // 2, Wp, We)
        limited[c] = A < (Wc - nmax) // 2
        if A <= 0:
            continue
        X = 0.0
        for code, q in ((W.SP_ELEC, -1.0), (W.SP_POSI, 1.0)):
            idx = np.nonzero(inc & (p["sp"] == code))[0]
            idx = sorted(idx, key=lambda i: key(p["id"][i], step))
            left = A
            for i in idx:
                if left == 0:
                    break
                d = min(int(wint[i]), left)
                left -= d
                wint[i] -= d
                X += q * d / WQ * (p["s"][i] - c)
        E[c] += 4 * np.pi * q_p * X
        removed += 2 * A
    keep = wint > 0
    out = {k: v[keep] for k, v in p.items()}
    out["w"] = wint[keep] / WQ
    return out, E, removed, limited


def test_annihilation_equals_brute_force():
    cfg = _cfg()
    st = _dense_pairs(cfg)
    A = _sim(cfg, st, 19)
    B = _sim(dict(cfg, annihilate_every=0), st, 19)
    A.step(1)
    B.step(1)
    pb = B.particles()
    Eb, _ = B.fields()
    exp, Ee, removed, _ = _brute_force(pb, Eb, cfg, 20)
    pa = A.particles()
    assert removed > 20 * WQ and A.diag()["annihilated"] == removed
    oa, oe = np.argsort(pa["id"]), np.argsort(exp["id"])
    assert np.array_equal(pa["id"][oa], exp["id"][oe])
    assert np.array_equal(pa["w"][oa], exp["w"][oe])
    assert np.array_equal(pa["s"][oa], exp["s"][oe])
    Ea, _ = A.fields()
    np.testing.assert_allclose(Ea, Ee, rtol=0, atol=1e-13 * max(1.0, np.max(np.abs(Ee))))


def test_charge_kept_and_cells_capped():
    cfg = _cfg()
    st = _dense_pairs(cfg, seed=4)
    A = _sim(cfg, st, 3)
    B = _sim(dict(cfg, annihilate_every=0), st, 3)
    A.step(1)
    B.step(1)
    qa, qb = A.diag()["charge"], B.diag()["charge"]
    assert qa == pytest.approx(qb, rel=1e-13, abs=1e-15)
    pb = B.particles()
    _, _, _, limited = _brute_force(pb, B.fields()[0], cfg, 4)
    pa = A.particles()
    nmax = math.floor(cfg["n_max_ppc"] * WQ)
    wint = np.rint(pa["w"] * WQ).astype(np.int64)
    lep = pa["sp"] != W.SP_ION
    Wc = np.bincount(np.floor(pa["s"][lep]).astype(np.int64), weights=wint[lep], minlength=cfg["n_cells"])
    assert len(limited) > 5
    for c, lim in limited.items():
        if not lim:
            assert nmax <= Wc[c] <= nmax + 1, c


def test_no_pass_below_n_max_and_only_on_the_cadence():
    st = _dense_pairs(_cfg(), seed=5)
    S = _sim(_cfg(n_max_ppc=1e6), st, 0)
    S.step(3)
    assert S.diag()["annihilated"] == 0
    S = _sim(_cfg(annihilate_every=4), st, 0)
    S.step(3)
    assert S.diag()["annihilated"] == 0
    S.step(1)
    assert S.diag()["annihilated"] > 0


def test_gauss_law_every_step_with_annihilation():
    """G2-a with annihilation: the discrete Gauss residual stays at its
    initial value to rounding while annihilation, drag, scattering and pairs
    act."""
    cfg = _cfg(drag_law=O.DRAG_CLOSED, mc_on=1, pairs_on=1, drag_scale=1e-3, annihilate_every=2, n_max_ppc=60.0)
    st = _dense_pairs(cfg, seed=6)
    beam = W.to_oracle(W.load_beam(cfg, 400, gamma_lo=30, gamma_hi=3e3, seed=4), cfg["n_cells"])
    beam["id"] = beam["id"] + 10**6
    both = {k: np.concatenate([st[k], beam[k]]) for k in st}
    S = _sim(cfg, both, 0)
    E, _ = S.fields()
    r = S.rho()
    N = cfg["n_cells"]
    g0 = (E[1:] - E[:-1]) - 4 * np.pi * r[1:N]
    for _ in range(12):
        S.step(1)
        E, _ = S.fields()
        r = S.rho()
        g = (E[1:] - E[:-1]) - 4 * np.pi * r[1:N]
        assert np.max(np.abs(g - g0)) <= 1e-12 * max(1.0, np.max(np.abs(E)))
    assert S.diag()["annihilated"] > 0


def test_gauss_law_with_the_atmosphere_and_annihilation_together():
    """Top-up pairs appear neutral at one point and annihilation carries its
    removed charge to a node first: with both on (and gravity, drag,
    scattering, pairs), the discrete Gauss residual stays constant."""
    cfg = _cfg(drag_law=O.DRAG_CLOSED, mc_on=1, pairs_on=1, drag_scale=1e-3, annihilate_every=3, n_max_ppc=60.0,
               inject_mode=O.INJECT_TOPUP, atmo_a0=2000.0, atmo_h=4.0)
    st = _dense_pairs(cfg, seed=8)
    S = _sim(cfg, st, 0)
    N = cfg["n_cells"]
    E, _ = S.fields()
    g0 = (E[1:] - E[:-1]) - 4 * np.pi * S.rho()[1:N]
    for _ in range(9):
        S.step(1)
        E, _ = S.fields()
        g = (E[1:] - E[:-1]) - 4 * np.pi * S.rho()[1:N]
        assert np.max(np.abs(g - g0)) <= 1e-12 * max(1.0, np.max(np.abs(E)))
    d = S.diag()
    assert d["annihilated"] > 0 and d["injected"] > 0


def test_a_cell_with_one_species_does_not_annihilate():
    """Degenerate cell: far above n_max but holding positrons only (no pair
    electrons), so A = min(..., W+, W-) = 0 and nothing is removed."""
    cfg = _cfg(n_max_ppc=5.0)
    rng = np.random.default_rng(2)
    n = 200
    st = dict(s=60 + rng.random(n), u=np.zeros(n), w=np.ones(n), sp=np.full(n, W.SP_POSI, np.int32),
              id=np.arange(n, dtype=np.uint64))
    S = _sim(cfg, st, 0)
    S.step(1)
    assert S.diag()["annihilated"] == 0
    assert S.particles()["s"].size == n
