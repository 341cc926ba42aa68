"""Parity of annihilation at n_max (Sec. 3) between the CUDA path (a pass
after the cell sort: per-cell scan, then a key bisection per crowded cell)
and the FP64 oracle (per-cell sort and walk), and the discrete Gauss law on
the device with annihilation on.

The weights left on the particles are integers in units of 2^-12 on both
sides and are compared exactly, as are the removed weight and the counts.
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


def _crowded_state(cfg, seed):
    """Electron-positron pairs crowded into a band of cells (weights 0.5, 1,
    1.5), a few atmospheric electrons and ions, and an energetic beam that
    scatters and makes pairs; u32 fixed-point positions."""
    N = cfg["n_cells"]
    F = W.fbits(N)
    rng = np.random.default_rng(seed)
    parts = []
    for c in range(56, 72):
        for code, n in ((W.SP_ELEC, 60), (W.SP_POSI, 60 + int(rng.integers(-10, 10))), (W.SP_ATMO, 8),
                        (W.SP_ION, 8)):
            st = W.empty_state(n)
            st["pos"][:] = ((c + rng.random(n)) * (1 << F)).astype(np.uint32)
            st["u"][:] = rng.normal(0.0, 0.05, n).astype(np.float32)
            st["w"][:] = rng.choice(np.array([0.5, 1.0, 1.5], np.float32), n)
            st["sp"][:] = code
            parts.append(st)
    parts.append(W.load_beam(cfg, 400, gamma_lo=30, gamma_hi=3e3, seed=seed))
    st = {k: np.concatenate([p[k] for p in parts]) for k in parts[0]}
    st["id"] = rng.permutation(len(st["pos"])).astype(np.uint64) * 5 + 7
    return st


def _cfg(**over):
    base = dict(n_cells=128, drag_law=O.DRAG_CLOSED, drag_scale=1e-3, n_max_ppc=60.0, annihilate_every=2,
                capacity=100000)
    base.update(over)
    return W.config("C1", **base)


@pytest.mark.parametrize("every,sort_every", [(2, 20), (3, 2)])
def test_annihilation_parity_over_steps(every, sort_every):
    from paper_2609_17661_b300 import Line
    cfg = _cfg(annihilate_every=every, sort_every=sort_every)
    N = cfg["n_cells"]
    F = W.fbits(N)
    st = _crowded_state(cfg, 21)
    line = Line(cfg)
    line.set_state(st, step=0)
    line.step(8)
    S = O.Sim(cfg)
    o = W.to_oracle(st, N)
    S.set_particles(o["s"], o["u"], o["w"], o["sp"], o["id"])
    S.step(8)
    dg, do = line.diag(), S.diag()
    assert do["annihilated"] > 50 * 4096
    for k in ("annihilated", "n_alive", "pairs_created", "pairs_rejected_nmax", "scatters", "lost_north",
              "lost_south"):
        assert dg[k] == do[k], (k, dg[k], do[k])
    g = _by_id(line.particles())
    og = _by_id(S.particles())
    assert g["id"].tolist() == og["id"].tolist()
    assert np.array_equal(g["w"].astype(np.float64), og["w"])
    assert np.array_equal(g["sp"].astype(np.int32), og["sp"])
    assert _relmax(g["u"].astype(np.float64), og["u"]) <= RTOL
    s = g["pos"].astype(np.float64) / float(1 << F)
    assert np.max(np.abs(s - og["s"])) <= 8 * (2.0 ** -F + cfg["cfl"] * RTOL)
    Eg, _ = line.fields()
    Eo, _ = S.fields()
    assert _relmax(Eg, Eo) <= RTOL


def test_gauss_law_on_the_device_with_annihilation():
    """The device's integer node charge and FP64 field keep the discrete
    Gauss residual constant step by step while annihilation removes charge
    (each removed charge first carried to its cell's left node)."""
    from paper_2609_17661_b300 import Line
    cfg = _cfg(annihilate_every=1)
    N = cfg["n_cells"]
    F = W.fbits(N)
    line = Line(cfg)
    line.set_state(_crowded_state(cfg, 22), step=0)
    scale = 4 * np.pi * line.diag()["q_p"] * 2.0 ** (-12 - F)

    def residual():
        E, _ = line.fields()
        r = line.rho().astype(np.float64)
        return (E[1:] - E[:-1]) - scale * r[1:N], np.max(np.abs(E))

    g0, _ = residual()
    for _ in range(6):
        line.step(1)
        g, emax = residual()
        assert np.max(np.abs(g - g0)) <= 1e-12 * max(1.0, emax)
    assert line.diag()["annihilated"] > 0


def test_annihilation_needs_the_density_limit():
    from paper_2609_17661_b300 import Line
    with pytest.raises(RuntimeError):
        Line(_cfg(n_max_ppc=0.0))
    with pytest.raises(RuntimeError):
        Line(_cfg(annihilate_every=-1))
