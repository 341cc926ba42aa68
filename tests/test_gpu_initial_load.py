"""The initial plasma loaded by pic1d_init (ppc_e > 0, Sec. 3) against the
oracle's load of the same parameters: ids, species and fixed-point positions
identical, momenta to the FP32 rounding of the Box-Muller Gaussians; the
pair cap's density counted; and the line stepped from it agrees with the
oracle stepped from its own load."""
import numpy as np
import pytest

import oracle as O
from paper_2609_17661_b300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _by_id(p):
    o = np.argsort(p["id"])
    return {k: v[o] for k, v in p.items()}


@pytest.mark.parametrize("n_cells,seed", [(1024, 1), (4096, 9), (65536, 3)])
def test_device_load_equals_the_oracle_load(n_cells, seed):
    from paper_2609_17661_b300 import Line
    cfg = W.config("C1", n_cells=n_cells, ppc_e=16, ppc_p=8, ppc_i=8, seed=seed, n_max_ppc=40.0)
    line = Line(cfg)
    g = _by_id(line.particles())
    S = O.Sim(cfg)
    o = _by_id(S.particles())
    F = W.fbits(n_cells)
    assert g["id"].size == n_cells * 32
    np.testing.assert_array_equal(g["id"], o["id"])
    np.testing.assert_array_equal(g["sp"].astype(np.int32), o["sp"])
    np.testing.assert_array_equal(g["pos"].astype(np.float64) / float(1 << F), o["s"])
    np.testing.assert_allclose(g["u"].astype(np.float64), o["u"], rtol=0, atol=2e-6)
    assert np.all(g["w"] == 1.0)
    d = line.diag()
    assert d["n_alive"][:3] == [n_cells * 16, n_cells * 8, n_cells * 8]
    line.close()


def test_line_from_its_load_steps_like_the_oracle():
    """C1 from pic1d_init's own load, 60 steps (within the plasma's
    predictable horizon): E and every momentum to 1e-5 of their largest
    value."""
    from paper_2609_17661_b300 import Line
    cfg = W.config("C1", ppc_e=16, ppc_p=8, ppc_i=8, pairs_on=0)
    line = Line(cfg)
    line.step(60)
    S = O.Sim(cfg)
    S.step(60)
    Eg, _ = line.fields()
    Eo, _ = S.fields()
    assert np.max(np.abs(Eg - Eo)) <= 1e-5 * np.max(np.abs(Eo))
    g = _by_id(line.particles())
    o = _by_id(S.particles())
    np.testing.assert_array_equal(g["id"], o["id"])
    assert np.max(np.abs(g["u"].astype(np.float64) - o["u"])) <= 1e-5 * np.max(np.abs(o["u"]))
    line.close()
