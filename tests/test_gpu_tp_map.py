"""The GPU test-particle drag map against the FP64 oracle, line by line."""
import numpy as np
import pytest

import oracle as O
from paper_2609_17661_b300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

CFG = W.config("C1", kT_keV=1.0, photon_model=O.PHOTON_RADIAL, drag_scale=1.0)


def test_map_matches_oracle_line_by_line():
    from paper_2609_17661_b300 import tp_map
    r = np.geomspace(2.1, 60.0, 48)
    g, ms = tp_map(CFG, r, gamma0=1000.0, dt=2e-3, t_max=60.0)
    assert ms > 0
    for k, rk in enumerate(r):
        o = O.tp_line(CFG, rk, gamma0=1000.0, dt=2e-3, t_max=60.0)
        # FP64 on both sides; the libraries' transcendentals differ in the last bit
        assert abs(g["steps"][k] - o["steps"]) <= 1, k
        for f in ("gamma_min", "theta_b", "s_b", "L", "b_eq"):
            assert g[f][k] == pytest.approx(o[f], rel=1e-9, abs=1e-12), (k, f)
        for f in ("theta_first", "s_first", "l_pp"):
            assert g[f][k] == pytest.approx(o[f], rel=1e-7, abs=1e-9), (k, f)
        assert g["region"][k] == o["region"], k
    assert set(g["region"].tolist()) == {1, 2, 3}


def test_map_rejects_bad_lines():
    from paper_2609_17661_b300 import PicError, tp_map
    with pytest.raises(PicError):
        tp_map(CFG, [3.0, 0.5])
