"""The synthetic input generators (no method arithmetic): the torch
generator of the pair-loaded line, which the full-size parity test draws on
the device, gives the host generator's per-cell counts exactly and its
species mix and momentum distribution statistically (run here on the CPU)."""
import numpy as np
import pytest

from paper_2609_17661_b300 import workloads as W

torch = pytest.importorskip("torch")


def test_torch_pair_loaded_matches_the_host_generator():
    cfg = W.config("C5")
    N = cfg["n_cells"]
    F = W.fbits(N)
    total = 2_000_000
    t = W.pair_loaded_torch(cfg, total, seed=5, device="cpu")
    h = W.load_pair_loaded(cfg, total)
    pos = t["pos"].numpy().view(np.uint32)
    assert pos.size == h["pos"].size
    assert np.array_equal(np.bincount(pos >> F, minlength=N), np.bincount(h["pos"] >> F, minlength=N))
    assert np.all(np.diff(pos >> F) >= 0)                         # cell-sorted
    assert np.array_equal(pos[0::2], pos[1::2])                   # pairs share a position
    assert np.array_equal(t["id"].numpy(), np.arange(pos.size))
    assert np.all(t["w"].numpy() == 1.0)
    sp, u = t["sp"].numpy(), t["u"].numpy()
    for k in (W.SP_ELEC, W.SP_POSI, W.SP_ION):
        assert abs((sp == k).mean() - (h["sp"] == k).mean()) < 2e-3
    lep = sp != W.SP_ION
    hl = h["sp"] != W.SP_ION
    for q in (0.1, 0.5, 0.9):
        a = np.quantile(np.log10(np.abs(u[lep])), q)
        b = np.quantile(np.log10(np.abs(h["u"][hl])), q)
        assert abs(a - b) < 0.01, q
    assert abs(np.sign(u[lep]).mean()) < 3e-3
    assert np.std(u[sp == W.SP_ION]) == pytest.approx(0.01, rel=0.02)
