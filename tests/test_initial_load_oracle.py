"""Pins of the oracle's initial plasma (Sec. 3: a pair plasma of multiplicity
M whose leptons drift at beta = -+1/M, the carriers of the twist current,
with ions; loaded when ppc_e > 0), CPU only.

* one cell recomputed from the recipe with the test's own plain-Python
  Philox4x32-10 and integer arithmetic equals the oracle's particles;
* electron k of a cell sits in the k-th of ppc_e equal parts of it, and the
  positrons and ions sit on electron positions, so every node is neutral
  (the CIC charge density is zero everywhere);
* the momenta are Gaussian with the stated spread around -u_d, +u_d and 0,
  u_d = beta_d / sqrt(1 - beta_d^2) with beta_d = 1/M;
* the load's current equals the external current j_ext = j_psi n0 e c of the
  C1 line within its statistical error.
"""
import math

import numpy as np
from scipy import stats

import oracle as O
from paper_2609_17661_b300 import workloads as W

TAG_INIT = 0x494E4954


def _py_philox(ctr, key):
    """Philox4x32-10 (Salmon et al. 2011), written out in plain Python."""
    c = list(ctr)
    k = list(key)
    M = 0xFFFFFFFF
    for _ in range(10):
        p0 = 0xD2511F53 * c[0]
        p1 = 0xCD9E8D57 * c[2]
        c = [((p1 >> 32) ^ c[1] ^ k[0]) & M, p1 & M, ((p0 >> 32) ^ c[3] ^ k[1]) & M, p0 & M]
        k = [(k[0] + 0x9E3779B9) & M, (k[1] + 0xBB67AE85) & M]
    return c


def _cfg(**over):
    return W.config("C1", ppc_e=16, ppc_p=8, ppc_i=8, **over)


def _sim(cfg):
    S = O.Sim(cfg)
    return S, S.particles()


def test_one_cell_from_the_recipe_with_an_independent_generator():
    cfg = _cfg(seed=77)
    N = cfg["n_cells"]
    F = W.fbits(N)
    S, p = _sim(cfg)
    ne, np_ = N * 16, N * 8
    key = [77, 0]
    for c in (0, 5, N - 1):
        for k in range(16):
            r = _py_philox([c, k, 0, TAG_INIT], key)
            A = (k << 24) + (r[0] >> 8)
            frac = (A << (F - 24)) // 16 if F >= 24 else A // (16 << (24 - F))
            s_want = ((c << F) + frac) / float(1 << F)
            for m, slot in ((0, c * 16 + k), (1, ne + c * 8 + k if k < 8 else None),
                            (2, ne + np_ + c * 8 + (k - 8) if k >= 8 else None)):
                if slot is None:
                    continue
                q = r if m == 0 else _py_philox([c, k, m, TAG_INIT], key)
                U1 = ((q[1] >> 8) + 1) / 16777216.0
                U2 = (q[2] >> 8) / 16777216.0
                g = math.sqrt(-2.0 * math.log(U1)) * math.cos(2.0 * math.pi * U2)
                beta = 0.25
                ud = beta / math.sqrt(1 - beta * beta)
                drift = (-ud, ud, 0.0)[m]
                assert p["id"][slot] == slot
                assert p["sp"][slot] == (W.SP_ELEC, W.SP_POSI, W.SP_ION)[m]
                assert p["s"][slot] == s_want
                assert p["u"][slot] == drift + 0.1 * g or abs(p["u"][slot] - (drift + 0.1 * g)) < 1e-15


def test_stratified_positions_and_neutral_nodes():
    cfg = _cfg()
    N = cfg["n_cells"]
    S, p = _sim(cfg)
    ne = N * 16
    assert S.n == N * 32
    s_e = p["s"][:ne].reshape(N, 16)
    lo = np.arange(N)[:, None] + np.arange(16)[None, :] / 16.0
    assert np.all(s_e >= lo) and np.all(s_e < lo + 1.0 / 16)
    assert np.array_equal(p["s"][ne:ne + N * 8].reshape(N, 8), s_e[:, :8])
    assert np.array_equal(p["s"][ne + N * 8:].reshape(N, 8), s_e[:, 8:])
    # every node neutral: exactly in integer charge units (CIC weights of
    # fixed-point positions), to rounding in the oracle's FP64 node charge
    F = W.fbits(N)
    pos = np.rint(p["s"] * (1 << F)).astype(np.int64)
    assert np.array_equal(pos.astype(np.float64) / (1 << F), p["s"])
    i = np.minimum(pos >> F, N - 1)
    f = pos - (i << F)
    qs = np.array([-1, 1, 1, -1], np.int64)[p["sp"]]
    rho = np.zeros(N + 1, np.int64)
    np.add.at(rho, i, qs * ((1 << F) - f))
    np.add.at(rho, i + 1, qs * f)
    assert np.all(rho == 0)
    assert np.max(np.abs(S.rho())) <= 1e-12 * 16 * S.scalars()["q_p"]
    counts = [np.sum(p["sp"] == sp) for sp in (W.SP_ELEC, W.SP_POSI, W.SP_ION)]
    assert counts == [N * 16, N * 8, N * 8]


def test_momenta_gaussian_around_the_drift():
    cfg = _cfg(n_cells=4096, u_sigma=0.1, init_multiplicity=4.0)
    S, p = _sim(cfg)
    ud = 0.25 / math.sqrt(1 - 0.25 ** 2)
    for sp, mean in ((W.SP_ELEC, -ud), (W.SP_POSI, ud), (W.SP_ION, 0.0)):
        u = p["u"][p["sp"] == sp]
        n = u.size
        assert abs(u.mean() - mean) < 4 * 0.1 / math.sqrt(n)
        assert abs(u.std() - 0.1) < 4 * 0.1 / math.sqrt(2 * n)
        assert stats.kstest((u - mean) / 0.1, "norm").pvalue > 1e-3


def test_the_load_carries_the_external_current():
    """sum over particles of q beta per cell (in units of the macro charge
    q_p) equals j_ext / q_p = j_psi n0_ppc on the C1 line (M = 4: 24 leptons
    per cell at beta 1/4 carry 6 = 28 x 6/28)."""
    cfg = _cfg(n_cells=4096)
    S, p = _sim(cfg)
    N = cfg["n_cells"]
    q = np.array([-1.0, 1.0, 1.0, -1.0])[p["sp"]]
    m = np.where(p["sp"] == W.SP_ION, cfg["mass_ratio"], 1.0)
    beta = p["u"] / np.sqrt(1.0 + p["u"] ** 2)
    j = np.sum(q * beta) / N
    want = cfg["j_psi"] * cfg["n0_ppc"]
    assert abs(j - want) < 4 * 24 * 0.1 / math.sqrt(N * 24) + 0.01 * want
    sc = S.scalars()
    assert abs(sc["j_ext"] / sc["q_p"] - want) < 1e-12 * want
    del m
