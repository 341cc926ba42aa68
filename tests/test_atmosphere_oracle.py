"""Pins of the oracle's atmosphere (inject mode TOPUP; Sec. 3 and App. B.1,
Eq. densprofile).  Each pin is computed here from the paper's definitions
with an independent dipole geometry (scipy quadrature of the arc length and a
root finder for theta(s)), not from the oracle's own tables:

* the first top-up of an empty line equals the profile
  n/n0 = a0 exp(-(r - R*)/h), cell by cell, in pairs of weight 1;
* after any step, every atmosphere cell holds its target weight to within
  one pair, and no particle is injected outside the atmosphere;
* gravity is -T/h along r: one step of a particle at rest at a cell centre
  changes u by -T/h mu_s dt / m (north: toward the star, south: likewise,
  with the opposite sign along s), and by nothing outside the atmosphere;
* the injected momenta are Maxwellian at T for both species (variance T/m),
  the positions uniform inside their cell.
"""
import math

import numpy as np
import pytest
from scipy import stats
from scipy.integrate import quad
from scipy.optimize import brentq

import oracle as O
from paper_2609_17661_b300 import workloads as W

WQ = 4096          # weight fixed point (w_int = rint(w 2^12))


def _cfg(**over):
    base = dict(inject_mode=O.INJECT_TOPUP, drag_law=O.DRAG_OFF, mc_on=0, pairs_on=0)
    base.update(over)
    return W.config("C1", **base)


class _Geometry:
    """Dipole line r = r_eq sin^2(theta), s from the northern footpoint."""

    def __init__(self, r_eq, n_cells):
        self.r_eq, self.N = r_eq, n_cells
        self.th0 = math.asin(math.sqrt(1.0 / r_eq))
        self.L = 2.0 * self.arc(math.pi / 2)
        self.R_cells = n_cells / self.L

    def arc(self, th):
        f = lambda t: self.r_eq * math.sin(t) * math.sqrt(1.0 + 3.0 * math.cos(t) ** 2)
        return quad(f, self.th0, th, epsabs=1e-12, epsrel=1e-12)[0]

    def at_cell_centre(self, c):
        s = self.L * (c + 0.5) / self.N
        th = brentq(lambda t: self.arc(t) - s, self.th0, math.pi - self.th0, xtol=1e-15)
        ct = math.cos(th)
        return self.r_eq * math.sin(th) ** 2, 2.0 * ct / math.sqrt(1.0 + 3.0 * ct * ct)

    def atmosphere(self, cfg):
        """{cell: (target w_int, mu_s)} over the cells with n/n0 >= n_cut,
        walking in from both footpoints (n falls monotonically with r)."""
        out = {}
        for cells in (range(self.N), range(self.N - 1, -1, -1)):
            for c in cells:
                x, mu = self.at_cell_centre(c)
                n = cfg["atmo_a0"] * math.exp(-(x - 1.0) * self.R_cells / cfg["atmo_h"])
                if n < cfg["atmo_ncut"]:
                    break
                out[c] = (int(math.floor(n * cfg["n0_ppc"] * WQ)), mu)
        return out


@pytest.fixture(scope="module")
def c1():
    cfg = _cfg()
    geo = _Geometry(cfg["r_eq"], cfg["n_cells"])
    return cfg, geo, geo.atmosphere(cfg)


def _cell_weights(p, N):
    cell = np.floor(p["s"]).astype(np.int64)
    wint = np.rint(p["w"] * WQ).astype(np.int64)
    return np.bincount(cell, weights=wint, minlength=N).astype(np.int64)


def test_first_top_up_follows_the_density_profile(c1):
    cfg, geo, atm = c1
    assert 20 < len(atm) < cfg["n_cells"] // 4        # an atmosphere at both ends, not the whole line
    S = O.Sim(cfg)
    S.step(1)
    p = S.particles()
    expect = {c: 2 * (t // (2 * WQ)) for c, (t, _) in atm.items()}
    assert S.diag()["injected"] == sum(expect.values()) > 1000
    got = np.bincount(np.floor(p["s"]).astype(np.int64), minlength=cfg["n_cells"])
    for c in range(cfg["n_cells"]):
        assert got[c] == expect.get(c, 0), c
    # one electron (atmospheric) and one ion per pair, weight 1, the same place
    assert np.sum(p["sp"] == W.SP_ATMO) == np.sum(p["sp"] == W.SP_ION) == len(p["s"]) // 2
    assert np.all(p["w"] == 1.0)
    # ids are the atmosphere's: pair k of cell c at step 0
    c0 = min(atm)
    assert O.atmo_id(0, c0, 0, 0) in set(p["id"].tolist())


def test_every_step_leaves_each_cell_within_one_pair_of_its_target(c1):
    cfg, geo, atm = c1
    S = O.Sim(cfg)
    rng = np.random.default_rng(5)
    N = cfg["n_cells"]
    # a warm state that moves weight between cells (and out of the line)
    n = 4000
    S.set_particles(rng.uniform(0, N, n), rng.normal(0, 0.5, n), np.ones(n),
                    rng.choice([W.SP_ELEC, W.SP_POSI, W.SP_ION], n).astype(np.int32),
                    np.arange(n, dtype=np.uint64))
    inside = np.zeros(N, bool)
    inside[list(atm)] = True
    tgt = np.zeros(N, np.int64)
    for c, (t, _) in atm.items():
        tgt[c] = t
    for step in range(6):
        before = set(S.particles()["id"].tolist())
        S.step(1)
        p = S.particles()
        Wc = _cell_weights(p, N)
        new = np.array([i not in before for i in p["id"].tolist()])
        # new particles (no pairs here) sit in atmosphere cells only
        assert np.all(inside[np.floor(p["s"][new]).astype(np.int64)])
        got_new = np.bincount(np.floor(p["s"][new]).astype(np.int64), minlength=N)
        for c in atm:
            if got_new[c]:
                assert tgt[c] - 2 * WQ < Wc[c] <= tgt[c], (step, c)
            else:
                assert Wc[c] > tgt[c] - 2 * WQ, (step, c)


@pytest.mark.parametrize("sp", [W.SP_ION, W.SP_ELEC])
def test_gravity_is_minus_T_over_h_along_r(c1, sp):
    cfg, geo, atm = c1
    cfg = dict(cfg, j_psi=0.0, cells_per_skin_depth=1e9)   # no external current, no self-field
    N = cfg["n_cells"]
    north = min(atm) + 3
    south = max(atm) - 3
    middle = N // 2
    assert middle not in atm
    S = O.Sim(cfg)
    s0 = np.array([north + 0.5, south + 0.5, middle + 0.5])
    S.set_particles(s0, np.zeros(3), np.ones(3), np.full(3, sp, np.int32), np.arange(3, dtype=np.uint64))
    S.step(1)
    p = S.particles()
    u = {int(i): v for i, v in zip(p["id"], p["u"])}
    m = cfg["mass_ratio"] if sp == W.SP_ION else 1.0
    dt = cfg["cfl"]
    g = cfg["inject_T"] / cfg["atmo_h"]
    for k, c in enumerate((north, south)):
        mu = atm[c][1]
        assert u[k] == pytest.approx(-g * mu * dt / m, rel=1e-12, abs=0.0)
    assert u[0] < 0.0 < u[1]              # both pulled toward the star
    assert u[2] == 0.0


def test_injected_momenta_are_maxwellian_at_T(c1):
    cfg, geo, atm = c1
    cfg = dict(cfg, atmo_a0=4 * cfg["atmo_a0"])   # about 7,000 particles
    S = O.Sim(cfg)
    S.step(1)
    p = S.particles()
    T = cfg["inject_T"]
    for sp, var in ((W.SP_ATMO, T), (W.SP_ION, T / cfg["mass_ratio"])):
        u = p["u"][p["sp"] == sp]
        n = u.size
        assert n > 3000
        assert abs(u.mean()) < 4.0 * math.sqrt(var / n)
        assert abs(u.var() / var - 1.0) < 4.0 * math.sqrt(2.0 / n)
        assert stats.kstest(u / math.sqrt(var), "norm").pvalue > 1e-4
    frac = p["s"] - np.floor(p["s"])
    assert stats.kstest(frac, "uniform").pvalue > 1e-4


def test_no_atmosphere_when_the_cut_is_above_the_surface_density():
    """Degenerate profile: atmo_ncut above atmo_a0 leaves no atmosphere
    cell, so nothing is topped up and there is no gravity anywhere."""
    cfg = _cfg(atmo_ncut=2.0 * 18.0 * 28.0, j_psi=0.0, cells_per_skin_depth=1e9)
    S = O.Sim(cfg)
    N = cfg["n_cells"]
    s0 = np.array([0.5, 3.5, N - 3.5])
    S.set_particles(s0, np.zeros(3), np.ones(3), np.full(3, W.SP_ION, np.int32), np.arange(3, dtype=np.uint64))
    S.step(2)
    assert S.diag()["injected"] == 0
    assert np.all(S.particles()["u"] == 0.0)
