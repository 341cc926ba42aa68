"""Pins of the oracle's test-particle drag map (the paper's appendix on the
extent of the pair-producing region): a free particle, an independent stiff
ODE solver (scipy's Radau), and the structure the paper describes."""
import math

import numpy as np
import pytest

import oracle as O
from paper_2609_17661_b300 import workloads as W

CFG = W.config("C1", kT_keV=1.0, photon_model=O.PHOTON_RADIAL, drag_scale=1.0)


def test_free_particle_reaches_the_equator_unchanged():
    d = O.tp_line(dict(CFG, drag_scale=0.0), 6.0, gamma0=100.0, dt=1e-3, t_max=1e3)
    assert d["gamma_min"] == pytest.approx(100.0, rel=1e-14)
    assert d["theta_first"] == -1.0 and d["l_pp"] == 0.0
    beta = math.sqrt(1 - 1e-4)
    assert d["t_end"] == pytest.approx(0.5 * d["L"] / beta, rel=2e-3)


def _radau(r_eq, gamma0=1000.0, t_max=60.0):
    """The same ODE -- du/dt = F(u, theta), dtheta/dt = beta/(ds/dtheta),
    dtau/dt = N -- by scipy's Radau at tight tolerance."""
    from scipy.integrate import solve_ivp
    cfg = dict(CFG, r_eq=r_eq)

    def rhs(t, y):
        u, th, tau = y
        x, b, mu = O.field_at_theta(cfg, th)
        F, N = O.photon(cfg, u, x, b, mu, model=O.PHOTON_RADIAL)
        c = math.cos(th)
        return [F, u / math.sqrt(1 + u * u) / (r_eq * math.sin(th) * math.sqrt(1 + 3 * c * c)), N]

    def eq(t, y):
        return y[1] - 0.5 * math.pi
    eq.terminal = True

    def first(t, y):
        return y[2] - 1.0

    y0 = [math.sqrt(gamma0 ** 2 - 1), O.theta0(r_eq), 0.0]
    sol = solve_ivp(rhs, (0, t_max), y0, method="Radau", rtol=1e-10, atol=[1e-9, 1e-12, 1e-12],
                    events=(eq, first), dense_output=True)
    ts = np.linspace(0, sol.t[-1], 20001)
    gmin = np.min(np.sqrt(1 + sol.sol(ts)[0] ** 2))
    th_first = sol.y_events[1][0][1] if len(sol.y_events[1]) else -1.0
    return gmin, th_first


def test_map_converges_to_a_stiff_solver():
    """A region-II line: gamma_min and the first-scattering point agree with
    Radau, with an error that falls as dt does."""
    g_ref, th_ref = _radau(6.0)
    errs = []
    for dt in (4e-3, 1e-3):
        d = O.tp_line(CFG, 6.0, dt=dt, t_max=60.0)
        errs.append((abs(d["gamma_min"] - g_ref) / g_ref, abs(d["theta_first"] - th_ref)))
    assert errs[1][0] < errs[0][0] and errs[1][1] < errs[0][1]
    assert errs[1][0] < 2e-3 and errs[1][1] < 2e-3


def test_regions_follow_the_papers_structure():
    """Short lines keep b > 0.1 to the equator (region I), then b falls below
    0.1 with gamma_min > 1 (II), and beyond the critical radius the leptons
    come to rest (III, gamma_min ~ 1); the pair zone of the long lines is
    about 2 R* (the paper's l_pp -> 2)."""
    rs = [2.2, 3.0, 4.0, 5.0, 6.0, 8.0, 12.0, 20.0, 30.0]
    ds = [O.tp_line(CFG, r, dt=2e-3, t_max=80.0) for r in rs]
    regions = [int(d["region"]) for d in ds]
    assert regions == sorted(regions) and regions[0] == 1 and regions[-1] == 3 and 2 in regions
    beq = [d["b_eq"] for d in ds]
    assert all(a > b for a, b in zip(beq, beq[1:]))
    for d, r in zip(ds, rs):
        if d["b_eq"] < 0.1:
            x, b, mu = O.field_at_theta(dict(CFG, r_eq=r), d["theta_b"])
            assert b == pytest.approx(0.1, rel=1e-9)
    for d, r in zip(ds, rs):
        if r >= 20.0:
            assert 1.0 < d["l_pp"] < 3.0
