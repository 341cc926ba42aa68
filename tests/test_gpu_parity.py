"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Tolerances (the FP32 path against FP64, stated by the method's targets):
fields and momenta to max relative error 1e-5 (max |difference| over max
|value|); integer currents, counts and ids bit-exact; positions to the
fixed-point quantum plus FP32 rounding of one step's displacement.
Decisions that floating point takes near a threshold (a scattering draw
against p_sc, a pair against 2 m_e c^2, a limiter branch) may differ when the
oracle's margin is below FP32 rounding; the inputs here are chosen so that
no decision sits that close, and the tests report any that does.
"""
import math

import numpy as np
import pytest

import oracle as O
from paper_2609_17661_b300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

RTOL = 1e-5


def _line(cfg):
    from paper_2609_17661_b300 import Line
    return Line(cfg)


def _by_id(p):
    o = np.argsort(p["id"])
    return {k: v[o] for k, v in p.items()}


def _gpu_particles(line, N):
    g = _by_id(line.particles())
    F = W.fbits(N)
    g["s"] = g["pos"].astype(np.float64) / float(1 << F)
    return g


def _orc(cfg, st, E=None, step=0):
    S = O.Sim(cfg)
    o = W.to_oracle(st, cfg["n_cells"])
    S.set_particles(o["s"], o["u"], o["w"], o["sp"], o["id"])
    if E is not None:
        S.set_field(E)
    S.set_step(step)
    return S


def _relmax(a, b):
    return np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300)


def _compare_particles(g, o, N, steps=1, pos_tol=None):
    assert g["id"].tolist() == o["id"].tolist(), "different particle sets"
    assert np.array_equal(g["sp"].astype(np.int32), o["sp"])
    assert _relmax(g["u"].astype(np.float64), o["u"]) <= RTOL
    F = W.fbits(N)
    if pos_tol is None:
        pos_tol = steps * (2.0 ** -F + 1e-6)
    assert np.max(np.abs(g["s"] - o["s"])) <= pos_tol


def _field0(N, amp=0.02, seed=3):
    rng = np.random.default_rng(seed)
    x = (np.arange(N) + 0.5) / N
    return amp * (np.sin(2 * np.pi * 3 * x) + 0.3 * np.cos(2 * np.pi * 7 * x + 1.0)) + 0.002 * rng.standard_normal(N)


# ------------------------------------------------------------------ pieces
def test_table_matches_oracle():
    """The device quadrature table (FP64 on the GPU, stored FP32) equals the
    oracle's FP64 table entry by entry."""
    cfg = W.config("C1", table_n_gamma=64, table_n_s=32, quad_n_mu=24, quad_n_phi=24)
    line = _line(cfg)
    g = line.table().astype(np.float64).reshape(2, 32, 64, 2)
    o = O.build_table(cfg).reshape(2, 32, 64, 2)
    # stored in FP32: relative rounding, values below FP32's normal range flush,
    # and entries near the drag's zero crossing (the attractor) carry the FP64
    # cancellation error of the disk sum, bounded by its row's scale
    tiny = 2.0 ** -126
    row = np.max(np.abs(o[..., 0]), axis=2, keepdims=True)
    err = np.abs(g[..., 0] - o[..., 0])
    bound = 1e-6 * np.abs(o[..., 0]) + 1e-12 * row + tiny
    bad = np.argwhere(err > bound)
    assert bad.size == 0, [(tuple(b), g[tuple(b)][0], o[tuple(b)][0]) for b in bad[:8]]
    assert np.max(np.abs(g[..., 1] - o[..., 1])) <= 1e-4
    for model in (O.PHOTON_RADIAL,):
        c2 = dict(cfg, photon_model=model)
        g2 = _line(c2).table().astype(np.float64).reshape(2, 32, 64, 2)
        o2 = O.build_table(c2).reshape(2, 32, 64, 2)
        row2 = np.max(np.abs(o2[..., 0]), axis=2, keepdims=True)
        assert np.all(np.abs(g2[..., 0] - o2[..., 0]) <= 1e-6 * np.abs(o2[..., 0]) + 1e-12 * row2 + tiny)


def test_integer_deposit_bit_exact():
    """pic1d_deposit equals the oracle's integer deposit, including paths
    clamped at both walls and zero-length paths."""
    N = 256
    F = W.fbits(N)
    cfg = W.config("C1", n_cells=N)
    line = _line(cfg)
    rng = np.random.default_rng(5)
    n = 200000
    p0 = rng.integers(0, N << F, n).astype(np.int64)
    step = rng.integers(-int(0.45 * (1 << F)), int(0.45 * (1 << F)), n)
    step[:1000] = 0
    p1 = p0 + step
    w = rng.choice(np.array([1.0, 0.5, 3.25, 1e-3], np.float32), n)
    sp = rng.integers(0, 4, n).astype(np.uint8)
    J = torch.zeros(N, dtype=torch.int64, device="cuda")
    line.deposit(torch.from_numpy(p0).cuda(), torch.from_numpy(p1).cuda(), torch.from_numpy(w).cuda(),
                 torch.from_numpy(sp).cuda(), J)
    ref = O.deposit_int(N, F, p0, p1, w.astype(np.float64), sp.astype(np.int32))
    assert np.array_equal(J.cpu().numpy(), ref)
    assert (p1 < 0).any() and (p1 >= (N << F)).any()


# --------------------------------------------------------- one-step parity
@pytest.mark.parametrize("drag_law", [O.DRAG_TABLE, O.DRAG_CLOSED])
def test_one_step_parity_drag_limiter(drag_law):
    """One step from an identical state with continuous drag on the whole
    line, limiter on (damping and Newton branches both taken)."""
    N = 1024
    cfg = W.config("C1", drag_law=drag_law, b_pair_threshold=1e30, mc_on=0, pairs_on=0, eta_min=1.0,
                   drag_scale=1e-3)
    st = W.load_random(cfg, 60000, u_scale=300.0, seed=21)
    E = _field0(N)
    line = _line(cfg)
    line.set_state(st, E=E)
    line.step(1)
    S = _orc(cfg, st, E)
    S.step(1)
    g = _gpu_particles(line, N)
    o = _by_id(S.particles())
    _compare_particles(g, o, N)
    Eg, Jg = line.fields()
    Eo, Jo = S.fields()
    assert _relmax(Eg, Eo) <= RTOL
    dg, do = line.diag(), S.diag()
    assert dg["n_alive"] == do["n_alive"]
    assert dg["lost_north"] == do["lost_north"] and dg["lost_south"] == do["lost_south"]
    assert dg["limiter_branch"] > 1000 and dg["newton_branch"] > 1000
    assert abs(dg["limiter_branch"] - do["limiter_branch"]) <= 2
    assert dg["kinetic_energy"] == pytest.approx(do["kinetic_energy"], rel=1e-5)


def test_one_step_parity_scattering_and_pairs():
    """One step of energetic leptons in the pair zone: the same scatterings,
    recoils and pairs (ids, positions, momenta)."""
    N = 1024
    cfg = W.config("C1", drag_law=O.DRAG_TABLE, drag_scale=3e-3)
    st = W.load_beam(cfg, 40000, gamma_lo=20, gamma_hi=2e4, seed=8)
    E = _field0(N)
    line = _line(cfg)
    line.set_state(st, E=E, step=17)
    line.step(1)
    S = _orc(cfg, st, E, step=17)
    S.step(1)
    dg, do = line.diag(), S.diag()
    assert do["scatters"] > 1000 and do["pairs_created"] > 500
    assert dg["scatters"] == do["scatters"]
    assert dg["pairs_created"] == do["pairs_created"]
    assert dg["psc_clamped"] == do["psc_clamped"]
    g = _gpu_particles(line, N)
    o = _by_id(S.particles())
    _compare_particles(g, o, N)
    Eg, _ = line.fields()
    Eo, _ = S.fields()
    assert _relmax(Eg, Eo) <= RTOL


def test_pair_cap_parity_over_steps():
    """The n_max cap: a pair is refused where the cell's lepton weight at the
    start of the step has reached n_max (integer fixed point).  The cap is set
    at the median cell weight so that about half the zone refuses; over three
    steps the weight of the created pairs feeds the next step's test.  The
    same pairs are created and refused, particle by particle."""
    N = 1024
    F = W.fbits(N)
    st = W.load_beam(W.config("C1"), 40000, gamma_lo=20, gamma_hi=2e4, seed=8)
    lep = (st["sp"] == 0) | (st["sp"] == 1)
    wint = np.rint(st["w"].astype(np.float64) * 4096).astype(np.int64)
    dens = np.bincount(np.minimum(st["pos"][lep].astype(np.int64) >> F, N - 1), weights=wint[lep], minlength=N)
    med = int(np.median(dens[dens > 0]))
    cfg = W.config("C1", drag_law=O.DRAG_TABLE, drag_scale=3e-3, n_max_ppc=(med + 0.5) / 4096.0)
    E = _field0(N)
    line = _line(cfg)
    line.set_state(st, E=E, step=17)
    line.step(3)
    S = _orc(cfg, st, E, step=17)
    S.step(3)
    dg, do = line.diag(), S.diag()
    assert do["pairs_rejected_nmax"] > 100 and do["pairs_created"] > 100
    for k in ("pairs_created", "pairs_rejected_nmax", "scatters", "n_alive"):
        assert dg[k] == do[k], k
    # positions over three steps: per step the fixed-point quantum plus the
    # displacement of a velocity that differs by the momentum tolerance (dt RTOL)
    pos_tol = 3 * (2.0 ** -F + cfg["cfl"] * RTOL)
    _compare_particles(_gpu_particles(line, N), _by_id(S.particles()), N, pos_tol=pos_tol)
    Eg, _ = line.fields()
    Eo, _ = S.fields()
    assert _relmax(Eg, Eo) <= RTOL


def test_drag_plus_pairs_mode_parity():
    N = 1024
    cfg = W.config("C1", drag_law=O.DRAG_TABLE, drag_scale=3e-3, rics_mode=O.RICS_DRAG_PLUS_PAIRS, eta_min=1e-2)
    st = W.load_beam(cfg, 20000, gamma_lo=20, gamma_hi=2e4, seed=9)
    line = _line(cfg)
    line.set_state(st, E=_field0(N))
    line.step(1)
    S = _orc(cfg, st, _field0(N))
    S.step(1)
    assert line.diag()["pairs_created"] == S.diag()["pairs_created"] > 100
    _compare_particles(_gpu_particles(line, N), _by_id(S.particles()), N)


def test_injection_parity():
    """RATE supply: the same injected particles (ids, positions, momenta)."""
    N = 4096
    cfg = W.config("C1", n_cells=N, inject_mode=O.INJECT_RATE, drag_law=0, mc_on=0, pairs_on=0)
    st = W.load_random(cfg, 5000, seed=2)
    line = _line(cfg)
    line.set_state(st, step=5)
    line.step(3)
    S = _orc(cfg, st, step=5)
    S.step(3)
    assert line.diag()["injected"] == S.diag()["injected"] > 0
    _compare_particles(_gpu_particles(line, N), _by_id(S.particles()), N, steps=3)


# ------------------------------------------------------ multi-step parity
def test_thousand_steps_parity_non_chaotic():
    """1000 steps, drag (implicit midpoint, no limiter) and Lorentz force in
    a static nonuniform E on a line with a negligible self-field (the regime
    where FP32 and FP64 can agree for long: no plasma instability amplifies
    rounding): fields and momenta to 1e-5 max relative."""
    N = 4096
    cfg = W.config("C1", n_cells=N, drag_law=O.DRAG_TABLE, b_pair_threshold=1e30, mc_on=0, pairs_on=0,
                   eta_min=0.0, drag_scale=1e-4, cells_per_skin_depth=1e6)
    st = W.load_random(cfg, 20000, u_scale=100.0, seed=4)
    F = W.fbits(N)
    keep = (st["pos"] > (1500 << F)) & (st["pos"] < (2600 << F))
    st = {k: v[keep] for k, v in st.items()}
    E = 0.02 * np.sin(2 * np.pi * 3 * (np.arange(N) + 0.5) / N) + 0.01
    line = _line(cfg)
    line.set_state(st, E=E)
    line.step(1000)
    S = _orc(cfg, st, E)
    S.step(1000)
    g = _gpu_particles(line, N)
    o = _by_id(S.particles())
    assert g["id"].size == st["id"].size
    # positions: relative to the line (a momentum error of 1e-5 max|u| moves a
    # slow particle by up to ~1e-5 max|u| dt per step)
    _compare_particles(g, o, N, pos_tol=RTOL * N)
    assert _relmax(g["s"], o["s"]) <= RTOL
    Eg, _ = line.fields()
    Eo, _ = S.fields()
    assert _relmax(Eg, Eo) <= RTOL
    assert line.diag()["newton_branch"] > 1e6


def test_c1_parity_over_the_predictable_horizon():
    """C1 (pairs off) is a chaotic plasma: the oracle against itself with
    1e-7 perturbed momenta departs by ~1e-6 in E after ~150 steps and by
    ~2% after 1000.  Over 100 steps the GPU stays within 1e-5 of the oracle."""
    cfg = W.config("C1", pairs_on=0)
    st = W.load_drifting_plasma(cfg)
    line = _line(cfg)
    line.set_state(st)
    line.step(100)
    S = _orc(cfg, st)
    S.step(100)
    Eg, _ = line.fields()
    Eo, _ = S.fields()
    assert _relmax(Eg, Eo) <= RTOL
    g = _gpu_particles(line, cfg["n_cells"])
    o = _by_id(S.particles())
    assert g["id"].tolist() == o["id"].tolist()
    assert _relmax(g["u"].astype(np.float64), o["u"]) <= RTOL


# ------------------------------------------------------ exact properties
def _rho_int(pos, w, sp, N, F):
    one = 1 << F
    q = np.array([-1, 1, 1, -1], np.int64)[sp.astype(np.int64)] * np.rint(w.astype(np.float64) * 4096).astype(np.int64)
    i = np.minimum(pos.astype(np.int64) >> F, N - 1)
    f = pos.astype(np.int64) - (i << F)
    r = np.zeros(N + 1, np.int64)
    np.add.at(r, i, q * (one - f))
    np.add.at(r, i + 1, q * f)
    return r


def test_push_current_equals_the_integer_deposit_of_its_paths():
    """G3: the int64 current the push deposits equals, in every cell (the
    wall cells included), the oracle's integer deposit of the same step's
    paths (old to new fixed-point position; a particle that leaves the line
    ends at its wall): the C1 plasma with beams in the end cells that leave
    through both walls, one step from the loaded state and one more after a
    cell sort (the push's flushes on the sorted layout)."""
    from deposit_ref import step_current
    cfg = W.config("C1")
    N = cfg["n_cells"]
    st = W.load_drifting_plasma(cfg)
    beam = W.load_beam(cfg, 4000, gamma_lo=3.0, gamma_hi=3e3, seed=12, cells=[0, 1, N - 2, N - 1])
    beam["id"] += 10**7
    st = {k: np.concatenate([st[k], beam[k]]) for k in st}
    line = _line(cfg)
    line.set_state(st, E=_field0(N))
    line.step(1)
    after = line.particles(alive_only=False)
    _, J = line.fields()
    np.testing.assert_array_equal(J, step_current(st, after, N))
    d = line.diag()
    assert d["lost_north"] > 0 and d["lost_south"] > 0 and d["pairs_created"] > 0
    line.sort()
    before = line.particles(alive_only=False)
    line.step(1)
    after = line.particles(alive_only=False)
    _, J = line.fields()
    np.testing.assert_array_equal(J, step_current(before, after, N))


@pytest.mark.parametrize("variant", [0, 5, 6, 7])
def test_streaming_push_equals_the_per_thread_push(variant):
    """The streaming push (variants 0, 6, 7: chunks staged in shared memory by
    the bulk-copy engine, damping-certainty flags, two-anchor current windows
    flushed per warp or per lane) and the per-thread push with the same two
    changes (variant 5) run the same FP32 arithmetic per particle as the
    per-thread push (variant 1): positions, momenta, ids, species, the
    integer current and every count are identical after 25 steps with
    scattering, pairs, the pair cap, the limiter (both branches), losses at
    both walls and a sort."""
    cfg = W.config("C1", n_max_ppc=40.0, sort_every=10, rics_mode=O.RICS_DRAG_PLUS_PAIRS, capacity=400_000)
    N = cfg["n_cells"]
    st = W.load_drifting_plasma(cfg)
    beam = W.load_beam(cfg, 6000, gamma_lo=2.0, gamma_hi=3e4, seed=13)
    beam["id"] += 10**7
    st = {k: np.concatenate([st[k], beam[k]]) for k in st}
    out = []
    for v in (variant, 1):
        line = _line(cfg)
        line.set_variant(v)
        line.set_state(st, E=_field0(N))
        line.step(25)
        out.append((_by_id(line.particles()), line.fields(), line.diag()))
        line.close()
    (p0, (E0, J0), d0), (p1, (E1, J1), d1) = out
    # with the capacity reached, which pairs are dropped would depend on the append order
    assert d0["pairs_dropped_cap"] == 0 and d1["pairs_dropped_cap"] == 0
    for k in ("id", "pos", "u", "w", "sp"):
        np.testing.assert_array_equal(p0[k], p1[k], err_msg=k)
    np.testing.assert_array_equal(J0, J1)
    np.testing.assert_array_equal(E0, E1)
    for k in ("n_alive", "pairs_created", "pairs_rejected_nmax", "scatters", "limiter_branch", "newton_branch",
              "lost_north", "lost_south", "rng_draws"):
        assert d0[k] == d1[k], (k, d0[k], d1[k])
    assert d0["limiter_branch"] > 0 and d0["newton_branch"] > 0 and d0["pairs_created"] > 0
    assert d0["lost_north"] > 0 and d0["lost_south"] > 0 and d0["pairs_rejected_nmax"] > 0
    assert d0["kinetic_energy"] == pytest.approx(d1["kinetic_energy"], rel=1e-6)


def test_table_law_instantiation_equals_the_per_thread_push():
    """On a line with the paper's setup (table law with the limiter, split
    RICS: continuous drag outside the pair zones, Monte-Carlo scattering and
    pairs inside them) the streaming push runs its instantiation with those
    switches as constants; its particles, integer current, field and counts
    equal the per-thread push's (variant 1, which tests them per particle)
    after 25 steps with both drag branches, scattering, pairs, the pair cap,
    losses at both walls and two sorts."""
    cfg = W.config("C1", n_max_ppc=40.0, sort_every=10, rics_mode=O.RICS_SPLIT, b_pair_threshold=0.3,
                   capacity=400_000)
    N = cfg["n_cells"]
    st = W.load_drifting_plasma(cfg)
    beam = W.load_beam(cfg, 6000, gamma_lo=2.0, gamma_hi=3e4, seed=13)
    beam["id"] += 10**7
    st = {k: np.concatenate([st[k], beam[k]]) for k in st}
    out = []
    for v in (0, 1):
        line = _line(cfg)
        line.set_variant(v)
        line.set_state(st, E=_field0(N))
        line.step(25)
        out.append((_by_id(line.particles()), line.fields(), line.diag()))
        line.close()
    (p0, (E0, J0), d0), (p1, (E1, J1), d1) = out
    assert d0["pairs_dropped_cap"] == 0 and d1["pairs_dropped_cap"] == 0
    for k in ("id", "pos", "u", "w", "sp"):
        np.testing.assert_array_equal(p0[k], p1[k], err_msg=k)
    np.testing.assert_array_equal(J0, J1)
    np.testing.assert_array_equal(E0, E1)
    for k in ("n_alive", "pairs_created", "pairs_rejected_nmax", "scatters", "limiter_branch", "newton_branch",
              "lost_north", "lost_south", "rng_draws"):
        assert d0[k] == d1[k], (k, d0[k], d1[k])
    assert d0["limiter_branch"] > 0 and d0["newton_branch"] > 0 and d0["pairs_created"] > 0
    assert d0["scatters"] > 0 and d0["pairs_rejected_nmax"] > 0
    assert d0["lost_north"] > 0 and d0["lost_south"] > 0


def test_gauss_law_integer_exact_every_step():
    """Discrete charge continuity in integers: rho(n+1) - rho(n) = -(J_i -
    J_{i-1}) at every interior node for every step, with J_int the step's own
    current, while drag, scattering, pairs and losses all act (pairs are
    created neutral, removed particles leave through the walls)."""
    N = 512
    F = W.fbits(N)
    cfg = W.config("C1", n_cells=N, drag_scale=3e-4, sort_every=3)
    st = W.load_drifting_plasma(cfg)
    beam = W.load_beam(cfg, 4000, gamma_lo=30, gamma_hi=3e3, seed=4)
    beam["id"] += 10**7
    st = {k: np.concatenate([st[k], beam[k]]) for k in st}
    line = _line(cfg)
    line.set_state(st, E=_field0(N))
    for k in range(12):
        p0 = line.particles()
        r0 = _rho_int(p0["pos"], p0["w"], p0["sp"], N, F)
        line.step(1)
        _, J = line.fields()
        p1 = line.particles()
        r1 = _rho_int(p1["pos"], p1["w"], p1["sp"], N, F)
        np.testing.assert_array_equal((r1 - r0)[1:N], -(J[1:N] - J[0:N - 1]))
    d = line.diag()
    assert d["pairs_created"] > 0 and d["lost_north"] + d["lost_south"] > 0


def test_device_rho_and_gauss_law_on_the_device():
    """pic1d_get_rho equals the node charge summed on the host from the
    particles, and the device rho and J obey the discrete Gauss law exactly
    step by step."""
    N = 512
    F = W.fbits(N)
    cfg = W.config("C1", n_cells=N, drag_scale=3e-4, sort_every=3)
    st = W.load_drifting_plasma(cfg)
    line = _line(cfg)
    line.set_state(st, E=_field0(N))
    r0 = line.rho()
    p = line.particles()
    np.testing.assert_array_equal(r0, _rho_int(p["pos"], p["w"], p["sp"], N, F))
    for k in range(6):
        line.step(1)
        r1 = line.rho()
        _, J = line.fields()
        np.testing.assert_array_equal((r1 - r0)[1:N], -(J[1:N] - J[0:N - 1]))
        r0 = r1


def test_current_invariant_under_permutation_and_sort_cadence():
    """J_int is an exact integer sum: identical under any storage order of
    the particles and any sort cadence."""
    N = 1024
    cfg = W.config("C1", drag_scale=1e-3)
    st = W.load_drifting_plasma(cfg)
    Js = []
    for perm_seed, sort_every in ((None, 20), (1, 20), (2, 1), (3, 7)):
        s2 = st
        if perm_seed is not None:
            p = np.random.default_rng(perm_seed).permutation(st["pos"].size)
            s2 = {k: v[p] for k, v in st.items()}
        line = _line(dict(cfg, sort_every=sort_every))
        line.set_state(s2, E=_field0(N))
        line.step(5)
        E, J = line.fields()
        Js.append((E, J))
    for E, J in Js[1:]:
        np.testing.assert_array_equal(J, Js[0][1])
        np.testing.assert_array_equal(E, Js[0][0])


def test_counts_exact_one_step():
    N = 1024
    cfg = W.config("C1", drag_scale=3e-4)
    st = W.load_drifting_plasma(cfg)
    beam = W.load_beam(cfg, 8000, gamma_lo=50, gamma_hi=5e3, seed=12)
    beam["id"] += 10**7
    st = {k: np.concatenate([st[k], beam[k]]) for k in st}
    line = _line(cfg)
    line.set_state(st, E=_field0(N))
    line.step(1)
    S = _orc(cfg, st, _field0(N))
    S.step(1)
    dg, do = line.diag(), S.diag()
    for k in ("n_alive", "pairs_created", "lost_north", "lost_south", "scatters"):
        assert dg[k] == do[k], k


# ------------------------------------------------------------ statistics
@pytest.mark.slow
def test_pair_yield_32_seeds_within_3_sigma():
    """Stochastic pair yield of a C1 line seeded with an energetic beam,
    200 steps, 32 seeds: mean over seeds of the GPU within 3 sigma of the
    oracle's."""
    N = 1024
    base = W.config("C1", drag_scale=1e-4)
    st0 = W.load_drifting_plasma(base)
    gy, oy = [], []
    for seed in range(1, 33):
        cfg = dict(base, seed=seed)
        beam = W.load_beam(cfg, 2000, gamma_lo=30, gamma_hi=3e3, seed=100 + seed)
        beam["id"] += 10**7
        st = {k: np.concatenate([st0[k], beam[k]]) for k in st0}
        line = _line(cfg)
        line.set_state(st)
        line.step(200)
        gy.append(line.diag()["pairs_created"])
        S = _orc(cfg, st)
        S.step(200)
        oy.append(S.diag()["pairs_created"])
    gy, oy = np.array(gy, float), np.array(oy, float)
    assert oy.mean() > 50
    sig = math.sqrt(gy.var(ddof=1) / 32 + oy.var(ddof=1) / 32)
    assert abs(gy.mean() - oy.mean()) <= 3 * sig + 1e-9


# ------------------------------------------------------------ edge cases
def test_empty_line_and_tiny_line():
    for N in (8, 1024):
        cfg = W.config("C1", n_cells=N, inject_mode=O.INJECT_RATE)
        line = _line(cfg)
        line.set_state(W.empty_state(0))
        line.step(4)
        S = _orc(cfg, W.empty_state(0))
        S.step(4)
        d = line.diag()
        assert d["injected"] == S.diag()["injected"]
        Eg, _ = line.fields()
        Eo, _ = S.fields()
        assert _relmax(Eg, Eo) <= RTOL


def test_ragged_tail_and_removed_slots():
    """Particle counts that are not a multiple of the tile, with removed
    slots in the middle of the array, and a sort that compacts them."""
    N = 1024
    cfg = W.config("C1", sort_every=1000)
    for n in (1, 3, 1023, 1025, 4099):
        st = W.load_random(cfg, n, u_scale=5.0, seed=n)
        st["sp"][::7] = 255
        line = _line(cfg)
        line.set_state(st, E=_field0(N))
        line.step(2)
        alive = {k: v[st["sp"] != 255] for k, v in st.items()}
        S = _orc(cfg, alive, _field0(N))
        S.step(2)
        g, o = _gpu_particles(line, N), _by_id(S.particles())
        if o["id"].size:
            _compare_particles(g, o, N, steps=2)
        else:
            assert g["id"].size == 0
        line.sort()
        assert line.slots() == sum(line.diag()["n_alive"])


def test_capacity_overflow_warns_and_stays_consistent():
    N = 512
    F = W.fbits(N)
    cfg = W.config("C1", n_cells=N, drag_scale=1e-2)
    st = W.load_beam(cfg, 3000, gamma_lo=100, gamma_hi=1e4, seed=3)
    cfg = dict(cfg, capacity=3000 + 64)
    line = _line(cfg)
    line.set_state(st)
    p0 = line.particles()
    line.step(1)
    d = line.diag()
    assert d["rc"] == 1 and d["pairs_dropped_cap"] > 0
    assert d["n_slots"] <= cfg["capacity"]
    p1 = line.particles()
    _, J = line.fields()
    r0 = _rho_int(p0["pos"], p0["w"], p0["sp"], N, F)
    r1 = _rho_int(p1["pos"], p1["w"], p1["sp"], N, F)
    np.testing.assert_array_equal((r1 - r0)[1:N], -(J[1:N] - J[0:N - 1]))


def test_nonfinite_momentum_reported():
    """A non-finite momentum in the input is caught by the step: the particle
    is removed and pic1d_diag returns PIC1D_ENUMERIC."""
    cfg = W.config("C1", n_cells=64, mc_on=0, pairs_on=0)
    st = W.load_random(cfg, 100, seed=1)
    st["u"][10] = np.nan
    line = _line(cfg)
    line.set_state(st)
    line.step(1)
    d = line.diag()
    assert d["rc"] == -4 and d["nonfinite"] == 1
    assert sum(d["n_alive"]) == 99


def test_invalid_state_rejected():
    """Bad species or positions beyond the line are refused, from host and
    from device arrays alike, and the refused call leaves an empty line."""
    from paper_2609_17661_b300 import PicError
    cfg = W.config("C1", n_cells=100)
    st = W.load_random(cfg, 10, seed=1)
    st["sp"][3] = 9
    line = _line(cfg)
    with pytest.raises(PicError):
        line.set_state(st)
    st = W.load_random(cfg, 10, seed=1)
    st["pos"][2] = 0xFFFFFFF0           # beyond 100 cells * 2^25
    with pytest.raises(PicError):
        line.set_state(st)
    dev = {k: torch.from_numpy(v).cuda() for k, v in st.items()}
    with pytest.raises(PicError):
        line.set_state(dev)
    assert line.slots() == 0 and sum(line.diag()["n_alive"]) == 0
    good = {k: torch.from_numpy(v).cuda() for k, v in W.load_random(cfg, 10, seed=2).items()}
    line.set_state(good)
    assert line.slots() == 10


def test_a_device_wait_that_gives_up_is_reported_and_the_line_goes_on():
    """A bounded device wait on a barrier that nothing completes (no copy in
    flight) gives up after its limit; the next pic1d_diag returns
    PIC1D_ETIMEOUT once, and the line then steps on with correct results."""
    cfg = W.config("C1", pairs_on=0)
    st = W.load_drifting_plasma(cfg)
    line = _line(cfg)
    line.set_state(st)
    assert line.diag()["rc"] == 0
    line.check_wait(2_000_000)            # about a millisecond of SM clocks
    d = line.diag()
    assert d["rc"] == -5                  # PIC1D_ETIMEOUT
    assert line.diag()["rc"] == 0         # reported once
    line.step(5)
    S = _orc(cfg, st)
    S.step(5)
    Eg, _ = line.fields()
    Eo, _ = S.fields()
    assert _relmax(Eg, Eo) <= RTOL
    assert line.diag()["rc"] == 0


def test_degenerate_particles_match_the_oracle():
    """Particles on the degenerate points of the method, two steps against
    the oracle particle by particle, and the push's J of the first step
    against the integer deposit of their paths: exactly on the wall nodes
    moving out and in, on interior nodes and cell centres, one quantum inside
    the line's ends, u = 0 and -0, |u| tiny and beyond the table's top
    (gamma > 10^G, the clamped lookup), every species, weights 0.5 .. 2;
    inside a random plasma so that the field is not trivial."""
    from deposit_ref import step_current
    cfg = W.config("C1", capacity=200000)
    N = cfg["n_cells"]
    F = W.fbits(N)
    top = N << F
    cell = 1 << F
    positions = [0, 1, cell - 1, cell, cell + cell // 2, (N // 2) * cell, (N // 2) * cell - 1, top - cell,
                 top - cell // 2, top - 2, top - 1]
    momenta = [0.0, -0.0, 1e-30, -1e-30, 0.3, -0.3, 30.0, -30.0, 3e3, -3e3, 1e9, -1e9]
    combos = [(p, u, s) for p in positions for u in momenta for s in (W.SP_ELEC, W.SP_POSI, W.SP_ION, W.SP_ATMO)]
    edge = W.empty_state(len(combos))
    edge["pos"][:] = np.array([c[0] for c in combos], np.uint32)
    edge["u"][:] = np.array([c[1] for c in combos], np.float32)
    edge["sp"][:] = np.array([c[2] for c in combos], np.uint8)
    edge["w"][:] = np.resize(np.array([0.5, 1.0, 2.0], np.float32), len(combos))
    edge["id"][:] = np.arange(len(combos), dtype=np.uint64) + 10**8
    bg = W.load_random(cfg, 4000, u_scale=10.0, seed=31)
    st = {k: np.concatenate([edge[k], bg[k]]) for k in edge}
    line = _line(cfg)
    E = _field0(N)
    line.set_state(st, E=E)
    line.step(1)
    after = line.particles(alive_only=False)
    _, J = line.fields()
    np.testing.assert_array_equal(J, step_current(st, after, N))
    line.step(1)
    S = _orc(cfg, st, E)
    S.step(2)
    dg, do = line.diag(), S.diag()
    for k in ("n_alive", "lost_north", "lost_south", "pairs_created", "scatters", "limiter_branch", "newton_branch"):
        assert dg[k] == do[k], (k, dg[k], do[k])
    g, o = _gpu_particles(line, N), _by_id(S.particles())
    assert g["id"].tolist() == o["id"].tolist()
    assert np.array_equal(g["sp"].astype(np.int32), o["sp"])
    # FP32 momenta agree to 1e-5 of the largest momentum in their arithmetic:
    # a particle's own |u| before and after, and for a pair child its
    # parent's |u| at the start of the step that made it (a scattering from
    # u = 3000 down to u ~ 90 cancels four digits)
    S1 = _orc(cfg, st, E)
    S1.step(1)
    p1 = S1.particles()
    scale_of = {}
    for step, (ids, us) in enumerate(((st["id"], st["u"]), (p1["id"], p1["u"]))):
        for i, u in zip(ids.tolist(), np.abs(us.astype(np.float64)).tolist()):
            scale_of[i] = max(scale_of.get(i, 0.0), u)
            for m in (0, 1):
                c = O.child_id(i, step, m)
                scale_of[c] = max(scale_of.get(c, 0.0), u)
    scale = np.array([max(scale_of.get(int(i), 0.0), abs(u)) for i, u in zip(o["id"].tolist(), o["u"].tolist())])
    err = np.abs(g["u"].astype(np.float64) - o["u"])
    tol = 1e-5 * scale + 1e-6
    assert np.all(err <= tol), float(np.max(err / tol))
    assert np.max(np.abs(g["s"] - o["s"])) <= 2 * (2.0 ** -F + 1e-6)
    assert dg["lost_north"] > 0 and dg["lost_south"] > 0
