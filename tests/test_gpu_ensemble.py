"""The ensemble engine (many lines per launch, captured super-steps,
autotuned schedule) against the same lines advanced one by one by the
single-line engine (itself checked against the FP64 oracle): per line the
results must be identical -- the per-particle arithmetic does not depend on
which other particles share a tile, the current is an exact integer sum and
the field update is the same FP64 expression."""
import numpy as np
import pytest

from paper_2609_17661_b300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _cfgs():
    cfgs = []
    for k, (r, N, n) in enumerate([(3.0, 512, 20000), (8.0, 1024, 50000), (20.0, 2048, 8000),
                                   (30.0, 1536, 120000), (5.0, 640, 3000)]):
        cfgs.append(W.config("C1", r_eq=r, n_cells=N, drag_law=W.DRAG_SURROGATE, n0_ppc=n / N / 140.0,
                             j_psi=28.0 * (0.3 + 0.15 * k), capacity=4 * n + 65536, seed=1 + k,
                             sort_every=20, drag_scale=0.05))
    states = [W.load_pair_loaded(c, n, seed=10 + k) for k, (c, n) in
              enumerate(zip(cfgs, (20000, 50000, 8000, 120000, 3000)))]
    return cfgs, states


def _theta():
    return W.sur_init_params(31)


def _by_id(p):
    o = np.argsort(p["id"])
    return {k: v[o] for k, v in p.items()}


def _relmax(a, b):
    return np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300)


def _singles(cfgs, states, steps):
    from paper_2609_17661_b300 import Line
    out = []
    for c, st in zip(cfgs, states):
        ln = Line(c)
        ln.sur_set_params(_theta())
        ln.set_state(st)
        ln.step(steps)
        out.append((_by_id(ln.particles()), ln.fields(), ln.diag()))
        ln.close()
    return out


def _compare(ens, singles):
    for k, (ln, (p1, (E1, J1), d1)) in enumerate(zip(ens.lines, singles)):
        p0 = _by_id(ln.particles())
        E0, J0 = ln.fields()
        d0 = ln.diag()
        # with a full capacity, which pairs are dropped depends on the append order
        assert d1["pairs_dropped_cap"] == 0 and d0["pairs_dropped_cap"] == 0, k
        assert p0["id"].tolist() == p1["id"].tolist(), k
        for f in ("pos", "u", "w", "sp"):
            np.testing.assert_array_equal(p0[f], p1[f], err_msg=f"line {k} {f}")
        np.testing.assert_array_equal(J0, J1)
        np.testing.assert_array_equal(E0, E1)
        for f in ("step", "n_alive", "pairs_created", "scatters", "limiter_branch", "newton_branch",
                  "lost_north", "lost_south", "rng_draws"):
            assert d0[f] == d1[f], (k, f, d0[f], d1[f])
        # per-thread FP32 (compensated) energy sums group the particles by schedule
        assert d0["kinetic_energy"] == pytest.approx(d1["kinetic_energy"], rel=1e-6)


def test_ensemble_equals_lines_alone():
    """80 steps through the captured graph plus 7 launched directly."""
    from paper_2609_17661_b300 import Ensemble
    cfgs, states = _cfgs()
    ens = Ensemble(cfgs)
    ens.lines[0].sur_set_params(_theta())
    for ln, st in zip(ens.lines, states):
        ln.set_state(st)
    ens.step(87)
    d = ens.lines[3].diag()
    assert d["newton_branch"] + d["limiter_branch"] > 0 and d["scatters"] > 0
    _compare(ens, _singles(cfgs, states, 87))
    # a second replay of the same graph continues exactly
    ens.step(80)
    _compare(ens, _singles(cfgs, states, 167))
    ens.close()


def test_autotuned_schedule_keeps_results():
    """The autotuner picks per line a chunk size and a sort cadence from its
    candidates; a schedule changes the order of particles, not the results."""
    from paper_2609_17661_b300 import Ensemble
    cfgs, states = _cfgs()
    ens = Ensemble(cfgs)
    ens.lines[0].sur_set_params(_theta())
    for ln, st in zip(ens.lines, states):
        ln.set_state(st)
    chunk, cad, cost = ens.tune(trial_steps=10)
    assert set(chunk.tolist()) <= {1, 4, 16} and set(cad.tolist()) <= {10, 20, 40}
    assert np.all(cost > 0)
    a, b = ens.schedule()
    np.testing.assert_array_equal(a, chunk)
    np.testing.assert_array_equal(b, cad)
    ens.step(80)
    steps = ens.lines[0].diag()["step"]
    assert steps == 80 + 10 * 3 + 20 * 3 + 40 * 3
    _compare(ens, _singles(cfgs, states, steps))
    ens.close()


def test_ensemble_lines_match_the_oracle():
    """Three small lines with drag law SURROGATE advanced 80 steps by the
    ensemble (one replay of its captured super-step) against the FP64
    oracle with the same network, line by line: drag (the implicit midpoint
    through the network, no limiter) and the Lorentz force in a static
    non-uniform field with a negligible self-field and no scattering, the
    regime where FP32 and FP64 can agree over many steps.  Momenta agree to
    1e-5 of the line's scale plus 3 % of the drag's own change of u over the
    run (the network's BF16 activations, as for one step of a single line),
    positions and E to 1e-5 of the line."""
    import oracle as O
    from oracle import surrogate as S
    from paper_2609_17661_b300 import Ensemble
    theta = S.bf16_tensor_layers(W.sur_init_params(21).astype(np.float64))
    cfgs, states, fields = [], [], []
    for k, (r, N, n) in enumerate([(3.0, 512, 1500), (8.0, 1024, 1500), (20.0, 2048, 1000)]):
        c = W.config("C1", r_eq=r, n_cells=N, drag_law=W.DRAG_SURROGATE, b_pair_threshold=1e30, mc_on=0,
                     pairs_on=0, eta_min=0.0, drag_scale=3e-3, cells_per_skin_depth=1e6, seed=1 + k,
                     sort_every=20, capacity=4 * n + 65536, table_n_gamma=64, table_n_s=32)
        st = W.load_random(c, 4 * n, u_scale=3000.0, seed=40 + k)
        F = W.fbits(N)
        keep = (st["pos"] >= (48 << F)) & (st["pos"] < ((N - 48) << F))      # 80 steps move < 37 cells
        st = {kk: v[keep][:n] for kk, v in st.items()}
        x = (np.arange(N) + 0.5) / N
        cfgs.append(c)
        states.append(st)
        fields.append(0.02 * np.sin(2 * np.pi * 3 * x) + 0.01)
    ens = Ensemble(cfgs)
    ens.lines[0].sur_set_params(theta.astype(np.float32))
    for ln, st, E in zip(ens.lines, states, fields):
        ln.set_state(st, E=E)
    ens.step(80)
    for k, (ln, c, st, E) in enumerate(zip(ens.lines, cfgs, states, fields)):
        N = c["n_cells"]
        F = W.fbits(N)
        g = _by_id(ln.particles())
        Eg, _ = ln.fields()
        o_ = W.to_oracle(st, N)
        runs = {}
        for law in (O.DRAG_SURROGATE, O.DRAG_OFF):
            So = O.Sim(dict(c, drag_law=law))
            if law == O.DRAG_SURROGATE:
                So.set_surrogate(theta)
            So.set_particles(o_["s"], o_["u"], o_["w"], o_["sp"], o_["id"])
            So.set_field(E)
            So.step(80)
            runs[law] = (_by_id(So.particles()), So.fields()[0], So.diag())
        o, Eo, do = runs[O.DRAG_SURROGATE]
        o0 = runs[O.DRAG_OFF][0]
        assert g["id"].tolist() == o["id"].tolist() == o0["id"].tolist(), k
        du_drag = np.abs(o["u"] - o0["u"])
        assert np.mean(du_drag > 1e-3) > 0.1, k                 # the drag acts
        tol = 1e-5 * np.max(np.abs(o["u"])) + 0.03 * du_drag
        err = np.abs(g["u"].astype(np.float64) - o["u"])
        assert np.all(err <= tol), (k, float(np.max(err / tol)), int(np.sum(err > tol)))
        s = g["pos"].astype(np.float64) / float(1 << F)
        assert np.max(np.abs(s - o["s"])) <= 1e-5 * N, k
        assert np.max(np.abs(Eg - Eo)) <= 1e-5 * np.max(np.abs(Eo)), k
        assert ln.diag()["newton_branch"] == do["newton_branch"], k
    ens.close()



def _crowded_band(cfg, seed, extra):
    """A line's state for supply and annihilation: electron-positron pairs
    crowded into 16 cells at the middle of the line (weights 0.5, 1, 1.5,
    about twice n_max), and `extra` random particles of all species."""
    N = cfg["n_cells"]
    F = W.fbits(N)
    rng = np.random.default_rng(seed)
    parts = [W.load_random(cfg, extra, u_scale=3000.0, seed=seed + 1)]
    for c in range(N // 2 - 8, N // 2 + 8):
        for code, n in ((W.SP_ELEC, 60), (W.SP_POSI, 60 + int(rng.integers(-10, 10)))):
            st = W.empty_state(n)
            st["pos"][:] = ((c + rng.random(n)) * (1 << F)).astype(np.uint32)
            st["u"][:] = rng.normal(0.0, 0.05, n).astype(np.float32)
            st["w"][:] = rng.choice(np.array([0.5, 1.0, 1.5], np.float32), n)
            st["sp"][:] = code
            parts.append(st)
    st = {k: np.concatenate([p[k] for p in parts]) for k in parts[0]}
    st["id"] = rng.permutation(len(st["pos"])).astype(np.uint64) * 3 + 5
    return st


def test_ensemble_with_supply_and_annihilation_equals_lines_alone():
    """Lines with the atmosphere's top-up, the surface supply at a rate, and
    annihilation at n_max (every 2, 4 and 5 steps): 80 steps through the
    captured super-step plus 6 launched directly give, line by line, the
    single-line engine's particles, fields and counts."""
    from paper_2609_17661_b300 import Ensemble
    import oracle as O
    cfgs, states = [], []
    for k, (r, N, n, mode, ae) in enumerate([(3.0, 512, 6000, O.INJECT_TOPUP, 2), (8.0, 1024, 20000, O.INJECT_RATE, 4),
                                             (20.0, 768, 4000, O.INJECT_TOPUP, 5)]):
        c = W.config("C1", r_eq=r, n_cells=N, drag_law=W.DRAG_SURROGATE, inject_mode=mode, annihilate_every=ae,
                     n_max_ppc=60.0, drag_scale=0.05, seed=3 + k, sort_every=20, capacity=400000)
        cfgs.append(c)
        states.append(_crowded_band(c, 50 + k, n))
    ens = Ensemble(cfgs)
    ens.lines[0].sur_set_params(_theta())
    for ln, st in zip(ens.lines, states):
        ln.set_state(st)
    ens.step(86)
    for k, ln in enumerate(ens.lines):
        d = ln.diag()
        assert d["annihilated"] > 0 and d["injected"] > 0, (k, d["annihilated"], d["injected"])
    singles = _singles(cfgs, states, 86)
    _compare(ens, singles)
    for k, (ln, (_, _, d1)) in enumerate(zip(ens.lines, singles)):
        d0 = ln.diag()
        for f in ("annihilated", "injected", "injected_dropped", "pairs_rejected_nmax"):
            assert d0[f] == d1[f], (k, f, d0[f], d1[f])
    ens.close()


def test_ensemble_with_top_up_and_annihilation_matches_the_oracle():
    """Three lines with drag law SURROGATE, the atmosphere's top-up and
    annihilation at n_max every 2 steps, five steps of the ensemble against
    the FP64 oracle with the same BF16-exact network, line by line: top-up,
    annihilated weight, losses and Newton-branch counts exact, the weights
    exact, momenta to 1e-5 of the line's scale plus 3 % of the drag's own
    change of u, positions and E to 1e-5 (continuous drag, no scattering
    draws that the network's BF16 rate could tip)."""
    import oracle as O
    from oracle import surrogate as SU
    from paper_2609_17661_b300 import Ensemble
    theta = SU.bf16_tensor_layers(W.sur_init_params(21).astype(np.float64))
    cfgs, states, fields = [], [], []
    for k, (r, N, n) in enumerate([(3.0, 512, 2000), (8.0, 1024, 4000), (20.0, 768, 3000)]):
        c = W.config("C1", r_eq=r, n_cells=N, drag_law=W.DRAG_SURROGATE, inject_mode=O.INJECT_TOPUP,
                     annihilate_every=2, n_max_ppc=60.0, b_pair_threshold=1e30, mc_on=0, pairs_on=0, eta_min=0.0,
                     drag_scale=3e-3, seed=7 + k, sort_every=20, capacity=200000)
        x = (np.arange(N) + 0.5) / N
        cfgs.append(c)
        states.append(_crowded_band(c, 60 + k, n))
        fields.append(0.01 * np.sin(2 * np.pi * 3 * x) + 0.003 * np.cos(2 * np.pi * 7 * x + 1.0))
    ens = Ensemble(cfgs)
    ens.lines[0].sur_set_params(theta.astype(np.float32))
    for ln, st, E in zip(ens.lines, states, fields):
        ln.set_state(st, E=E, step=3)
    ens.step(5)
    for k, (ln, c, st, E) in enumerate(zip(ens.lines, cfgs, states, fields)):
        N = c["n_cells"]
        F = W.fbits(N)
        o_ = W.to_oracle(st, N)
        runs = {}
        for law in (O.DRAG_SURROGATE, O.DRAG_OFF):
            So = O.Sim(dict(c, drag_law=law))
            if law == O.DRAG_SURROGATE:
                So.set_surrogate(theta)
            So.set_particles(o_["s"], o_["u"], o_["w"], o_["sp"], o_["id"])
            So.set_field(E)
            So.set_step(3)
            So.step(5)
            runs[law] = (_by_id(So.particles()), So.fields()[0], So.diag())
        o, Eo, do = runs[O.DRAG_SURROGATE]
        o0 = runs[O.DRAG_OFF][0]
        dg = ln.diag()
        for f in ("injected", "annihilated", "n_alive", "lost_north", "lost_south", "newton_branch"):
            assert dg[f] == do[f], (k, f, dg[f], do[f])
        assert do["injected"] > 500 and do["annihilated"] > 20 * 4096, k
        g = _by_id(ln.particles())
        assert g["id"].tolist() == o["id"].tolist(), k
        assert np.array_equal(g["w"].astype(np.float64), o["w"]), k
        assert np.array_equal(g["sp"].astype(np.int32), o["sp"]), k
        du_drag = np.zeros(o["u"].size)
        common = np.isin(o["id"], o0["id"])
        du_drag[common] = np.abs(o["u"][common] - o0["u"][np.searchsorted(o0["id"], o["id"][common])])
        tol = 1e-5 * np.max(np.abs(o["u"])) + 0.03 * du_drag
        err = np.abs(g["u"].astype(np.float64) - o["u"])
        assert np.all(err <= tol), (k, float(np.max(err / tol)), int(np.sum(err > tol)))
        s = g["pos"].astype(np.float64) / float(1 << F)
        assert np.max(np.abs(s - o["s"])) <= 5 * (2.0 ** -F + c["cfl"] * 1e-5), k
        Eg, _ = ln.fields()
        assert _relmax(Eg, Eo) <= 1e-5, k
    ens.close()
