"""Pins of the surrogate's FP64 oracle (``oracle/surrogate.py`` and the
sample functions of ``pic1d_oracle.c``) against things other than itself:
finite differences, PyTorch autograd and ``torch.optim.Adam`` (independent
library routines), invariances of the network, and the closed forms of the
photon field (Sec. 2.2)."""
import math

import numpy as np
import pytest

import oracle as O
from oracle import surrogate as S
from paper_2609_17661_b300 import workloads as W


def _theta(seed=1, scale=1.0):
    return W.sur_init_params(seed).astype(np.float64) * scale


def _batch(n=64, seed=2):
    rng = np.random.default_rng(seed)
    X = rng.uniform(-1, 1, (n, 4))
    X[:, 3] = rng.choice([-1.0, 1.0], n)
    return X, rng.uniform(-1, 1, n), rng.normal(0, 1, n), (rng.random(n) < 0.8).astype(float)


def test_layout_matches_the_abi_count():
    assert S.N_PARAMS == W.SUR_N_PARAMS == 8770
    th = _theta()
    Ws, bs = S.unpack(th)
    np.testing.assert_array_equal(S.pack(Ws, bs), th)


def test_backward_matches_central_differences():
    """Every layer's weights and biases: relative error <= 1e-6."""
    th = _theta(scale=2.0)
    X, T1, T2, M = _batch()
    _, g = S.loss_grad(th, X, T1, T2, M)
    rng = np.random.default_rng(5)
    idx = np.concatenate([rng.choice(np.arange(kw, kb + SIZE[0]), 12, replace=False)
                          for (kw, kb), SIZE in zip(S.OFFSETS, S.SIZES)])
    h = 1e-6
    for k in idx:
        tp, tm = th.copy(), th.copy()
        tp[k] += h
        tm[k] -= h
        fd = (S.loss_grad(tp, X, T1, T2, M)[0] - S.loss_grad(tm, X, T1, T2, M)[0]) / (2 * h)
        assert abs(fd - g[k]) <= 1e-6 * max(abs(g[k]), 1e-3), (k, fd, g[k])


def test_forward_and_backward_match_torch_autograd():
    torch = pytest.importorskip("torch")
    th = _theta(scale=1.5)
    X, T1, T2, M = _batch(128, seed=7)
    Ws, bs = S.unpack(th)
    tw = [torch.tensor(w, dtype=torch.float64, requires_grad=True) for w in Ws]
    tb = [torch.tensor(b, dtype=torch.float64, requires_grad=True) for b in bs]
    h = torch.tensor(X)
    for layer in range(4):
        h = torch.nn.functional.linear(h, tw[layer], tb[layer])
        if layer < 3:
            h = torch.nn.functional.silu(h)
    t1, t2, m = (torch.tensor(a) for a in (T1, T2, M))
    loss = ((h[:, 0] - t1) ** 2 * m + (h[:, 1] - t2) ** 2).mean()
    loss.backward()
    Y, _ = S.forward(th, X)
    np.testing.assert_allclose(Y, h.detach().numpy(), rtol=1e-13, atol=1e-13)
    lo, g = S.loss_grad(th, X, T1, T2, M)
    assert lo == pytest.approx(float(loss.detach()), rel=1e-13)
    gt = S.pack([w.grad.numpy() for w in tw], [b.grad.numpy() for b in tb])
    np.testing.assert_allclose(g, gt, rtol=1e-11, atol=1e-14)


def test_hidden_unit_permutation_leaves_outputs_unchanged():
    """Permuting the units of a hidden layer (rows of W_l and b_l, columns of
    W_{l+1}) is a symmetry of the network: catches transposed or misindexed
    layers."""
    th = _theta(scale=1.3)
    X, *_ = _batch(32, seed=9)
    Ws, bs = S.unpack(th)
    rng = np.random.default_rng(1)
    for layer in range(3):
        p = rng.permutation(64)
        Ws[layer] = Ws[layer][p]
        bs[layer] = bs[layer][p]
        Ws[layer + 1] = Ws[layer + 1][:, p]
    Y0, _ = S.forward(th, X)
    Y1, _ = S.forward(S.pack(Ws, bs), X)
    np.testing.assert_allclose(Y1, Y0, rtol=1e-12, atol=1e-13)


def test_jvp_matches_differences_in_the_first_input():
    th = _theta(scale=1.7)
    X, *_ = _batch(16, seed=4)
    Y, Yd = S.jvp_log10g(th, X)
    h = 1e-6
    Xp, Xm = X.copy(), X.copy()
    Xp[:, 0] += h
    Xm[:, 0] -= h
    fd = (S.forward(th, Xp)[0] - S.forward(th, Xm)[0]) / (2 * h)
    np.testing.assert_allclose(Yd, fd, rtol=1e-6, atol=1e-9)
    np.testing.assert_allclose(Y, S.forward(th, X)[0], rtol=1e-14)


def test_silu_special_values():
    assert S.silu(np.array(0.0)) == 0.0
    assert S.dsilu(np.array(0.0)) == 0.5
    assert S.silu(np.array(40.0)) == pytest.approx(40.0, rel=1e-15)
    assert abs(S.silu(np.array(-40.0))) < 1e-15
    # the minimum of x sigma(x) is where the derivative vanishes (x = -1.2785)
    assert abs(S.dsilu(np.array(-1.2784645427610738))) < 1e-12


def test_adam_matches_torch_and_the_constant_gradient_step():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(3)
    th = rng.normal(size=50)
    t = torch.tensor(th.copy(), requires_grad=True)
    opt = torch.optim.Adam([t], lr=1e-3)
    A = S.Adam(50, lr=1e-3)
    for k in range(7):
        g = rng.normal(size=50) * (k + 1)
        t.grad = torch.tensor(g)
        opt.step()
        th = A.step(th, g)
    np.testing.assert_allclose(th, t.detach().numpy(), rtol=1e-13, atol=1e-15)
    # a constant gradient gives m^ = g and v^ = g^2 at every step: each step
    # moves by lr * g / (|g| + eps)
    A = S.Adam(3, lr=0.01)
    g = np.array([2.0, -0.5, 1e-3])
    x = np.zeros(3)
    for k in range(5):
        x1 = A.step(x, g)
        np.testing.assert_allclose(x1 - x, -0.01 * g / (np.abs(g) + 1e-8), rtol=1e-12)
        x = x1


def test_bf16_rounding():
    # exactly representable values stay, halfway cases go to even
    assert S.bf16(1.0) == 1.0 and S.bf16(-2.5) == -2.5
    one_ulp = 2.0 ** -7
    assert S.bf16(1.0 + one_ulp / 2) == 1.0              # tie -> even (1.0)
    assert S.bf16(1.0 + 1.5 * one_ulp) == 1.0 + 2 * one_ulp  # tie -> even
    assert S.bf16(1.0 + 0.6 * one_ulp) == 1.0 + one_ulp


# ------------------------------------------------------------ samples
def test_radial_samples_are_the_aberrated_cosine():
    """With radially streaming photons the drag and the rate are separate
    closed forms; their ratio must be gamma b mu~, mu~ = (mu - beta)/(1 -
    beta mu), the momentum per scattering (Sec. 2.2)."""
    cfg = W.config("C2", photon_model=O.PHOTON_RADIAL)
    for lg, sf, neg in [(0.3, 0.2, 0), (2.0, 0.5, 1), (4.0, 0.8, 0), (6.5, 0.05, 1)]:
        p = O.sur_point(cfg, 20.0, sf, lg, neg)
        gam = math.sqrt(1 + p["u"] ** 2)
        beta = p["u"] / gam
        mut = (p["mu"] - beta) / (1 - beta * p["mu"])
        assert p["t1"] == pytest.approx(mut, rel=1e-12, abs=1e-14)
        if p["mask"]:
            assert p["F"] / (gam * p["b"] * math.exp(p["lnN"])) == pytest.approx(mut, rel=1e-10, abs=1e-12)


def test_disk_samples_bounds_and_far_limit():
    """<mu~> is a weighted mean of cosines (in [-1, 1]); |F| <= F_abs; the
    drag is gamma b N^ <mu~>; and far from the star (x >> 1) the disk sample
    tends to the radial one."""
    cfg = W.config("C2")
    X = O.sur_samples(cfg, 7, 0, 3000, 2.0, 30.0)
    D = dict(zip(O.SUR_FIELDS, X.T))
    m = D["mask"] > 0
    assert np.all(np.abs(D["t1"]) <= 1 + 1e-12)
    assert np.all(np.abs(D["F"]) <= D["F_abs"] * (1 + 1e-12) + 1e-300)
    gam = np.sqrt(1 + D["u"] ** 2)
    np.testing.assert_allclose(D["F"][m], (gam * D["b"] * np.exp(D["lnN"]) * D["t1"])[m], rtol=1e-9,
                               atol=1e-12 * np.max(np.abs(D["F"])))
    for f in ("f0", "f1", "f2"):
        assert np.all(np.abs(D[f]) <= 1.0)
    # far limit: near the equator of a long line the disk is small
    cr = W.config("C2", photon_model=O.PHOTON_RADIAL)
    pd = O.sur_point(cfg, 300.0, 0.5, 3.0, 0)
    pr = O.sur_point(cr, 300.0, 0.5, 3.0, 0)
    assert pd["x"] > 299
    assert pd["t1"] == pytest.approx(pr["t1"], abs=1e-4)
    assert pd["lnN"] == pytest.approx(pr["lnN"], abs=1e-4)


def test_sample_draws_cover_the_box():
    cfg = W.config("C2")
    X = O.sur_samples(cfg, 11, 0, 4000, 2.0, 30.0)
    D = dict(zip(O.SUR_FIELDS, X.T))
    lg = (D["f0"] + 1) * 4
    assert lg.min() < 0.01 and lg.max() > 7.99
    assert abs(np.mean(D["f3"])) < 0.05
    # the same index gives the same sample; start offsets are consistent
    Y = O.sur_samples(cfg, 11, 1000, 5, 2.0, 30.0)
    np.testing.assert_array_equal(Y, X[1000:1005])


def test_reconstruction_inverts_the_targets():
    """Feeding the targets back through the reconstruction returns the
    quadrature's drag and rate wherever the rate is above the floor."""
    cfg = W.config("C2")
    X = O.sur_samples(cfg, 5, 0, 2000, 20.0, 20.0)
    D = dict(zip(O.SUR_FIELDS, X.T))
    m = D["mask"] > 0
    gam = np.sqrt(1 + D["u"] ** 2)
    F, lnN = S.reconstruct(np.stack([D["t1"], D["t2"]], 1), D["lnN_base"], gam, D["b"])
    np.testing.assert_allclose(lnN[m], D["lnN"][m], atol=1e-12)
    assert np.max(S.drag_error(F[m], D["F"][m], D["F_abs"][m])) < 1e-10


# ------------------------------------------------- the surrogate drag law
def test_c_network_matches_numpy_network():
    """Two separate FP64 implementations of the same network (the C oracle's,
    used by the drag law, and the numpy one, pinned to autograd) agree."""
    th = _theta(11, scale=1.7)
    X, *_ = _batch(20, seed=12)
    Y, Yd = S.jvp_log10g(th, X)
    for k in range(20):
        y, dy = O.sur_forward(th, X[k])
        np.testing.assert_allclose(y, Y[k], rtol=1e-12, atol=1e-13)
        np.testing.assert_allclose(dy, Yd[k], rtol=1e-12, atol=1e-13)


def _sur_sim(theta, **over):
    cfg = W.config("C2", n_cells=2048, drag_law=O.DRAG_SURROGATE, **over)
    S_ = O.Sim(cfg)
    S_.set_surrogate(theta)
    return S_, cfg


def test_surrogate_drag_is_the_reconstruction_of_the_samples():
    """The drag law evaluates F^ = gamma b N^ y0 and ln N^ = max(B, LT) + y1
    from the network at the particle's place: equal to the reconstruction
    from the sample definitions (orc_sur_point: features and baseline B) fed
    through the numpy network."""
    th = _theta(13, scale=0.8)
    Sim, cfg = _sur_sim(th)
    N = cfg["n_cells"]
    k = cfg["drag_scale"] / Sim.scalars()["R_cells"]     # code units per F^ (and per N^)
    for s_cells, u in [(300.5, 40.0), (1024.0, -3.0), (1800.25, 2500.0), (77.0, 0.3)]:
        x = Sim.node_interp(0, s_cells)
        b = Sim.node_interp(1, s_cells)
        mu = Sim.node_interp(2, s_cells)
        F, dF, rate = Sim.drag(u, s_cells)
        lg = math.log10(math.sqrt(1 + u * u))
        f = S.features(np.array([lg]), np.array([s_cells / N]), np.array([b]), np.array([u]),
                       cfg["table_log10g_max"])
        Y, _ = S.forward(th, f)
        base = O.lib().orc_sur_baseline(C_params(cfg), u, x, b, mu)
        gam = math.sqrt(1 + u * u)
        Fr, lnNr = S.reconstruct(Y, np.array([base]), gam, b)
        assert F / k == pytest.approx(Fr[0], rel=1e-9)
        assert math.log(rate / k) == pytest.approx(lnNr[0], abs=1e-9)


def C_params(cfg):
    import ctypes
    return ctypes.byref(O.make_params(cfg))


def test_surrogate_drag_derivative_matches_differences():
    """dF/du of the surrogate law (used by Newton in the implicit midpoint)
    equals the central difference of F, across the box and both signs."""
    th = _theta(14, scale=1.2)
    Sim, _ = _sur_sim(th)
    for s_cells, u in [(300.5, 40.0), (1024.0, -3.0), (1800.25, 2500.0), (77.0, 0.3), (1500.0, -700.0)]:
        F, dF, _ = Sim.drag(u, s_cells)
        h = 1e-6 * max(1.0, abs(u))
        Fp, _, _ = Sim.drag(u + h, s_cells)
        Fm, _, _ = Sim.drag(u - h, s_cells)
        fd = (Fp - Fm) / (2 * h)
        assert dF == pytest.approx(fd, rel=2e-5, abs=1e-12 * max(abs(F), 1e-300) + 1e-300)


def test_surrogate_law_outside_the_box_is_the_table_law():
    """Outside the training box (gamma above 10^G, or b beyond the network's
    range) the quadrature stands in: the surrogate law equals the table law
    on the line's own quadrature table (a small table keeps the CPU build
    short), in F, dF and the rate."""
    th = _theta(15)
    small = dict(table_n_gamma=32, table_n_s=16, quad_n_mu=8, quad_n_phi=8)
    Sim, cfg = _sur_sim(th, **small)
    St = O.Sim(dict(cfg, drag_law=O.DRAG_TABLE))
    for u, s in ((3.0e8, 500.0), (-4.0e8, 1900.0), (1.0e9, 0.0)):     # gamma above 10^8
        assert Sim.drag(u, s) == pytest.approx(St.drag(u, s), rel=1e-14)
    # a line whose field reaches below the network's b range (b < 10^-4 at its
    # equator): there too the table law, inside the gamma box
    far = dict(cfg, r_eq=60.0)
    Sf = O.Sim(far)
    Sf.set_surrogate(th)
    Sft = O.Sim(dict(far, drag_law=O.DRAG_TABLE))
    mid = far["n_cells"] / 2
    assert Sf.node_interp(1, mid) < 1e-4
    for u in (30.0, -2.0e3):
        assert Sf.drag(u, mid) == pytest.approx(Sft.drag(u, mid), rel=1e-14)
