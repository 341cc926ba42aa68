"""The learned surrogate on the GPU (through the C ABI) against its FP64
oracle: quadrature samples, the tensor-core forward pass and its derivative,
gradients (GPU BF16 vs CPU FP64 within 1e-2), Adam steps, and training.

BF16 tolerance: the GPU rounds the hidden activations that feed the tensor
cores to BF16 (relative 2^-9) and accumulates in FP32; with BF16-exact
weights the outputs and gradients then differ from FP64 by a few 1e-3 of
their scale, checked at 1e-2."""
import math

import numpy as np
import pytest

import oracle as O
from oracle import surrogate as S
from paper_2609_17661_b300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _line(**over):
    from paper_2609_17661_b300 import Line
    return Line(W.config("C2", n_cells=1024, **over))


def _bf16_params(seed, scale=1.0):
    """Parameters whose W2 and W3 are BF16-exact (the GPU's tensor-core operands)."""
    return S.bf16_tensor_layers((W.sur_init_params(seed).astype(np.float64) * scale).astype(np.float32))


FIELDS = ("f0", "f1", "f2", "f3", "t1", "t2", "mask", "base", "lnN", "F", "F_abs", "gamma", "b", "u", "x", "mu")


@pytest.mark.parametrize("model,r_lo,r_hi", [(O.PHOTON_DISK, 2.0, 30.0), (O.PHOTON_DISK, 20.0, 20.0),
                                             (O.PHOTON_RADIAL, 4.0, 4.0)])
def test_samples_match_oracle(model, r_lo, r_hi):
    """Records from the device quadrature equal the oracle's FP64 records
    (the same Philox draws), to FP32 storage."""
    line = _line(photon_model=model)
    n = 3000
    g = line.sur_samples(9, 100, n, r_lo, r_hi).cpu().numpy().astype(np.float64)
    o = O.sur_samples(W.config("C2", photon_model=model), 9, 100, n, r_lo, r_hi)
    D = dict(zip(O.SUR_FIELDS, o.T))
    G = dict(zip(FIELDS, g.T))
    for k in ("f0", "f1", "f2", "f3", "x", "mu", "u"):
        np.testing.assert_allclose(G[k], D[k], rtol=2e-6, atol=2e-6, err_msg=k)
    np.testing.assert_allclose(G["b"], D["b"], rtol=1e-5)
    m = D["mask"] > 0
    # the mask flips only where ln N sits at the floor itself
    flip = G["mask"] != D["mask"]
    assert np.all(np.abs(D["lnN"][flip] - S.LT) < 1e-4)
    keep = m & ~flip
    np.testing.assert_allclose(G["t1"][keep], D["t1"][keep], rtol=1e-5, atol=1e-6)
    np.testing.assert_allclose(G["t2"], D["t2"], rtol=1e-5, atol=2e-5)
    np.testing.assert_allclose(G["lnN"][keep], D["lnN"][keep], rtol=1e-6, atol=2e-5)
    np.testing.assert_allclose(G["base"], np.maximum(D["lnN_base"], -745.0), rtol=1e-6, atol=2e-5)
    big = keep & (np.abs(D["F"]) > 1e-30)
    np.testing.assert_allclose(G["F"][big], D["F"][big], rtol=1e-5, atol=1e-6 * np.max(np.abs(D["F"][big])))
    np.testing.assert_allclose(G["F_abs"][big], D["F_abs"][big], rtol=1e-5)


def test_infer_matches_oracle_forward_and_derivative():
    """Tensor-core forward pass (and its derivative in f0) against the FP64
    network with the same BF16 weights: a wrong operand layout, descriptor or
    transposition would miss by O(1)."""
    line = _line()
    th = _bf16_params(4, scale=2.0)
    line.sur_set_params(th.astype(np.float32))
    rec = W.sur_random_records(1000, seed=3)      # 7 full tiles + a ragged one
    Y = line.sur_infer(torch.from_numpy(rec).cuda()).cpu().numpy().astype(np.float64)
    X = rec[:, :4].astype(np.float64)
    Yo, Yd = S.jvp_log10g(th, X)
    scale = np.max(np.abs(Yo), axis=0)
    assert np.max(np.abs(Y[:, :2] - Yo) / scale) <= 1e-2
    dscale = np.max(np.abs(Yd), axis=0)
    assert np.max(np.abs(Y[:, 2:] - Yd) / dscale) <= 2e-2
    # and far below an O(1) miss: the typical error is at BF16 level
    assert np.median(np.abs(Y[:, :2] - Yo) / scale) <= 3e-3


def test_gradient_matches_oracle():
    """Gradient of the mean loss, GPU (BF16 activations, FP32 sums) against
    CPU FP64 backprop on the same records: within 1e-2 relative per layer."""
    line = _line()
    th = _bf16_params(5, scale=1.5)
    line.sur_set_params(th.astype(np.float32))
    rec = W.sur_random_records(1000, seed=6)
    g, loss = line.sur_grad(torch.from_numpy(rec).cuda())
    X = rec[:, :4].astype(np.float64)
    lo, go = S.loss_grad(th, X, rec[:, 4].astype(np.float64), rec[:, 5].astype(np.float64),
                         rec[:, 6].astype(np.float64))
    assert loss == pytest.approx(lo, rel=1e-2)
    for (kw, kb), (o, i) in zip(S.OFFSETS, S.SIZES):
        for a, b in ((kw, kw + o * i), (kb, kb + o)):
            err = np.linalg.norm(g[a:b] - go[a:b]) / np.linalg.norm(go[a:b])
            assert err <= 1e-2, (a, b, err)


def test_adam_steps_follow_the_oracle():
    """Three Adam steps on consecutive batches: the parameter updates point the
    same way as the FP64 oracle's and have the same size."""
    line = _line()
    th0 = _bf16_params(7)
    line.sur_set_params(th0.astype(np.float32))
    rec = W.sur_random_records(768, seed=8)
    line.sur_train_steps(torch.from_numpy(rec).cuda(), 256, 3, 1e-3)
    th_g = line.sur_get_params().astype(np.float64)
    A = S.Adam(S.N_PARAMS, lr=1e-3)
    th = th0.copy()
    for k in range(3):
        r = rec[256 * k:256 * (k + 1)].astype(np.float64)
        # the GPU computes with the BF16 rounding of its FP32 W2 and W3
        _, g = S.loss_grad(S.bf16_tensor_layers(th), r[:, :4], r[:, 4], r[:, 5], r[:, 6])
        th = A.step(th, g)
    dg, do = th_g - th0, th - th0
    big = np.abs(do) > 1e-3     # parameters that moved by about lr each step
    assert big.mean() > 0.5
    assert np.mean(np.sign(dg[big]) == np.sign(do[big])) > 0.99
    # Adam divides by the gradient's running size, so a parameter whose
    # gradient is near zero in one step can move differently when its BF16
    # and FP64 gradients differ in that step; all but a few agree within 5 %
    close = np.isclose(dg[big], do[big], rtol=0.05, atol=5e-5)
    assert close.mean() > 0.99, close.mean()


def test_training_run_learns_the_quadrature():
    """A short training run on the r_eq = 20 line (2e5 samples, 5 epochs):
    the loss falls by a factor 20 and the held-out drag and rate errors
    against quadrature are reported."""
    line = _line()
    line.sur_set_params(W.sur_init_params(0))
    rep = line.train_surrogate(n_samples=200_000, epochs=5, batch=8192, lr=3e-3, r_lo=20.0, r_hi=20.0, seed=3,
                               n_val=20_000, val_seed=1003)
    assert rep["steps"] == 5 * (200_000 // 8192)
    assert rep["loss_last"] < rep["loss_first"] / 5
    assert rep["val_count"] > 15_000
    print(rep)
    assert rep["drag_err_median"] < 0.05 and rep["lnN_err_median"] < 0.1


# ------------------------------------------------- the surrogate in the push
def _sur_cfg(**over):
    base = dict(drag_law=O.DRAG_SURROGATE, b_pair_threshold=1e30, mc_on=0, pairs_on=0, eta_min=0.0,
                drag_scale=3e-3)
    base.update(over)
    return W.config("C1", n_cells=1024, **base)


def _by_id(p):
    o = np.argsort(p["id"])
    return {k: v[o] for k, v in p.items()}


def test_push_with_surrogate_drag_matches_oracle():
    """One step with drag law SURROGATE (the network in the push, Newton on
    its exact derivative), no limiter: momenta agree with the FP64 oracle to
    1e-5 of the line's scale plus 3 % of the drag's own change of u (the
    network's BF16 activations), and the integer current matches where the
    motion does."""
    from paper_2609_17661_b300 import Line
    cfg = _sur_cfg()
    th = _bf16_params(21, scale=1.0)
    st = W.load_random(cfg, 50_000, u_scale=3000.0, seed=22)
    line = Line(cfg)
    line.sur_set_params(th.astype(np.float32))
    line.set_state(st)
    line.step(1)
    g = _by_id(line.particles())
    S_ = O.Sim(cfg)
    S_.set_surrogate(th)
    o_ = W.to_oracle(st, cfg["n_cells"])
    S_.set_particles(o_["s"], o_["u"], o_["w"], o_["sp"], o_["id"])
    S_.step(1)
    o = _by_id(S_.particles())
    S0 = O.Sim(dict(cfg, drag_law=O.DRAG_OFF))
    S0.set_particles(o_["s"], o_["u"], o_["w"], o_["sp"], o_["id"])
    S0.step(1)
    o0 = _by_id(S0.particles())
    assert g["id"].tolist() == o["id"].tolist()
    du_drag = np.abs(o["u"] - o0["u"])
    assert np.mean(du_drag > 1e-3) > 0.1          # the drag acts (elsewhere the rate is in the Wien tail)
    tol = 1e-5 * np.max(np.abs(o["u"])) + 0.03 * du_drag
    err = np.abs(g["u"].astype(np.float64) - o["u"])
    assert np.all(err <= tol), (np.max(err / tol), int(np.sum(err > tol)))
    dg, do = line.diag(), S_.diag()
    assert dg["newton_branch"] == do["newton_branch"] > 10_000


def test_push_with_surrogate_limiter_and_scattering_statistics():
    """Limiter on, scattering and pairs on: branch counts and yields of the
    GPU's surrogate law agree with the oracle's within what a 1 % drag or rate
    difference can move (decisions near a threshold may flip)."""
    from paper_2609_17661_b300 import Line
    cfg = W.config("C1", n_cells=1024, drag_law=O.DRAG_SURROGATE, drag_scale=3e-3, eta_min=1.0)
    th = _bf16_params(23, scale=1.0)
    st = W.load_beam(cfg, 40_000, gamma_lo=20, gamma_hi=2e4, seed=8)
    line = Line(cfg)
    line.sur_set_params(th.astype(np.float32))
    line.set_state(st)
    line.step(2)
    S_ = O.Sim(cfg)
    S_.set_surrogate(th)
    o_ = W.to_oracle(st, cfg["n_cells"])
    S_.set_particles(o_["s"], o_["u"], o_["w"], o_["sp"], o_["id"])
    S_.step(2)
    dg, do = line.diag(), S_.diag()
    assert do["scatters"] > 1000
    for k in ("scatters", "limiter_branch", "newton_branch", "pairs_created"):
        assert abs(dg[k] - do[k]) <= 0.02 * do[k] + 20, (k, dg[k], do[k])


def test_gain_over_quadrature_and_tables():
    """What the trained network gains (G8 of the method's design):
    (i) against the method without it -- the quadrature evaluated per point --
        it is much faster per evaluation (both on this GPU);
    (ii) against tables for an ensemble of lines it is one 35 KB network for
        every line of r_eq in [2, 30] where a table is 1 MiB per line; its
        accuracy off the table nodes is measured against quadrature beside the
        bilinear table's (both reported; the table is faster per lookup)."""
    from paper_2609_17661_b300 import Line
    cfg = W.config("C2", n_cells=1024)
    line = Line(cfg)
    line.sur_set_params(W.sur_init_params(0))
    rep = line.train_surrogate(**dict(W.SUR_TRAIN_ENSEMBLE, n_samples=4_000_000, epochs=10, lr=3e-3,
                                      lr_final=1e-5, n_val=50_000))
    # (i) speed per point: quadrature (32 x 32 directions, FP64) vs network
    n = 1_000_000
    e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
    e0.record()
    rec = line.sur_samples(77, 0, n, 2.0, 30.0)
    e1.record()
    y = line.sur_infer(rec)
    e2.record()
    torch.cuda.synchronize()
    t_quad, t_net = e0.elapsed_time(e1), e1.elapsed_time(e2)
    assert t_quad / t_net > 20, (t_quad, t_net)
    # (ii) accuracy off the nodes of a 256 x 256 table on one line (r_eq = 20):
    # the network (GPU) and the bilinear table (FP64 oracle), both against
    # quadrature at the same random points
    m = 4000
    pts = O.sur_samples(cfg, 78, 0, m, 20.0, 20.0)
    D = dict(zip(O.SUR_FIELDS, pts.T))
    keep = (D["lnN"] > S.LE) & (D["F_abs"] > 0)
    X = torch.from_numpy(np.ascontiguousarray(pts[:, :4], dtype=np.float32)).cuda()
    Y = line.sur_infer(X).cpu().numpy().astype(np.float64)
    gam = np.sqrt(1 + D["u"] ** 2)
    Fn, lnNn = S.reconstruct(Y, D["lnN_base"], gam, D["b"])
    err_net = S.drag_error(Fn[keep], D["F"][keep], D["F_abs"][keep])
    T = O.Sim(dict(cfg, r_eq=20.0, n_cells=4096, drag_law=O.DRAG_TABLE))
    k = cfg["drag_scale"] / T.scalars()["R_cells"]
    s_cells = (D["f1"] + 1) / 2 * 4096
    Ft = np.array([T.drag(u, s)[0] / k for u, s in zip(D["u"], s_cells)])
    err_tab = S.drag_error(Ft[keep], D["F"][keep], D["F_abs"][keep])
    print("gain: quadrature %.1f ms, network %.2f ms per 1e6 points (x%.0f); network 35 KB for all lines vs "
          "1 MiB table per line; drag error median/p99 network %.2e/%.2e, table %.2e/%.2e; training %s"
          % (t_quad, t_net, t_quad / t_net, np.median(err_net), np.percentile(err_net, 99),
             np.median(err_tab), np.percentile(err_tab, 99), {k2: rep[k2] for k2 in ("train_ms", "steps")}))
    assert np.median(err_net) < 2e-2


def test_push_outside_the_training_box_uses_the_table_law():
    """Above gamma = 10^G (the network's box) the surrogate law hands over to
    the line's own quadrature table: one step of such leptons with drag law
    SURROGATE gives bit for bit the momenta and positions of the same step
    with drag law TABLE."""
    from paper_2609_17661_b300 import Line
    cfg = _sur_cfg(eta_min=1.0)
    st = W.load_beam(cfg, 20_000, gamma_lo=2e8, gamma_hi=3e9, seed=31)
    out = {}
    for law in (O.DRAG_SURROGATE, O.DRAG_TABLE):
        line = Line(dict(cfg, drag_law=law))
        if law == O.DRAG_SURROGATE:
            line.sur_set_params(_bf16_params(32, scale=1.0).astype(np.float32))
        line.set_state(st)
        line.step(1)
        out[law] = _by_id(line.particles())
        line.close()
    a, b = out[O.DRAG_SURROGATE], out[O.DRAG_TABLE]
    np.testing.assert_array_equal(a["id"], b["id"])
    np.testing.assert_array_equal(a["u"], b["u"])
    np.testing.assert_array_equal(a["pos"], b["pos"])


@pytest.mark.slow
def test_full_training_run_holds_its_measured_accuracy():
    """The workload's training run on the r_eq = 20 line (1e7 quadrature
    samples, 20 epochs of 8192, Adam with the cosine decay 1e-2 -> 1e-5):
    the held-out drag error against quadrature stays below the target at
    the median (measured 4.6e-4; bound 1e-3) and at its measured tail (p99
    1.6e-2; bound 2.5e-2, where the 1e-3 target is not met), and the rate's
    median within 1e-3 in ln N (measured 5e-4)."""
    line = _line()
    line.sur_set_params(W.sur_init_params(0))
    rep = line.train_surrogate(**W.SUR_TRAIN_COSINE)
    print({k: rep[k] for k in rep if "err" in k})
    assert rep["drag_err_median"] <= 1e-3, rep["drag_err_median"]
    assert rep["drag_err_p99"] <= 2.5e-2, rep["drag_err_p99"]
    assert rep["lnN_err_median"] <= 1e-3, rep["lnN_err_median"]


@pytest.mark.slow
def test_shared_network_holds_its_measured_accuracy():
    """One network for every line with r_eq in [2, 30] (the ensemble's),
    trained on 2e7 quadrature samples over 40 epochs of 8192 with the cosine
    decay from 1e-2: held-out median drag error against quadrature <= 1.3e-3
    (measured 9.2e-4 .. 9.7e-4 on two lines; the 1e-3 target sits at the
    edge of what the 64-wide network reaches over the whole family of lines,
    while a line's own network meets it with room), p99 <= 3.5e-2 (measured
    2.6e-2 .. 2.7e-2)."""
    line = _line()
    line.sur_set_params(W.sur_init_params(0))
    rep = line.train_surrogate(**W.SUR_TRAIN_SHARED)
    print({k: rep[k] for k in rep if "err" in k})
    assert rep["drag_err_median"] <= 1.3e-3, rep["drag_err_median"]
    assert rep["drag_err_p99"] <= 3.5e-2, rep["drag_err_p99"]
    assert rep["lnN_err_median"] <= 2e-3, rep["lnN_err_median"]

