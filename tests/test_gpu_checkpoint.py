"""Checkpoint and resume (pic1d_save / pic1d_load): a line saved at step k
and resumed in a fresh context continues exactly as the saved one does --
the same particles (ids, positions, momenta, weights, species), the same
integer current and FP64 field, the same counters."""
import numpy as np
import pytest

import oracle as O
from paper_2609_17661_b300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _by_id(p):
    o = np.argsort(p["id"])
    return {k: v[o] for k, v in p.items()}


def _state(line):
    p = _by_id(line.particles())
    E, J = line.fields()
    return p, E, J, line.diag()


def _same(a, b):
    (pa, Ea, Ja, da), (pb, Eb, Jb, db) = a, b
    assert pa["id"].tolist() == pb["id"].tolist()
    for f in ("pos", "u", "w", "sp"):
        np.testing.assert_array_equal(pa[f], pb[f], err_msg=f)
    np.testing.assert_array_equal(Ea, Eb)
    np.testing.assert_array_equal(Ja, Jb)
    for f in ("step", "n_alive", "pairs_created", "pairs_rejected_nmax", "injected", "scatters", "limiter_branch",
              "newton_branch", "lost_north", "lost_south", "rng_draws", "ext_work", "field_energy", "vc"):
        assert da[f] == db[f], (f, da[f], db[f])
    assert da["pairs_dropped_cap"] == 0
    assert da["kinetic_energy"] == pytest.approx(db["kinetic_energy"], rel=1e-6)


def test_resume_continues_exactly(tmp_path):
    from paper_2609_17661_b300 import Line
    N = 1024
    cfg = W.config("C1", n_cells=N, drag_scale=3e-3, inject_mode=O.INJECT_RATE, n_max_ppc=40.0,
                   capacity=400_000, sort_every=20)
    st = W.load_drifting_plasma(cfg)
    beam = W.load_beam(cfg, 20000, gamma_lo=30, gamma_hi=3e3, seed=4)
    beam["id"] += 10**7
    st = {k: np.concatenate([st[k], beam[k]]) for k in st}
    a = Line(cfg)
    a.set_state(st)
    a.step(30)
    path = tmp_path / "line.ckpt"
    a.save(path)
    a.step(25)
    ref = _state(a)
    assert ref[3]["pairs_created"] > 0 and ref[3]["injected"] > 0
    b = Line(cfg)
    b.load(path)
    assert b.diag()["step"] == 30
    b.step(25)
    _same(_state(b), ref)


def test_resume_with_the_surrogate_network(tmp_path):
    from paper_2609_17661_b300 import Line
    cfg = W.config("C1", drag_law=W.DRAG_SURROGATE, drag_scale=0.05, capacity=200_000)
    st = W.load_drifting_plasma(cfg)
    a = Line(cfg)
    a.sur_set_params(W.sur_init_params(41))
    a.set_state(st)
    a.step(5)
    a.save(tmp_path / "sur.ckpt")
    a.step(4)
    ref = _state(a)
    b = Line(cfg)
    b.load(tmp_path / "sur.ckpt")
    np.testing.assert_array_equal(b.sur_get_params(), a.sur_get_params())
    b.step(4)
    _same(_state(b), ref)


def test_load_refuses_other_parameters_and_other_files(tmp_path):
    from paper_2609_17661_b300 import Line, PicError
    cfg = W.config("C1", capacity=100_000)
    a = Line(cfg)
    a.set_state(W.load_random(cfg, 1000, seed=1))
    a.save(tmp_path / "a.ckpt")
    with pytest.raises(PicError):
        Line(dict(cfg, j_psi=27.0)).load(tmp_path / "a.ckpt")
    (tmp_path / "junk").write_bytes(b"not a checkpoint at all")
    with pytest.raises(PicError):
        Line(cfg).load(tmp_path / "junk")
    # the stream and the capacity may differ
    Line(dict(cfg, capacity=50_000)).load(tmp_path / "a.ckpt")
