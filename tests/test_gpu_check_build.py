"""The checking build (libpic1d_check.so, compiled with -DPIC1D_CHECK): its
kernels test the indexes they use (cells from positions, slots against the
capacity, gathers, sort keys and destinations) and the host fills the slack
past every particle array with a guard pattern that it tests after each
step.  On lines with drag, scattering, pairs, surface supply, the atmosphere
and annihilation, no test fails (pic1d_diag returns 0) and the results equal
the product build's bit for bit."""
import os
import subprocess
import sys
import textwrap

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)

pytestmark = pytest.mark.gpu

SCRIPT = textwrap.dedent("""
    import sys
    sys.path.insert(0, %(root)r)
    import numpy as np
    import oracle as O
    from paper_2609_17661_b300 import Line, workloads as W

    def run(name, cfg, st, steps):
        line = Line(cfg)
        line.set_state(st, step=0)
        line.step(steps)
        d = line.diag()
        p = line.particles()
        o = np.argsort(p["id"])
        E, J = line.fields()
        np.savez(%(out)r + "/" + name + ".npz", rc=d["rc"], pos=p["pos"][o], u=p["u"][o], w=p["w"][o],
                 sp=p["sp"][o], id=p["id"][o], E=E, J=J, pairs=d["pairs_created"], injected=d["injected"],
                 annihilated=d["annihilated"])
        line.close()

    cfg = W.config("C1", inject_mode=O.INJECT_RATE, sort_every=4, capacity=400000)
    st = W.load_drifting_plasma(cfg, seed=3)
    beam = W.load_beam(cfg, 3000, gamma_lo=30, gamma_hi=1e5, seed=4, cells=[0, 1, 2, 1021, 1022, 1023])
    st = {k: np.concatenate([st[k], beam[k]]) for k in st}
    st["id"] = np.arange(st["pos"].size, dtype=np.uint64) * 7 + 2
    run("pairs_rate", cfg, st, 12)

    cfg = W.config("C1", n_cells=128, inject_mode=O.INJECT_TOPUP, drag_law=O.DRAG_CLOSED, drag_scale=1e-3,
                   n_max_ppc=60.0, annihilate_every=2, capacity=200000)
    F = W.fbits(128)
    rng = np.random.default_rng(5)
    parts = [W.load_random(cfg, 3000, u_scale=30.0, seed=6)]
    for c in range(56, 72):
        for code, n in ((W.SP_ELEC, 60), (W.SP_POSI, 64)):
            s = W.empty_state(n)
            s["pos"][:] = ((c + rng.random(n)) * (1 << F)).astype(np.uint32)
            s["u"][:] = rng.normal(0.0, 0.05, n).astype(np.float32)
            s["sp"][:] = code
            parts.append(s)
    st = {k: np.concatenate([p[k] for p in parts]) for k in parts[0]}
    st["id"] = np.arange(st["pos"].size, dtype=np.uint64) * 3 + 1
    run("atmosphere_annihilation", cfg, st, 10)
    print("done")
""")


def _run(tmp, lib):
    env = dict(os.environ)
    if lib:
        env["PIC1D_LIB"] = lib
    out = str(tmp)
    r = subprocess.run([sys.executable, "-c", SCRIPT % {"root": ROOT, "out": out}], env=env, capture_output=True,
                       text=True, timeout=900)
    assert r.returncode == 0 and r.stdout.strip().endswith("done"), r.stderr[-3000:]
    return out


def test_checking_build_runs_clean_and_matches_the_product_build(tmp_path):
    from paper_2609_17661_b300 import build as B
    lib = B.build(check=True)
    (tmp_path / "check").mkdir()
    (tmp_path / "product").mkdir()
    a = _run(tmp_path / "check", lib)
    b = _run(tmp_path / "product", None)
    for name in ("pairs_rate", "atmosphere_annihilation"):
        x = np.load(os.path.join(a, name + ".npz"))
        y = np.load(os.path.join(b, name + ".npz"))
        assert int(x["rc"]) == 0, (name, int(x["rc"]))
        assert int(y["rc"]) == 0, (name, int(y["rc"]))
        for k in ("pos", "u", "w", "sp", "id", "E", "J", "pairs", "injected", "annihilated"):
            np.testing.assert_array_equal(x[k], y[k], err_msg=f"{name} {k}")
    x = np.load(os.path.join(a, "pairs_rate.npz"))
    assert int(x["pairs"]) > 0 and int(x["injected"]) > 0
    assert int(np.load(os.path.join(a, "atmosphere_annihilation.npz"))["annihilated"]) > 0
