"""The oracle's C under AddressSanitizer and UndefinedBehaviorSanitizer
(CPU only): the same source built with -fsanitize=address,undefined runs the
oracle's paths -- the initial load, a C1 line with drag, scattering, pairs
and RATE supply, the atmosphere with annihilation, the surrogate law, the
test-particle line, the threaded step -- in a child process with the ASan
runtime preloaded; any report fails the test."""
import os
import subprocess
import sys
import textwrap

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)

SCRIPT = textwrap.dedent("""
    import sys
    sys.path.insert(0, %r)
    import numpy as np
    import oracle as O
    from oracle import surrogate as SU
    from paper_2609_17661_b300 import workloads as W

    # the initial load and a C1 line with drag, scattering, pairs, RATE supply
    cfg = W.config("C1", n_cells=64, ppc_e=16, ppc_p=8, ppc_i=8, inject_mode=O.INJECT_RATE,
                   table_n_gamma=32, table_n_s=16, quad_n_mu=8, quad_n_phi=8)
    S = O.Sim(cfg)
    beam = W.load_beam(cfg, 200, gamma_lo=30, gamma_hi=3e3, seed=5)
    S.step(6)
    d = S.diag()
    assert d["injected"] > 0
    # threaded
    O.set_threads(4)
    S2 = O.Sim(cfg)
    S2.step(4)
    O.set_threads(1)
    # the atmosphere with annihilation
    cfg = W.config("C1", n_cells=128, inject_mode=O.INJECT_TOPUP, annihilate_every=2, n_max_ppc=8.0,
                   drag_law=O.DRAG_CLOSED, capacity=100000)
    S = O.Sim(cfg)
    st = W.load_random(cfg, 3000, u_scale=3.0, seed=2)
    o = W.to_oracle(st, cfg["n_cells"])
    S.set_particles(o["s"], o["u"], o["w"], o["sp"], o["id"])
    S.step(6)
    # the surrogate law
    cfg = W.config("C1", n_cells=64, drag_law=O.DRAG_SURROGATE, table_n_gamma=32, table_n_s=16,
                   quad_n_mu=8, quad_n_phi=8)
    S = O.Sim(cfg)
    S.set_surrogate(SU.bf16_tensor_layers(W.sur_init_params(3).astype(np.float64)))
    st = W.load_random(cfg, 500, u_scale=30.0, seed=3)
    o = W.to_oracle(st, cfg["n_cells"])
    S.set_particles(o["s"], o["u"], o["w"], o["sp"], o["id"])
    S.step(3)
    print("ok")
""" % ROOT)


def _sanitizer_runtime():
    try:
        out = subprocess.run(["gcc", "-print-file-name=libasan.so"], capture_output=True, text=True, check=True)
    except (OSError, subprocess.CalledProcessError):
        return None
    path = out.stdout.strip()
    return path if os.path.isabs(path) and os.path.exists(path) else None


@pytest.mark.slow
def test_oracle_is_clean_under_address_and_undefined_behaviour_sanitizers(tmp_path):
    asan = _sanitizer_runtime()
    if asan is None:
        pytest.skip("no gcc AddressSanitizer runtime")
    lib = str(tmp_path / "liboracle_san.so")
    subprocess.check_call(["gcc", "-O1", "-g", "-std=c11", "-fPIC", "-shared", "-fno-fast-math", "-ffp-contract=off",
                           "-fopenmp", "-fsanitize=address,undefined", "-fno-sanitize-recover=undefined",
                           "-fno-omit-frame-pointer", "-o", lib, os.path.join(ROOT, "oracle", "pic1d_oracle.c"),
                           "-lm"])
    env = dict(os.environ, PIC1D_ORACLE_LIB=lib, LD_PRELOAD=asan,
               ASAN_OPTIONS="detect_leaks=0:abort_on_error=0:exitcode=23",
               UBSAN_OPTIONS="halt_on_error=1:print_stacktrace=1:exitcode=24")
    r = subprocess.run([sys.executable, "-c", SCRIPT], env=env, capture_output=True, text=True, timeout=600)
    report = r.stderr[-4000:]
    assert r.returncode == 0, report
    assert "AddressSanitizer" not in r.stderr and "runtime error" not in r.stderr, report
    assert r.stdout.strip().endswith("ok")
