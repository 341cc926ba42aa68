"""The C-ABI library loads and exports every entry point include/pic1d.h
declares (CPU only: no compute call is made here)."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    txt = open(os.path.join(ROOT, "include", "pic1d.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(pic1d_[a-z_0-9]+)\s*\(", txt)))


def _lib_path():
    from paper_2609_17661_b300 import build
    return build.build()


def test_header_declares_the_boundary():
    names = _declared()
    for n in ("pic1d_init", "pic1d_step", "pic1d_diag", "pic1d_set_state", "pic1d_free", "pic1d_last_error"):
        assert n in names


def test_library_exports_every_declared_symbol():
    path = _lib_path()
    lib = ctypes.CDLL(path)
    for n in _declared():
        assert hasattr(lib, n), n
    out = subprocess.run(["nm", "-D", "--defined-only", path], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT (pic1d_\w+)", out))
    assert set(_declared()) <= exported


def test_binding_mirrors_header_structs():
    """The ctypes structs list the header's fields in the header's order."""
    from paper_2609_17661_b300 import _lib
    txt = open(os.path.join(ROOT, "include", "pic1d.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    for struct, cls in (("pic1d_params", _lib.Params), ("pic1d_diag_t", _lib.Diag)):
        body = re.search(r"typedef struct " + struct + r"\s*\{(.*?)\}\s*" + struct, txt, flags=re.S).group(1)
        names = []
        for decl in body.split(";"):
            decl = decl.strip()
            if not decl:
                continue
            decl = re.sub(r"^\w+\*?\s+", "", decl)
            for piece in decl.split(","):
                names.append(re.sub(r"\[.*\]", "", piece).strip().lstrip("*"))
        assert names == [f[0] for f in cls._fields_], struct


def test_binding_signatures_cover_header():
    from paper_2609_17661_b300 import _lib
    assert sorted(_lib.SIGNATURES) == _declared()


def test_no_cpu_fallback_without_device():
    """Constructing a line without a CUDA device fails loudly."""
    import torch
    if torch.cuda.is_available():
        pytest.skip("a device is present")
    from paper_2609_17661_b300 import Line, workloads as W
    with pytest.raises(RuntimeError):
        Line(W.config("C1"))


def test_init_rejects_bad_parameters_before_any_device_work():
    """pic1d_init and pic1d_ens_init check their parameters before touching a
    device: each rule below returns PIC1D_EINVAL on a machine without one."""
    import ctypes as C
    from paper_2609_17661_b300 import _lib, make_params, workloads as W
    L = _lib.load()
    bad = [
        dict(inject_mode=W.INJECT_TOPUP, atmo_h=0.0),
        dict(inject_mode=W.INJECT_TOPUP, atmo_a0=-1.0),
        dict(inject_mode=W.INJECT_TOPUP, atmo_ncut=0.0),
        dict(inject_mode=3),
        dict(annihilate_every=1, n_max_ppc=0.0),                        # annihilation needs n_max
        dict(annihilate_every=-1),
        dict(sort_every=0),
        dict(n_cells=0),
        dict(ppc_e=16, ppc_p=8, ppc_i=4),                                # initial load not neutral
        dict(ppc_e=16, ppc_p=8, ppc_i=8, init_multiplicity=1.0),         # drift beta = 1/M = 1
        dict(ppc_e=16, ppc_p=8, ppc_i=8, u_sigma=-0.1),
        dict(ppc_e=-1),
        dict(capacity=-1),
        dict(capacity=2**31),                                            # slot indices are 32-bit
        dict(n_cells=65536, ppc_e=32768, ppc_p=16384, ppc_i=16384),      # an initial load past the slots
    ]
    for over in bad:
        p = make_params(W.config("C1", **over))
        h = C.c_void_p()
        assert L.pic1d_init(C.byref(p), C.byref(h)) == _lib.EINVAL, over
        assert not h.value
    # the ensemble refuses lines without the surrogate drag law, and an
    # annihilation cadence that does not divide its captured super-step of 80
    for over in (dict(annihilate_every=30, n_max_ppc=10.0), dict(drag_law=W.DRAG_TABLE)):
        cfg = W.config("C1", drag_law=W.DRAG_SURROGATE)
        cfg.update(over)
        arr = (_lib.Params * 1)(make_params(cfg))
        h = C.c_void_p()
        assert L.pic1d_ens_init(arr, 1, C.byref(h)) == _lib.EINVAL, over


def test_header_is_plain_c99_and_links(tmp_path):
    """include/pic1d.h compiles as strict C99 (no C++ or torch types at the
    boundary) and a C program links against the library and calls it."""
    import shutil
    import subprocess
    if shutil.which("gcc") is None:
        pytest.skip("no C compiler")
    from paper_2609_17661_b300 import _lib
    _lib.load()
    libdir = os.path.join(ROOT, "paper_2609_17661_b300")
    src = tmp_path / "use_abi.c"
    src.write_text(
        '#include "pic1d.h"\n'
        "int main(void) {\n"
        "  pic1d_params p = {0};\n"
        "  pic1d_ctx* c = 0;\n"
        "  pic1d_diag_t d;\n"
        "  (void)d;\n"
        "  return pic1d_init(&p, &c) == PIC1D_EINVAL && c == 0 ? 0 : 1;\n"
        "}\n")
    exe = tmp_path / "use_abi"
    cc = subprocess.run(["gcc", "-std=c99", "-Wall", "-Wextra", "-Werror", "-pedantic", "-I",
                         os.path.join(ROOT, "include"), str(src), "-L", libdir, "-lpic1d",
                         f"-Wl,-rpath,{libdir}", "-o", str(exe)], capture_output=True, text=True)
    assert cc.returncode == 0, cc.stderr
    run = subprocess.run([str(exe)], capture_output=True, text=True, timeout=120)
    assert run.returncode == 0, run.stderr
