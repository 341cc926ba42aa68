"""FP64 CPU oracle of the per-step particle loop (test infrastructure).

Only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` may import this package.  It shares
no code with the CUDA library (``paper_2609_17661_b300``) and neither imports
the other; the two meet only in the tests, fed by the same seeded inputs.

The arithmetic lives in ``pic1d_oracle.c`` (plain C, FP64, one particle at a
time, in the order the paper's Sec. 3 gives).  This module is a ctypes
binding: argument marshalling only.

Parity pins (see ``tests/test_oracle_pins.py``) tie every function here to
something other than itself: closed forms, printed numbers of the paper,
library routines (numpy/scipy), brute force on tiny inputs and linear
theory.  The de-excitation angular law, the pair-momentum split, the
choice of omega_p in tau_min, the b-convention, the initial species split
and the photon model are readings the paper leaves open: for those the
oracle is "parity unpinned" beyond internal identities.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "pic1d_oracle.c")
# a build of the same source made elsewhere (the sanitizer test's) can be
# loaded instead through PIC1D_ORACLE_LIB
_LIB_ENV = os.environ.get("PIC1D_ORACLE_LIB")
_LIB = _LIB_ENV or os.path.join(_HERE, "liboracle.so")

PHOTON_RADIAL, PHOTON_DISK = 0, 1
DRAG_OFF, DRAG_CLOSED, DRAG_TABLE, DRAG_SURROGATE = 0, 1, 2, 3
RICS_SPLIT, RICS_DRAG_PLUS_PAIRS = 0, 1
INJECT_NONE, INJECT_RATE, INJECT_TOPUP = 0, 1, 2
S_BITS = 12


def build(force: bool = False) -> str:
    """Compile the oracle into ``oracle/liboracle.so`` (gcc, -O2, strict FP,
    OpenMP for the step's particle blocks; one thread unless set_threads)."""
    if _LIB_ENV:
        return _LIB
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        subprocess.check_call(
            ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fno-fast-math", "-ffp-contract=off", "-fopenmp",
             "-o", _LIB, _SRC, "-lm"])
    return _LIB


class OrcParams(C.Structure):
    _fields_ = [
        ("r_eq", C.c_double), ("n_cells", C.c_int32), ("cfl", C.c_double), ("b_star", C.c_double),
        ("b_convention", C.c_int32),
        ("kT_keV", C.c_double), ("photon_model", C.c_int32), ("drag_law", C.c_int32), ("drag_scale", C.c_double),
        ("table_n_gamma", C.c_int32), ("table_n_s", C.c_int32), ("table_log10g_max", C.c_double),
        ("quad_n_mu", C.c_int32), ("quad_n_phi", C.c_int32),
        ("eta_min", C.c_double), ("rics_mode", C.c_int32), ("mc_on", C.c_int32),
        ("cells_per_skin_depth", C.c_double), ("j_psi", C.c_double), ("n0_ppc", C.c_double),
        ("mass_ratio", C.c_double),
        ("ppc_e", C.c_int32), ("ppc_p", C.c_int32), ("ppc_i", C.c_int32), ("init_multiplicity", C.c_double),
        ("u_sigma", C.c_double),
        ("inject_mode", C.c_int32), ("inject_T", C.c_double),
        ("atmo_a0", C.c_double), ("atmo_h", C.c_double), ("atmo_ncut", C.c_double),
        ("pairs_on", C.c_int32), ("b_pair_threshold", C.c_double), ("pair_energy_threshold", C.c_double),
        ("n_max_ppc", C.c_double), ("annihilate_every", C.c_int32),
        ("seed", C.c_uint64), ("r_star_cm", C.c_double),
    ]


class OrcDiag(C.Structure):
    _fields_ = [
        ("n_alive", C.c_int64 * 4),
        ("pairs_created", C.c_int64), ("pairs_dropped_cap", C.c_int64), ("pairs_rejected_nmax", C.c_int64),
        ("pairs_lost_wall", C.c_int64),
        ("lost_north", C.c_int64), ("lost_south", C.c_int64), ("injected", C.c_int64), ("scatters", C.c_int64),
        ("psc_clamped", C.c_int64), ("limiter_branch", C.c_int64), ("newton_branch", C.c_int64),
        ("annihilated", C.c_int64),
        ("field_energy", C.c_double), ("kinetic_energy", C.c_double), ("ext_work", C.c_double),
        ("vc", C.c_double), ("charge", C.c_double), ("ke_lost", C.c_double),
    ]


_lib = None
_D = C.POINTER(C.c_double)
_I64 = C.POINTER(C.c_int64)
_I32 = C.POINTER(C.c_int32)
_U64 = C.POINTER(C.c_uint64)
_U32 = C.POINTER(C.c_uint32)
_U8 = C.POINTER(C.c_uint8)


def lib():
    global _lib
    if _lib is None:
        L = C.CDLL(build())
        sig = {
            "orc_philox4x32_10": (None, [_U32, _U32, _U32]),
            "orc_philox4x32_10_n": (None, [_U32, C.c_int64, _U32, _U32]),
            "orc_splitmix64": (C.c_uint64, [C.c_uint64]),
            "orc_child_id": (C.c_uint64, [C.c_uint64, C.c_int64, C.c_int]),
            "orc_inject_id": (C.c_uint64, [C.c_int64, C.c_int, C.c_int64, C.c_int]),
            "orc_atmo_id": (C.c_uint64, [C.c_int64, C.c_int, C.c_int64, C.c_int]),
            "orc_annih_key": (C.c_uint64, [C.c_uint64, C.c_int64]),
            "orc_gauss_legendre": (None, [C.c_int, _D, _D]),
            "orc_theta0": (C.c_double, [C.c_double]),
            "orc_arc_length": (C.c_double, [C.c_double, C.c_double]),
            "orc_line_length": (C.c_double, [C.c_double]),
            "orc_theta_of_s": (C.c_double, [C.c_double, C.c_double]),
            "orc_field_at_theta": (None, [C.POINTER(OrcParams), C.c_double, _D, _D, _D]),
            "orc_g": (C.c_double, [C.c_double]),
            "orc_radial": (None, [C.POINTER(OrcParams), C.c_double, C.c_double, C.c_double, C.c_double, _D, _D]),
            "orc_disk": (None, [C.POINTER(OrcParams), C.c_double, C.c_double, C.c_double, C.c_double, _D, _D]),
            "orc_build_table": (None, [C.POINTER(OrcParams), _D]),
            "orc_create": (C.c_void_p, [C.POINTER(OrcParams), _D]),
            "orc_free": (None, [C.c_void_p]),
            "orc_set_particles": (None, [C.c_void_p, C.c_int64, _D, _D, _D, _I32, _U64]),
            "orc_set_field": (None, [C.c_void_p, _D]),
            "orc_set_step": (None, [C.c_void_p, C.c_int64]),
            "orc_get_n": (C.c_int64, [C.c_void_p]),
            "orc_get_particles": (None, [C.c_void_p, _D, _D, _D, _I32, _U64]),
            "orc_get_fields": (None, [C.c_void_p, _D, _D]),
            "orc_get_nodes": (None, [C.c_void_p, _D, _D, _D, _U8]),
            "orc_get_scalars": (None, [C.c_void_p, _D]),
            "orc_get_density": (None, [C.c_void_p, _I64]),
            "orc_drag_code": (None, [C.c_void_p, C.c_double, C.c_double, _D, _D, _D]),
            "orc_rics_kinematics": (None, [C.c_double, C.c_double, C.c_double, C.c_double, _D]),
            "orc_cos_dipole": (C.c_double, [C.c_double]),
            "orc_deposit_int": (None, [C.c_int, C.c_int, C.c_int64, _I64, _I64, _D, _I32, _I64]),
            "orc_step": (None, [C.c_void_p]),
            "orc_set_threads": (None, [C.c_int]),
            "orc_get_threads": (C.c_int, []),
            "orc_run": (None, [C.c_void_p, C.c_int64]),
            "orc_rho": (None, [C.c_void_p, _D]),
            "orc_get_diag": (None, [C.c_void_p, C.POINTER(OrcDiag)]),
            "orc_drag_half_public": (C.c_double, [C.c_void_p, C.c_double, C.c_double]),
            "orc_gather_public": (C.c_double, [C.c_void_p, C.c_double]),
            "orc_node_interp_public": (C.c_double, [C.c_void_p, C.c_int, C.c_double]),
            "orc_sur_edge_mu": (C.c_double, [C.c_double, C.c_double, C.c_double]),
            "orc_set_surrogate": (None, [C.c_void_p, _D]),
            "orc_tp_line": (None, [C.POINTER(OrcParams), C.c_double, C.c_double, C.c_double, C.c_double,
                                   C.c_double, C.c_double, _D]),
            "orc_sur_forward": (None, [_D, _D, _D, _D]),
            "orc_sur_baseline": (C.c_double, [C.POINTER(OrcParams), C.c_double, C.c_double, C.c_double, C.c_double]),
            "orc_sur_point": (None, [C.POINTER(OrcParams), C.c_double, C.c_double, C.c_double, C.c_int, _D]),
            "orc_sur_sample": (None, [C.POINTER(OrcParams), C.c_uint64, C.c_uint64, C.c_double, C.c_double, _D]),
            "orc_sur_samples": (None, [C.POINTER(OrcParams), C.c_uint64, C.c_uint64, C.c_int64, C.c_double,
                                       C.c_double, _D]),
        }
        for name, (res, args) in sig.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _ptr(a, t):
    return a.ctypes.data_as(t)


def make_params(cfg: dict) -> OrcParams:
    p = OrcParams()
    for name, _ in OrcParams._fields_:
        setattr(p, name, cfg[name])
    return p


# ---------------------------------------------------------------- functions
def set_threads(n: int) -> int:
    """Threads of the oracle's step (process-wide; results do not depend on
    it: the step sums its particles in fixed blocks merged in order).
    Returns the count in effect."""
    lib().orc_set_threads(int(n))
    return int(lib().orc_get_threads())


def philox4x32_10(ctr, key):
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, np.uint32)
    lib().orc_philox4x32_10(_ptr(c, _U32), _ptr(k, _U32), _ptr(out, _U32))
    return out


def philox4x32_10_n(ctr, key):
    """The generator on an (n, 4) array of counters."""
    c = np.ascontiguousarray(ctr, dtype=np.uint32).reshape(-1, 4)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros_like(c)
    lib().orc_philox4x32_10_n(_ptr(c, _U32), c.shape[0], _ptr(k, _U32), _ptr(out, _U32))
    return out


def splitmix64(z):
    return int(lib().orc_splitmix64(int(z) & 0xFFFFFFFFFFFFFFFF))


def child_id(parent, step, member):
    return int(lib().orc_child_id(int(parent), int(step), int(member)))


def inject_id(step, foot, slot, member):
    return int(lib().orc_inject_id(int(step), int(foot), int(slot), int(member)))


def atmo_id(step, cell, slot, member):
    return int(lib().orc_atmo_id(int(step), int(cell), int(slot), int(member)))


def annih_key(pid, step):
    return int(lib().orc_annih_key(int(pid), int(step)))


def gauss_legendre(n):
    x = np.zeros(n)
    w = np.zeros(n)
    lib().orc_gauss_legendre(n, _ptr(x, _D), _ptr(w, _D))
    return x, w


def theta0(r_eq):
    return lib().orc_theta0(r_eq)


def arc_length(r_eq, theta):
    return lib().orc_arc_length(r_eq, theta)


def line_length(r_eq):
    return lib().orc_line_length(r_eq)


def theta_of_s(r_eq, s):
    return lib().orc_theta_of_s(r_eq, s)


def field_at_theta(cfg, theta):
    p = make_params(cfg)
    x, b, mu = C.c_double(), C.c_double(), C.c_double()
    lib().orc_field_at_theta(C.byref(p), theta, C.byref(x), C.byref(b), C.byref(mu))
    return x.value, b.value, mu.value


def g(y):
    return lib().orc_g(y)


def photon(cfg, u, x, b, mu, model=None):
    """(F^, N^) for one lepton: model RADIAL (closed form) or DISK (quadrature)."""
    p = make_params(cfg)
    F, N = C.c_double(), C.c_double()
    m = cfg["photon_model"] if model is None else model
    fn = lib().orc_disk if m == PHOTON_DISK else lib().orc_radial
    fn(C.byref(p), u, x, b, mu, C.byref(F), C.byref(N))
    return F.value, N.value


_table_cache = {}


def build_table(cfg):
    key = tuple((k, cfg[k]) for k in ("r_eq", "b_star", "b_convention", "kT_keV", "photon_model",
                                       "table_n_gamma", "table_n_s", "table_log10g_max",
                                       "quad_n_mu", "quad_n_phi", "r_star_cm"))
    if key not in _table_cache:
        p = make_params(cfg)
        t = np.zeros(2 * cfg["table_n_s"] * cfg["table_n_gamma"] * 2)
        lib().orc_build_table(C.byref(p), _ptr(t, _D))
        _table_cache[key] = t
    return _table_cache[key]


def rics_kinematics(b, d, u_i, ct):
    out = np.zeros(5)
    lib().orc_rics_kinematics(b, d, u_i, ct, _ptr(out, _D))
    return out


def cos_dipole(U):
    return lib().orc_cos_dipole(U)


def deposit_int(n_cells, fbits, p0, p1, w, sp):
    p0 = np.ascontiguousarray(p0, np.int64)
    p1 = np.ascontiguousarray(p1, np.int64)
    w = np.ascontiguousarray(w, np.float64)
    sp = np.ascontiguousarray(sp, np.int32)
    J = np.zeros(n_cells, np.int64)
    lib().orc_deposit_int(n_cells, fbits, len(p0), _ptr(p0, _I64), _ptr(p1, _I64), _ptr(w, _D),
                          _ptr(sp, _I32), _ptr(J, _I64))
    return J


def diag_dict(d: OrcDiag) -> dict:
    out = {}
    for name, _ in OrcDiag._fields_:
        v = getattr(d, name)
        out[name] = list(v) if name == "n_alive" else v
    return out


class Sim:
    """One field line advanced by the oracle."""

    def __init__(self, cfg: dict, table=None):
        self.cfg = dict(cfg)
        self._p = make_params(cfg)
        if cfg["drag_law"] == DRAG_TABLE and table is None:
            table = build_table(cfg)
        tptr = _ptr(np.ascontiguousarray(table, np.float64), _D) if table is not None else None
        self._keep = table
        self.h = lib().orc_create(C.byref(self._p), tptr)
        self.N = cfg["n_cells"]

    def __del__(self):
        if getattr(self, "h", None):
            lib().orc_free(self.h)
            self.h = None

    def set_particles(self, s, u, w, sp, pid):
        s = np.ascontiguousarray(s, np.float64)
        u = np.ascontiguousarray(u, np.float64)
        w = np.ascontiguousarray(w, np.float64)
        sp = np.ascontiguousarray(sp, np.int32)
        pid = np.ascontiguousarray(pid, np.uint64)
        lib().orc_set_particles(self.h, len(s), _ptr(s, _D), _ptr(u, _D), _ptr(w, _D), _ptr(sp, _I32),
                                _ptr(pid, _U64))

    def set_field(self, E):
        E = np.ascontiguousarray(E, np.float64)
        assert E.shape == (self.N,)
        lib().orc_set_field(self.h, _ptr(E, _D))

    def set_surrogate(self, theta):
        """Parameters (8770) of the network that drag law SURROGATE evaluates."""
        self._sur = np.ascontiguousarray(theta, dtype=np.float64)
        lib().orc_set_surrogate(self.h, _ptr(self._sur, _D))

    def set_step(self, step):
        lib().orc_set_step(self.h, int(step))

    def step(self, n=1):
        lib().orc_run(self.h, int(n))

    @property
    def n(self):
        return lib().orc_get_n(self.h)

    def particles(self):
        n = self.n
        s, u, w = np.zeros(n), np.zeros(n), np.zeros(n)
        sp = np.zeros(n, np.int32)
        pid = np.zeros(n, np.uint64)
        lib().orc_get_particles(self.h, _ptr(s, _D), _ptr(u, _D), _ptr(w, _D), _ptr(sp, _I32), _ptr(pid, _U64))
        return dict(s=s, u=u, w=w, sp=sp, id=pid)

    def fields(self):
        E, J = np.zeros(self.N), np.zeros(self.N)
        lib().orc_get_fields(self.h, _ptr(E, _D), _ptr(J, _D))
        return E, J

    def nodes(self):
        x, b, mu = np.zeros(self.N + 1), np.zeros(self.N + 1), np.zeros(self.N + 1)
        zone = np.zeros(self.N, np.uint8)
        lib().orc_get_nodes(self.h, _ptr(x, _D), _ptr(b, _D), _ptr(mu, _D), _ptr(zone, _U8))
        return dict(x=x, b=b, mu=mu, zone=zone)

    def scalars(self):
        out = np.zeros(8)
        lib().orc_get_scalars(self.h, _ptr(out, _D))
        return dict(L_R=out[0], R_cells=out[1], dt=out[2], q_p=out[3], j_ext=out[4], tau_min=out[5],
                    inj_acc=(out[6], out[7]))

    def density(self):
        d = np.zeros(self.N, np.int64)
        lib().orc_get_density(self.h, _ptr(d, _I64))
        return d

    def drag(self, u, s):
        F, dF, r = C.c_double(), C.c_double(), C.c_double()
        lib().orc_drag_code(self.h, u, s, C.byref(F), C.byref(dF), C.byref(r))
        return F.value, dF.value, r.value

    def drag_half(self, u0, s):
        return lib().orc_drag_half_public(self.h, u0, s)

    def gather(self, s):
        return lib().orc_gather_public(self.h, s)

    def node_interp(self, which, s):
        return lib().orc_node_interp_public(self.h, which, s)

    def rho(self):
        r = np.zeros(self.N + 1)
        lib().orc_rho(self.h, _ptr(r, _D))
        return r

    def diag(self):
        d = OrcDiag()
        lib().orc_get_diag(self.h, C.byref(d))
        return diag_dict(d)


SUR_FIELDS = ("f0", "f1", "f2", "f3", "t1", "t2", "mask", "lnN", "lnN_base", "F", "F_abs", "b", "x", "mu", "u")


def sur_point(cfg, r_eq, s_frac, log10g, neg):
    """One surrogate training sample at a given point (dict of SUR_FIELDS)."""
    p = make_params(cfg)
    out = np.zeros(15)
    lib().orc_sur_point(C.byref(p), r_eq, s_frac, log10g, int(neg), _ptr(out, _D))
    return dict(zip(SUR_FIELDS, out))


def sur_samples(cfg, seed, start, n, r_lo, r_hi):
    """n Philox-drawn samples from index `start`: array n x 15 (SUR_FIELDS)."""
    p = make_params(cfg)
    out = np.zeros((n, 15))
    lib().orc_sur_samples(C.byref(p), seed, start, n, r_lo, r_hi, _ptr(out, _D))
    return out


def sur_forward(theta, x):
    """The C oracle's FP64 network at one input: (y[2], dy/df0[2])."""
    th = np.ascontiguousarray(theta, dtype=np.float64)
    xx = np.ascontiguousarray(x, dtype=np.float64)
    y, dy = np.zeros(2), np.zeros(2)
    lib().orc_sur_forward(_ptr(th, _D), _ptr(xx, _D), _ptr(y, _D), _ptr(dy, _D))
    return y, dy


TP_FIELDS = ("gamma_min", "theta_first", "theta_b", "s_first", "s_b", "L", "l_pp", "region", "b_eq", "steps",
             "t_end", "u_end")


def tp_line(cfg, r_eq, gamma0=1000.0, dt=1e-3, t_max=1e3, b_thr=0.1, gamma_eps=0.01):
    """One line of the test-particle drag map (dict of TP_FIELDS)."""
    p = make_params(cfg)
    out = np.zeros(12)
    lib().orc_tp_line(C.byref(p), r_eq, gamma0, dt, t_max, b_thr, gamma_eps, _ptr(out, _D))
    return dict(zip(TP_FIELDS, out))
