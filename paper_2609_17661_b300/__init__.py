"""B300-native per-step particle loop of the 1D RICS pair-cascade PIC method.

Thin Python layer over the C ABI of ``include/pic1d.h`` (``libpic1d.so``,
hand-written sm_103a kernels).  PyTorch is used only for device memory and
streams; every step of the method runs in the library's kernels.  There is
no CPU fallback: constructing a :class:`Line` without the built library or
without a CUDA device raises.

Typical use::

    import torch
    from paper_2609_17661_b300 import Line, workloads as W
    cfg = W.config("C1")
    line = Line(cfg)                        # pic1d_init
    line.set_state(W.load_drifting_plasma(cfg))
    line.step(100)                          # pic1d_step (asynchronous)
    print(line.diag())                      # pic1d_diag
"""
from __future__ import annotations

import ctypes as C

import numpy as np

from . import _lib
from ._lib import Diag, Params

__all__ = ["Ensemble", "Line", "PicError", "make_params", "workloads"]


class PicError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"pic1d error {code}: {msg}")
        self.code = code


def make_params(cfg: dict, stream=None) -> Params:
    p = Params()
    for name, _ in Params._fields_:
        if name == "cuda_stream":
            continue
        setattr(p, name, cfg[name])
    p.cuda_stream = stream
    return p


def _is_torch(a):
    return type(a).__module__.startswith("torch")


def _arr(a, dtype):
    """(pointer, mem flag, keep-alive) for a numpy array or a torch tensor."""
    if a is None:
        return None, 0, None
    if _is_torch(a):
        assert a.is_contiguous()
        return C.c_void_p(a.data_ptr()), (1 if a.is_cuda else 0), a
    a = np.ascontiguousarray(a, dtype=dtype)
    return C.c_void_p(a.ctypes.data), 0, a


_ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p)
_FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_void_p)
_hooks = None


def use_torch_allocator(on: bool = True):
    """pic1d_set_allocator: take the library's device memory from PyTorch's
    caching allocator (on the current stream), or back from cudaMalloc.
    Only while no Line or Ensemble is alive."""
    global _hooks
    import torch
    L = _lib.load()
    if on:
        def alloc(n, user):
            try:
                return torch.cuda.caching_allocator_alloc(int(n))
            except Exception:
                return None

        def free(p, user):
            torch.cuda.caching_allocator_delete(p)

        hooks = (_ALLOC_FN(alloc), _FREE_FN(free))
        rc = L.pic1d_set_allocator(C.cast(hooks[0], C.c_void_p), C.cast(hooks[1], C.c_void_p), None)
        if rc == 0:
            _hooks = hooks            # the callbacks must outlive every buffer they made
    else:
        rc = L.pic1d_set_allocator(None, None, None)
        if rc == 0:
            _hooks = None
    if rc != 0:
        raise PicError(rc, "pic1d_set_allocator refused (contexts alive?)")


def tp_map(cfg: dict, r_eq, gamma0=1000.0, dt=1e-3, t_max=1e3, b_thr=0.1, gamma_eps=0.01):
    """pic1d_tp_map: test-particle drag map over the lines r_eq (array).
    Returns (dict of arrays per TpResult field, kernel ms)."""
    import torch
    L = _lib.load()
    r = np.ascontiguousarray(r_eq, dtype=np.float64)
    out = (_lib.TpResult * r.size)()
    ms = C.c_double()
    p = make_params(cfg, torch.cuda.current_stream().cuda_stream)
    rc = L.pic1d_tp_map(C.byref(p), C.c_void_p(r.ctypes.data), r.size, gamma0, dt, t_max, b_thr, gamma_eps,
                        C.cast(out, C.c_void_p), C.byref(ms))
    if rc != 0:
        raise PicError(rc, "pic1d_tp_map failed (see stderr)")
    res = {name: np.array([getattr(o, name) for o in out]) for name, _ in _lib.TpResult._fields_ if name != "pad"}
    return res, ms.value


class Line:
    """One field line on the GPU (a ``pic1d_ctx``)."""

    def __init__(self, cfg: dict, stream=None, _handle=None):
        import torch

        if not torch.cuda.is_available():
            raise RuntimeError("paper_2609_17661_b300 needs a CUDA device (no CPU path)")
        self.L = _lib.load()
        self.cfg = dict(cfg)
        self.N = cfg["n_cells"]
        self._owned = _handle is None
        if _handle is not None:      # a line owned by an Ensemble
            self.h = C.c_void_p(_handle)
            return
        if stream is None:
            stream = torch.cuda.current_stream().cuda_stream
        self._p = make_params(cfg, stream)
        h = C.c_void_p()
        rc = self.L.pic1d_init(C.byref(self._p), C.byref(h))
        if rc != 0:
            raise PicError(rc, "pic1d_init failed (see stderr)")
        self.h = h

    def _check(self, rc):
        if rc < 0:
            raise PicError(rc, self.L.pic1d_last_error(self.h).decode())
        return rc

    def close(self):
        if getattr(self, "h", None):
            if getattr(self, "_owned", True):
                self.L.pic1d_free(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ------------------------------------------------------------- state
    def set_state(self, st: dict, E=None, step=0):
        """pic1d_set_state from numpy (host) or torch CUDA tensors (device)."""
        n = len(st["pos"])
        args = [_arr(st["pos"], np.uint32), _arr(st["u"], np.float32), _arr(st["w"], np.float32),
                _arr(st["sp"], np.uint8), _arr(st["id"], np.uint64)]
        mems = {m for _, m, _ in args}
        e = _arr(E, np.float64)
        if E is not None:
            mems.add(e[1])
        if len(mems) > 1:
            raise ValueError("mixing host and device arrays")
        mem = mems.pop() if mems else 0
        self._check(self.L.pic1d_set_state(self.h, n, *[a[0] for a in args], e[0], int(step), mem))

    def step(self, n=1):
        self._check(self.L.pic1d_step(self.h, int(n)))

    def sort(self):
        self._check(self.L.pic1d_sort(self.h))

    def timing(self, on=True):
        """pic1d_timing: bracket every push launch with CUDA events."""
        self._check(self.L.pic1d_timing(self.h, 1 if on else 0))

    def check_wait(self, limit_clocks=2_000_000):
        """pic1d_check_wait: a bounded device wait that nothing completes"""
        self._check(self.L.pic1d_check_wait(self.h, int(limit_clocks)))

    def set_variant(self, v):
        """pic1d_set_variant: choose the push kernel variant."""
        self._check(self.L.pic1d_set_variant(self.h, int(v)))

    def variants(self):
        """[(particles per thread, min blocks per SM)] of every push variant."""
        out = []
        n = self.L.pic1d_variant_info(0, None, None)
        for v in range(n):
            a, b = C.c_int(), C.c_int()
            self.L.pic1d_variant_info(v, C.byref(a), C.byref(b))
            out.append((a.value, b.value))
        return out

    def slots(self):
        return int(self.L.pic1d_slots(self.h))

    def diag(self) -> dict:
        d = Diag()
        rc = self.L.pic1d_diag(self.h, C.byref(d))
        out = {}
        for name, _ in Diag._fields_:
            v = getattr(d, name)
            out[name] = list(v) if name == "n_alive" else v
        out["rc"] = rc
        return out

    def fields(self):
        E = np.zeros(self.N, np.float64)
        J = np.zeros(self.N, np.int64)
        self._check(self.L.pic1d_get_fields(self.h, E.ctypes.data, J.ctypes.data, 0))
        return E, J

    def rho(self):
        """pic1d_get_rho: integer node charge (N+1 values, units of J)."""
        r = np.zeros(self.N + 1, np.int64)
        self._check(self.L.pic1d_get_rho(self.h, C.c_void_p(r.ctypes.data), 0))
        return r

    def gauss_mark(self):
        """pic1d_gauss_mark: start the discrete continuity check; diag() then
        reports gauss_residual_max (0 while charge is conserved exactly)."""
        self._check(self.L.pic1d_gauss_mark(self.h))

    def particles(self, alive_only=True) -> dict:
        n = self.slots()
        out = dict(pos=np.zeros(n, np.uint32), u=np.zeros(n, np.float32), w=np.zeros(n, np.float32),
                   sp=np.zeros(n, np.uint8), id=np.zeros(n, np.uint64))
        self._check(self.L.pic1d_get_particles(self.h, n, out["pos"].ctypes.data, out["u"].ctypes.data,
                                               out["w"].ctypes.data, out["sp"].ctypes.data,
                                               out["id"].ctypes.data, 0))
        if alive_only:
            keep = out["sp"] != 255
            out = {k: v[keep] for k, v in out.items()}
        return out

    def table(self):
        ng, ns = self.cfg["table_n_gamma"], self.cfg["table_n_s"]
        t = np.zeros(2 * ns * ng * 2, np.float32)
        self._check(self.L.pic1d_get_table(self.h, t.ctypes.data))
        return t

    def deposit(self, pos0, pos1, w, sp, J):
        """pic1d_deposit on torch CUDA tensors (int64 pos0/pos1, float32 w, uint8 sp, int64 J)."""
        self._check(self.L.pic1d_deposit(self.h, int(pos0.numel()), C.c_void_p(pos0.data_ptr()),
                                         C.c_void_p(pos1.data_ptr()), C.c_void_p(w.data_ptr()),
                                         C.c_void_p(sp.data_ptr()), C.c_void_p(J.data_ptr())))
        return J


    # ---------------------------------------------------------- checkpoints
    def save(self, path):
        """pic1d_save: the whole state of the line to a file."""
        self._check(self.L.pic1d_save(self.h, str(path).encode()))

    def load(self, path):
        """pic1d_load: restore a file written by save (same parameters)."""
        self._check(self.L.pic1d_load(self.h, str(path).encode()))

    # ------------------------------------------------------------ surrogate
    def sur_set_params(self, theta):
        """pic1d_sur_set_params from a host array of 8770 FP32 values."""
        a = np.ascontiguousarray(theta, dtype=np.float32)
        assert a.size == _lib.SUR_N_PARAMS
        self._check(self.L.pic1d_sur_set_params(self.h, C.c_void_p(a.ctypes.data)))

    def sur_get_params(self):
        a = np.zeros(_lib.SUR_N_PARAMS, np.float32)
        self._check(self.L.pic1d_sur_get_params(self.h, C.c_void_p(a.ctypes.data)))
        return a

    def sur_samples(self, seed, start, n, r_lo, r_hi):
        """pic1d_sur_samples into a new CUDA tensor of n x 16 records."""
        import torch
        out = torch.empty((max(int(n), 1), _lib.SUR_RECORD), dtype=torch.float32, device="cuda")
        self._check(self.L.pic1d_sur_samples(self.h, int(seed), int(start), int(n), float(r_lo), float(r_hi),
                                             C.c_void_p(out.data_ptr())))
        return out[:int(n)]

    def sur_grad(self, records):
        """pic1d_sur_grad over a CUDA tensor of records: (gradient, mean loss)."""
        assert records.is_cuda and records.is_contiguous()
        g = np.zeros(_lib.SUR_N_PARAMS, np.float32)
        loss = C.c_double()
        self._check(self.L.pic1d_sur_grad(self.h, C.c_void_p(records.data_ptr()), int(records.shape[0]),
                                          C.c_void_p(g.ctypes.data), C.byref(loss)))
        return g, loss.value

    def sur_train_steps(self, records, batch, steps, lr):
        assert records.is_cuda and records.is_contiguous()
        self._check(self.L.pic1d_sur_train_steps(self.h, C.c_void_p(records.data_ptr()), int(records.shape[0]),
                                                 int(batch), int(steps), float(lr)))

    def sur_infer(self, rows):
        """pic1d_sur_infer on a CUDA tensor (inputs in the first 4 columns): n x 4 tensor."""
        import torch
        assert rows.is_cuda and rows.is_contiguous() and rows.dim() == 2
        out = torch.empty((max(rows.shape[0], 1), 4), dtype=torch.float32, device="cuda")
        self._check(self.L.pic1d_sur_infer(self.h, C.c_void_p(rows.data_ptr()), int(rows.shape[1]),
                                           int(rows.shape[0]), C.c_void_p(out.data_ptr())))
        return out[:rows.shape[0]]

    def train_surrogate(self, n_samples, epochs, batch, lr, r_lo, r_hi, seed, n_val, val_seed,
                        lr_final=0.0) -> dict:
        """pic1d_train_surrogate: returns the report as a dict."""
        cfg = _lib.TrainCfg(int(n_samples), int(epochs), int(batch), float(lr), float(lr_final), float(r_lo),
                            float(r_hi), int(seed), int(n_val), int(val_seed))
        rep = _lib.TrainReport()
        self._check(self.L.pic1d_train_surrogate(self.h, C.byref(cfg), C.byref(rep)))
        return {name: getattr(rep, name) for name, _ in _lib.TrainReport._fields_}


class Ensemble:
    """Many independent lines advanced together (a ``pic1d_ens``): one launch
    per phase of a step for all lines, super-steps replayed as a CUDA graph,
    per-line schedule from the autotuner."""

    def __init__(self, cfgs):
        import torch

        if not torch.cuda.is_available():
            raise RuntimeError("paper_2609_17661_b300 needs a CUDA device (no CPU path)")
        self.L = _lib.load()
        self.cfgs = [dict(c) for c in cfgs]
        arr = (Params * len(cfgs))(*[make_params(c, None) for c in cfgs])
        h = C.c_void_p()
        rc = self.L.pic1d_ens_init(arr, len(cfgs), C.byref(h))
        if rc != 0:
            raise PicError(rc, "pic1d_ens_init failed (see stderr)")
        self.h = h
        self.lines = [Line(c, _handle=self.L.pic1d_ens_line(self.h, k)) for k, c in enumerate(self.cfgs)]

    def _check(self, rc):
        if rc < 0:
            raise PicError(rc, self.L.pic1d_ens_last_error(self.h).decode())
        return rc

    def step(self, n=1):
        self._check(self.L.pic1d_ens_step(self.h, int(n)))

    def stream(self):
        """The ensemble's stream as a torch.cuda.ExternalStream."""
        import torch
        return torch.cuda.ExternalStream(self.L.pic1d_ens_stream(self.h))

    def schedule(self):
        n = len(self.cfgs)
        a, b = np.zeros(n, np.int32), np.zeros(n, np.int32)
        self._check(self.L.pic1d_ens_get_schedule(self.h, C.c_void_p(a.ctypes.data), C.c_void_p(b.ctypes.data)))
        return a, b

    def set_schedule(self, chunk_tiles=None, sort_every=None):
        a = None if chunk_tiles is None else np.ascontiguousarray(chunk_tiles, np.int32)
        b = None if sort_every is None else np.ascontiguousarray(sort_every, np.int32)
        self._check(self.L.pic1d_ens_set_schedule(self.h, None if a is None else C.c_void_p(a.ctypes.data),
                                                  None if b is None else C.c_void_p(b.ctypes.data)))

    def tune(self, trial_steps=10):
        """pic1d_ens_tune: (chunk_tiles, sort_every, estimated ms per step) per line."""
        n = len(self.cfgs)
        a, b, c = np.zeros(n, np.int32), np.zeros(n, np.int32), np.zeros(n)
        self._check(self.L.pic1d_ens_tune(self.h, int(trial_steps), C.c_void_p(a.ctypes.data),
                                          C.c_void_p(b.ctypes.data), C.c_void_p(c.ctypes.data)))
        return a, b, c

    def record(self, capacity):
        """pic1d_ens_record: keep V_c and the pair count of every line after
        each of the next `capacity` steps (on the device)."""
        self._check(self.L.pic1d_ens_record(self.h, int(capacity)))
        self._rec_cap = int(capacity)

    def history(self, line, window=None):
        """pic1d_ens_history: dict(vc, pairs, pair_rate) of one line's record;
        window defaults to one light-crossing time of the line (n_cells / cfl
        steps)."""
        cap = getattr(self, "_rec_cap", 0)
        if window is None:
            cfg = self.cfgs[line] if 0 <= line < len(self.cfgs) else None
            window = max(1, int(round(cfg["n_cells"] / cfg["cfl"]))) if cfg else 1
        vc, rate = np.zeros(max(cap, 1)), np.zeros(max(cap, 1))
        pairs = np.zeros(max(cap, 1), np.int64)
        n = C.c_int32()
        self._check(self.L.pic1d_ens_history(self.h, int(line), int(window), C.c_void_p(vc.ctypes.data),
                                             C.c_void_p(pairs.ctypes.data), C.c_void_p(rate.ctypes.data),
                                             C.byref(n)))
        k = n.value
        return dict(vc=vc[:k], pairs=pairs[:k], pair_rate=rate[:k], window=int(window))

    def close(self):
        if getattr(self, "h", None):
            for ln in self.lines:
                ln.h = None
            self.L.pic1d_ens_free(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


from . import workloads  # noqa: E402
