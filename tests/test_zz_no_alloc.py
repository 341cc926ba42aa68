"""The scratch-free cell sort (pic1d_sort_static) against the context sort.

pic1d_sort_static serves callers that cannot allocate device memory (code
running inside a memory pool it does not own, or on a device whose memory is
reserved in full): it keeps its scratch in a fixed array inside the library.
This file is collected last on purpose, so that a run stopping at the first
failure has run every other test before it.
"""
import ctypes as C

import numpy as np
import pytest

from paper_2609_17661_b300 import workloads as W

torch = pytest.importorskip("torch")


def _key(pos, sp, u, F, N):
    # the octave of gamma^2 = 1 + u^2, rounded once to FP32 (exact in FP64
    # for |u| < 6e7): its exponent; 32 bands, the last one open
    q = (u.astype(np.float64) ** 2 + 1.0).astype(np.float32)
    band = np.minimum((q.view(np.uint32) >> 23).astype(np.int64) - 127, 31)
    return ((2 * (sp == W.SP_ION) + (u < 0)) * N + (pos.astype(np.int64) >> F)) * 32 + band


@pytest.mark.gpu
def test_static_sort_matches_context_sort_on_two_calls():
    from paper_2609_17661_b300 import Line, _lib
    L = _lib.load()
    N = 4096
    F = W.fbits(N)
    cfg = W.config("C1", n_cells=N)
    stream = torch.cuda.current_stream()
    for call, (n, seed) in enumerate(((300001, 5), (123457, 6))):
        st = W.load_random(cfg, n, seed=seed)
        st["sp"][seed::11] = 255      # removed slots are dropped by the sort
        # the existing entry point: a context's sort
        line = Line(cfg)
        line.set_state(st)
        line.sort()
        ref = line.particles(alive_only=False)
        line.close()
        # the new entry point, on device copies of the same arrays
        dev = {k: torch.from_numpy(v.copy()).cuda() for k, v in st.items()}
        out = {k: torch.empty_like(v) for k, v in dev.items()}
        n_out = torch.full((1,), -1, dtype=torch.int64, device="cuda")
        rc = L.pic1d_sort_static(N, n, *[C.c_void_p(dev[k].data_ptr()) for k in ("pos", "u", "w", "sp", "id")],
                                 *[C.c_void_p(out[k].data_ptr()) for k in ("pos", "u", "w", "sp", "id")],
                                 C.c_void_p(n_out.data_ptr()), C.c_void_p(stream.cuda_stream))
        assert rc == 0
        torch.cuda.synchronize()
        m = int(n_out.item())
        assert m == ref["pos"].size == int((st["sp"] != 255).sum()), call
        got = {k: v[:m].cpu().numpy() for k, v in out.items()}
        # same key sequence (the sort's order is unique up to order inside a key)
        kg, kr = _key(got["pos"], got["sp"], got["u"], F, N), _key(ref["pos"], ref["sp"], ref["u"], F, N)
        np.testing.assert_array_equal(kg, kr)
        assert np.all(np.diff(kg) >= 0)
        # same particles under each key
        og = np.lexsort((got["id"], kg))
        orf = np.lexsort((ref["id"], kr))
        for k in ("pos", "u", "w", "sp", "id"):
            np.testing.assert_array_equal(got[k][og], ref[k][orf])


@pytest.mark.gpu
def test_static_sort_rejects_lines_beyond_its_scratch():
    from paper_2609_17661_b300 import _lib
    L = _lib.load()
    z = torch.zeros(8, dtype=torch.int64, device="cuda")
    p = C.c_void_p(z.data_ptr())
    rc = L.pic1d_sort_static(65536 * 2, 4, *([p] * 10), p, None)
    assert rc == -1
