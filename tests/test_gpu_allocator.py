"""The library's device memory from a caller's allocator (pic1d_set_allocator
with PyTorch's caching allocator): the buffers appear in PyTorch's pool and
leave it when the line is freed, and the line's results do not depend on
where its memory came from."""
import numpy as np
import pytest

from paper_2609_17661_b300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _run(cfg, st):
    from paper_2609_17661_b300 import Line
    line = Line(cfg)
    line.set_state(st)
    line.step(12)
    E, J = line.fields()
    p = line.particles()
    o = np.argsort(p["id"])
    return line, E, J, {k: v[o] for k, v in p.items()}


def test_torch_allocator_hooks():
    from paper_2609_17661_b300 import PicError, use_torch_allocator
    cfg = W.config("C1", capacity=300_000, drag_scale=3e-3)
    st = W.load_drifting_plasma(cfg)
    ref, E0, J0, p0 = _run(cfg, st)
    with pytest.raises(PicError):          # a context is alive
        use_torch_allocator(True)
    ref.close()
    import gc
    gc.collect()                           # lines of earlier tests that are no longer referenced
    torch.cuda.synchronize()
    base = torch.cuda.memory_allocated()
    use_torch_allocator(True)
    try:
        line, E1, J1, p1 = _run(cfg, st)
        # both particle buffers (21 B per slot each) now sit in PyTorch's pool
        assert torch.cuda.memory_allocated() - base >= 2 * 21 * 300_000
        np.testing.assert_array_equal(E1, E0)
        np.testing.assert_array_equal(J1, J0)
        for f in ("id", "pos", "u", "w", "sp"):
            np.testing.assert_array_equal(p1[f], p0[f])
        line.close()
        torch.cuda.synchronize()
        assert torch.cuda.memory_allocated() == base
    finally:
        use_torch_allocator(False)


def test_allocator_that_refuses_gives_enomem():
    """A caller's allocator that runs out (returns NULL) makes pic1d_init fail
    with PIC1D_ENOMEM, after it has handed back every buffer it did get; the
    process is left able to make lines again once the hooks are restored."""
    import ctypes as C
    import gc

    from paper_2609_17661_b300 import Line, PicError, _lib
    from paper_2609_17661_b300 import _ALLOC_FN, _FREE_FN
    L = _lib.load()
    gc.collect()
    torch.cuda.synchronize()
    given, freed = [], []
    budget = [12]                      # the first 12 requests succeed, then the pool is "full"

    def alloc(n, user):
        if budget[0] <= 0:
            return None
        budget[0] -= 1
        p = torch.cuda.caching_allocator_alloc(int(n))
        given.append(p)
        return p

    def free(p, user):
        freed.append(p)
        torch.cuda.caching_allocator_delete(p)

    hooks = (_ALLOC_FN(alloc), _FREE_FN(free))
    assert L.pic1d_set_allocator(C.cast(hooks[0], C.c_void_p), C.cast(hooks[1], C.c_void_p), None) == 0
    try:
        with pytest.raises(PicError) as e:
            Line(W.config("C1"))
        assert e.value.code == -2                       # PIC1D_ENOMEM
        assert budget[0] == 0 and len(given) == 12
        assert sorted(freed) == sorted(given)           # nothing leaked
    finally:
        assert L.pic1d_set_allocator(None, None, None) == 0
    line = Line(W.config("C1"))                         # cudaMalloc again
    line.close()
