"""Caller-supplied device allocator (trstmi_options.dev_alloc / dev_free).

A handle created with an allocator takes every device allocation from it: an
instance's state block and temporary buffers, a batch's arena and launch
plan, a server's tables and arena.  The tests back the callbacks with
PyTorch's caching allocator (the binding's TorchAllocator) and check that
(1) results are bit-identical to the same handle on cudaMalloc, (2) memory
went through the callbacks and all of it came back at destroy, (3) a
callback that fails makes creation return TRSTMI_ENOMEM, (4) an allocator
without its release callback is refused, and (5) the calls leave the
caller's current device as they found it.
"""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

T = pytest.importorskip("paper_2207_06374_gb300.trstmi")
torch = pytest.importorskip("torch")


def _need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")


@pytest.mark.parametrize("precision", ["fp32", "bf16"])
def test_search_on_torch_memory_equals_search_on_cudamalloc(precision):
    _need_gpu()
    alloc = T.TorchAllocator(0)
    before = torch.cuda.memory_allocated(0)
    kw = dict(K=64, precision=precision, screen_min_delta=0.0)
    with T.Search(300, 16, 5, **kw) as ref:
        ref.step(6)
        ref_tr, ref_phi = ref.trace(), ref.get_phi()
        ref_s = ref.score(2, 0, 8, 0.1, "fp32")
    with T.Search(300, 16, 5, allocator=alloc, **kw) as s:
        assert alloc.allocs >= 1 and alloc.live
        assert torch.cuda.memory_allocated(0) > before   # the block sits in torch's pool
        s.step(6)
        tr, phi = s.trace(), s.get_phi()
        sc = s.score(2, 0, 8, 0.1, "fp32")             # temporary buffer through the hook
        s.certificates()
    assert np.array_equal(tr, ref_tr)
    assert np.array_equal(phi, ref_phi)
    assert np.array_equal(sc, ref_s)
    assert alloc.frees == alloc.allocs and not alloc.live
    assert torch.cuda.memory_allocated(0) == before


def test_batch_and_server_on_torch_memory():
    _need_gpu()
    alloc = T.TorchAllocator(0)
    Ns, ds, seeds = [20, 300, 9], [4, 16, 3], [1, 2, 3]
    with T.Batch(Ns, ds, seeds, K=32, precision="fp32") as ref:
        ref.step(5)
        ref_mu = ref.mu()[0]
    with T.Batch(Ns, ds, seeds, K=32, precision="fp32", allocator=alloc) as b:
        assert alloc.allocs >= 2   # arena and launch plan
        b.step(5)
        mu = b.mu()[0]
    assert np.array_equal(mu, ref_mu)
    assert alloc.frees == alloc.allocs and not alloc.live

    alloc2 = T.TorchAllocator(0)
    with T.Server(hbm_budget=64 << 20, max_slots=8, iters_per_round=5, K=32, precision="fp32",
                  allocator=alloc2) as srv:
        assert alloc2.allocs >= 3   # tables, arena, plan
        t = srv.submit(40, 4, 11, 10)
        st, res, _ = srv.wait(t, 60000)
        assert st == T.TRSTMI_OK and res.iters == 10
    assert alloc2.frees == alloc2.allocs and not alloc2.live
    with T.Search(40, 4, 11, K=32, precision="fp32") as s:
        info = s.step(10)
    assert res.mu == info.mu


def test_failing_or_incomplete_allocator_is_reported():
    _need_gpu()
    fail = T.DEV_ALLOC_FN(lambda n, ctx: None)
    nop = T.DEV_FREE_FN(lambda p, ctx: None)
    o = T.make_options(K=16, precision="fp32")
    o.dev_alloc, o.dev_free = fail, nop
    h = ctypes.c_void_p()
    assert T.lib().trstmi_create(64, 4, 1, ctypes.byref(o), ctypes.byref(h)) == T.TRSTMI_ENOMEM
    assert not h.value
    o2 = T.make_options(K=16, precision="fp32")
    o2.dev_alloc = fail   # no release callback
    assert T.lib().trstmi_create(64, 4, 1, ctypes.byref(o2), ctypes.byref(h)) == T.TRSTMI_EINVAL


def test_entry_points_leave_the_callers_device_current():
    _need_gpu()
    torch.cuda.set_device(0)
    n = torch.cuda.device_count()
    with T.Search(64, 4, 3, K=16, precision="fp32", device=n - 1) as s:
        s.step(2)
        s.coherence()
        assert torch.cuda.current_device() == 0
    assert torch.cuda.current_device() == 0
    # a device that does not exist is refused, and the current device stays
    o = T.make_options(K=16, precision="fp32", device=n)
    h = ctypes.c_void_p()
    assert T.lib().trstmi_create(64, 4, 1, ctypes.byref(o), ctypes.byref(h)) == T.TRSTMI_EINVAL
    assert torch.cuda.current_device() == 0
    # the stateless entry points run on the caller's current device
    phi = np.linalg.qr(np.random.default_rng(1).standard_normal((8, 8)))[0][:, :6].astype(complex)
    assert abs(T.mu2_frame(phi, "fp64")) < 1e-28
    assert torch.cuda.current_device() == 0
