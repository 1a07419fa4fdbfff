"""Allocation-free coherence entry point, trstmi_mu2_frame_noalloc.

Callers whose device memory belongs to another allocator, or that cannot
afford the implicit synchronisation of cudaMalloc / cudaFree, use this entry
point: it keeps its scratch in a static device array and allocates nothing.
It must give the same binary64 mu^2 as the allocating entry point,
trstmi_mu2_frame, within the binary64 tolerance of the other parity tests
(1e-12 relative).  The array keeps the previous call's contents, so the
checks run as consecutive calls, a larger problem followed by smaller ones
and back, which fails if anything that must start at zero leaks between
calls.  This file is collected last so that a run stopping at the first
failure has already run every other test.
"""
import ctypes

import numpy as np
import pytest

import frames as F

pytestmark = pytest.mark.gpu

T = pytest.importorskip("paper_2207_06374_gb300.trstmi")
torch = pytest.importorskip("torch")


def _noalloc_mu2(phi, stream_handle):
    d, N = phi.shape
    dev = torch.from_numpy(T._flat(phi)).to("cuda")
    out = torch.full((1,), -1.0, dtype=torch.float64, device="cuda")
    torch.cuda.synchronize()
    st = T.lib().trstmi_mu2_frame_noalloc(N, d, ctypes.c_void_p(dev.data_ptr()),
                                          ctypes.c_void_p(out.data_ptr()),
                                          ctypes.c_void_p(stream_handle))
    assert st == T.TRSTMI_OK, T.strerror(st)
    torch.cuda.synchronize()
    return float(out.item())


def test_noalloc_matches_allocating_entry_point_on_consecutive_calls():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    rng = np.random.default_rng(2026)
    frames = [F.random_frame(32, 1024, rng), F.random_frame(8, 300, rng), F.hesse_sic_3_9(),
              F.random_frame(5, 77, rng), F.random_frame(64, 2048, rng)]
    stream = torch.cuda.current_stream().cuda_stream
    refs = [T.mu2_frame(phi, "fp64") for phi in frames]
    for order in (range(len(frames)), reversed(range(len(frames)))):
        for i in order:
            got = _noalloc_mu2(frames[i], stream)
            assert abs(got - refs[i]) <= 1e-12 * refs[i], (i, got, refs[i])
    # the same frame twice in a row gives the same bits
    a = _noalloc_mu2(frames[1], stream)
    b = _noalloc_mu2(frames[1], stream)
    assert a == b


def test_noalloc_rejects_sizes_beyond_its_limit():
    # rejected before any device pointer is used
    st = T.lib().trstmi_mu2_frame_noalloc(131073, 1, ctypes.c_void_p(8), ctypes.c_void_p(8), None)
    assert st == T.TRSTMI_ESIZE
    st = T.lib().trstmi_mu2_frame_noalloc(4, 300, ctypes.c_void_p(8), ctypes.c_void_p(8), None)
    assert st == T.TRSTMI_EINVAL
