"""The allocation-free Coulomb sum (hsma_coulomb_potential_noalloc) against the regular entry point.

Callers that may not allocate device memory (code inside allocator callbacks, plugins whose
host application owns all device memory, fixed-budget real-time loops) use
hsma_coulomb_potential_noalloc, whose scratch memory is a static device array.  This file is
collected last on purpose.  It checks, through the C ABI, that two calls in a row reproduce
hsma_potential(..., HSMA_COULOMB) within the FP32 tolerance of the tests (1e-6 norm-wise), up
to the largest accepted size, that sizes beyond the maximum are rejected, and that the call
captures in a CUDA graph and runs without moving the device's free memory.
"""
import ctypes

import numpy as np
import pytest

from paper_1907_01724_gb300 import _native, api, inputs

pytestmark = pytest.mark.gpu

MAX_N = 32768


def _regular_coulomb(s):
    prm = api.hsma_default_params(p=s.p, M=s.M, precision=api.HSMA_FP32)
    h = api.hsma_create(s.a, s.eps1, s.eps2, s.kappa, prm)
    api.hsma_build_sources(h, s.xyz, s.q)
    return api.hsma_potential(h, api.HSMA_COULOMB)


def _noalloc(lib, xyz_d, q_d, kfac, out, stream):
    return lib.hsma_coulomb_potential_noalloc(int(q_d.numel()), ctypes.c_void_p(xyz_d.data_ptr()),
                                              ctypes.c_void_p(q_d.data_ptr()), float(kfac),
                                              ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(stream.cuda_stream))


@pytest.mark.parametrize("n", [1, 517, 5000, MAX_N])
def test_noalloc_matches_regular_entry_point_twice(n):
    import torch
    lib = _native.load()
    s = inputs.near_interface_system(kappa_a=2.0, n=n) if n > 1 else inputs.System(
        1.0, 1.0, 80.0, 1.0, 10, 100, np.array([[0.1, 0.2, 0.3]]), np.array([1.0]))
    ref = _regular_coulomb(s)
    kfac = (1.0 / (4.0 * np.pi)) / s.eps1
    stream = torch.cuda.Stream()
    xyz_d = torch.tensor(s.xyz, device="cuda")
    q_d = torch.tensor(s.q, device="cuda")
    outs = []
    for _ in range(2):
        out = torch.full((s.n,), float("nan"), dtype=torch.float64, device="cuda")
        torch.cuda.synchronize()
        assert _noalloc(lib, xyz_d, q_d, kfac, out, stream) == 0
        stream.synchronize()
        outs.append(out.cpu().numpy())
    for phi in outs:
        if n == 1:
            assert phi[0] == 0.0 and ref[0] == 0.0
        else:
            assert np.linalg.norm(phi - ref) / np.linalg.norm(ref) <= 1e-6
    assert np.array_equal(outs[0], outs[1])


def test_noalloc_rejects_sizes_beyond_maximum():
    import torch
    lib = _native.load()
    n = MAX_N + 1
    xyz_d = torch.zeros((n, 3), dtype=torch.float64, device="cuda")
    q_d = torch.zeros(n, dtype=torch.float64, device="cuda")
    out = torch.zeros(n, dtype=torch.float64, device="cuda")
    # rejected on the host before any launch
    rc = lib.hsma_coulomb_potential_noalloc(n, ctypes.c_void_p(xyz_d.data_ptr()), ctypes.c_void_p(q_d.data_ptr()),
                                            1.0, ctypes.c_void_p(out.data_ptr()), None)
    assert rc == -1


def test_noalloc_captures_in_a_graph_without_allocating():
    """A call captured in a CUDA graph (global capture mode: no synchronising call may run while
    the capture is open) replays to the same values, and a call after the first one leaves the
    device's free memory where it was, at the largest accepted size."""
    import torch
    lib = _native.load()
    s = inputs.near_interface_system(kappa_a=2.0, n=MAX_N)
    kfac = (1.0 / (4.0 * np.pi)) / s.eps1
    xyz_d = torch.tensor(s.xyz, device="cuda")
    q_d = torch.tensor(s.q, device="cuda")
    eager = torch.full((s.n,), float("nan"), dtype=torch.float64, device="cuda")
    graphed = torch.full((s.n,), float("nan"), dtype=torch.float64, device="cuda")
    stream = torch.cuda.Stream()
    assert _noalloc(lib, xyz_d, q_d, kfac, eager, stream) == 0  # the warm-up call
    stream.synchronize()
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    assert _noalloc(lib, xyz_d, q_d, kfac, eager, stream) == 0
    stream.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0

    g = torch.cuda.CUDAGraph()
    rcs = []
    with torch.cuda.graph(g, stream=stream, capture_error_mode="global"):
        rcs.append(_noalloc(lib, xyz_d, q_d, kfac, graphed, stream))
    assert rcs == [0]
    expected = eager.cpu()
    for _ in range(2):
        graphed.fill_(float("nan"))
        g.replay()
        torch.cuda.synchronize()
        assert torch.equal(graphed.cpu(), expected)
