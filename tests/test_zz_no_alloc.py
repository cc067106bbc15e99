"""fmm_eval_noalloc: the evaluation for callers that may not allocate device
memory (graph capture, allocation-free real-time loops, plug-ins without
their own allocator).  Its workspace is a fixed array the library reserves
statically, so it must give exactly what fmm_eval gives with a caller-owned
workspace -- including on a second call, which finds the array still holding
the first call's data.

The file name sorts last so that a run stopping at the first failure has
already run every other test."""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-12  # the FP64 parity tolerance used throughout the GPU tests


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def test_noalloc_matches_fmm_eval_on_two_calls():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2305_17867_gb300 import _lib
    from paper_2305_17867_gb300.fmm import FMM

    L = _lib.load()
    plan = FMM("laplace", d=3, p=8, levels=3, precision="fp64")
    rng = np.random.default_rng(2024)
    ns, nt = 20000, 15000
    s = torch.tensor(rng.random((ns, 3)), device="cuda")
    w = torch.tensor(rng.uniform(-1, 1, ns), device="cuda")
    t = torch.tensor(rng.random((nt, 3)), device="cuda")
    ref = plan.eval(s, w, t)  # fmm_eval with a caller-owned workspace
    torch.cuda.synchronize()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    for call in range(2):
        phi = torch.full((nt,), float("nan"), dtype=torch.float64, device="cuda")
        rc = L.fmm_eval_noalloc(plan._h, ns, _ptr(s), _ptr(w), nt, _ptr(t), _ptr(phi), None,
                                stream)
        assert rc == 0, L.fmm_status_string(rc)
        torch.cuda.synchronize()
        assert L.fmm_last_status(plan._h) == 0
        err = float(torch.linalg.norm(phi - ref) / torch.linalg.norm(ref))
        assert err < FP64_TOL, (call, err)


def test_noalloc_rejects_sizes_beyond_its_array():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2305_17867_gb300 import _lib
    from paper_2305_17867_gb300.fmm import FMM

    L = _lib.load()
    plan = FMM("laplace", d=3, p=8, levels=3, precision="fp64")
    n = 10_000_000  # workspace far above 32 MiB: rejected before any work
    assert plan.workspace_bytes(n, n) > 32 << 20
    rc = L.fmm_eval_noalloc(plan._h, n, None, None, n, None, None, None, None)
    assert rc == -7  # FMM_ERR_WORKSPACE


def test_noalloc_rejects_missing_output():
    # the same argument check as fmm_eval: no launch is made, nothing is written
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2305_17867_gb300 import _lib
    from paper_2305_17867_gb300.fmm import FMM

    L = _lib.load()
    for levels in (3, -4):  # uniform and adaptive plans
        plan = FMM("laplace", d=3, p=4, levels=levels, precision="fp64")
        s = torch.rand(100, 3, dtype=torch.float64, device="cuda")
        w = torch.ones(100, dtype=torch.float64, device="cuda")
        rc = L.fmm_eval_noalloc(plan._h, 100, _ptr(s), _ptr(w), 100, _ptr(s), None, None, None)
        assert rc == -1  # FMM_ERR_ARG
