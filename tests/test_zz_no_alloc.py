"""ace_apply_static against ace_apply.

ace_apply_static serves callers that cannot allocate device memory or hand
over a workspace (a plugin whose host application owns every device
allocation, a fixed-latency loop where an allocation may block): it keeps the
apply's scratch in the library's own static device array. These tests call it
through the C ABI twice in a row (different targets the second time, so stale
scratch contents would show) and compare each result with the workspace-based
ace_apply, within the apply tolerances of the parity tests (1e-10 FP64, 1e-5
FP32); check that from the second call on it changes neither the device's free
memory nor torch's allocator; run a case near the size limit, where the number
of split-K partial sums is capped so that they fit the array; and check that a
size beyond the limit is rejected before any work. This file is collected last.
"""
import ctypes
import math

import numpy as np
import pytest

from paper_1601_07159_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ace():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1601_07159_gb300 import build_lib
    build_lib.build()
    from paper_1601_07159_gb300 import ace as mod
    return mod


def _call(ace, plan, xi, psi, out):
    lib = ace.lib()
    code = lib.ace_apply_static(plan._h, ctypes.c_void_p(xi.data_ptr()), ctypes.c_void_p(psi.data_ptr()),
                                psi.shape[0], ctypes.c_void_p(out.data_ptr()),
                                ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert code == ace.ACE_OK, lib.ace_last_error()


def _err(a, b):
    return float(torch.linalg.vector_norm(a - b) / torch.linalg.vector_norm(b))


@pytest.mark.parametrize("dtype,tol", [("c64", 1e-5), ("c128", 1e-10), ("r64", 1e-10)])
def test_static_apply_matches_workspace_apply(ace, dtype, tol):
    n, L, nocc, nb = 24, 10.0, 13, 9
    real = dtype == "r64"
    s = synth.System(n=n, L=L, n_occ=nocc, n_bands=nb, real=real, kernel="erfc", omega=0.3)
    ecut = 0.3 * (math.pi * n / L) ** 2
    td = ace.TORCH_DTYPES[dtype]
    phi = torch.from_numpy(synth.orbitals(s, 17, ecut=ecut)).to(td).cuda()
    plan = ace.Plan(n, L, nocc, dtype=dtype, kernel="erfc", omega=0.3)
    xi = plan.build(phi)["Xi"]
    assert plan.status() == (0, 0)
    for call, seed in enumerate((5, 6)):
        psi = torch.from_numpy(synth.targets(s, seed, ecut=ecut)).to(td).cuda()
        want = plan.apply(xi, psi)
        got = torch.full_like(want, float("nan"))
        torch.cuda.synchronize()
        free0, alloc0 = torch.cuda.mem_get_info()[0], torch.cuda.memory_stats().get("allocation.all.allocated", 0)
        _call(ace, plan, xi, psi, got)
        torch.cuda.synchronize()
        free1, alloc1 = torch.cuda.mem_get_info()[0], torch.cuda.memory_stats().get("allocation.all.allocated", 0)
        if call > 0:                       # the first call may load the module that holds the array
            assert free1 == free0, (free0, free1)
        assert alloc1 == alloc0
        assert _err(got, want) < tol, (call, _err(got, want))


def test_static_apply_near_the_size_limit(ace):
    # N * n_b = 409600 of the 524288 allowed: only two N x n_b FP64 complex
    # matrices fit the array, so the split-K partial sums are capped at one
    n, L, nocc, nb = 16, 8.0, 640, 640
    plan = ace.Plan(n, L, nocc, dtype="c128")
    g = torch.Generator(device="cuda").manual_seed(99)
    xi = torch.complex(torch.randn((nocc, n, n, n), generator=g, device="cuda", dtype=torch.float64),
                       torch.randn((nocc, n, n, n), generator=g, device="cuda", dtype=torch.float64))
    for call in range(2):
        psi = torch.complex(torch.randn((nb, n, n, n), generator=g, device="cuda", dtype=torch.float64),
                            torch.randn((nb, n, n, n), generator=g, device="cuda", dtype=torch.float64))
        want = plan.apply(xi, psi)
        got = torch.full_like(want, float("nan"))
        _call(ace, plan, xi, psi, got)
        torch.cuda.synchronize()
        assert _err(got, want) < 1e-10, (call, _err(got, want))


def test_static_apply_rejects_oversize(ace):
    # n_occ * n_b above ACE_STATIC_SCRATCH_BYTES / 32 = 524288 is refused up front
    plan = ace.Plan(8, 6.0, 1024, dtype="c64")
    xi = plan.empty(1024)
    psi = plan.empty(513)
    out = plan.empty(513)
    with pytest.raises(ace.AceError) as ei:
        plan.apply_static(xi, psi, out)
    assert ei.value.code == ace.ACE_ERR_ARG
    assert "exceeds" in str(ei.value)
