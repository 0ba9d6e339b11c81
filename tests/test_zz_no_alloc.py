"""ace_apply_static against ace_apply.

ace_apply_static serves callers that cannot allocate device memory or hand
over a workspace: it keeps the apply's scratch in the library's own static
device array. This test calls it through the C ABI twice in a row (different
targets the second time, so stale scratch contents would show) and compares
each result with the workspace-based ace_apply, within the apply tolerances
of the parity tests (1e-10 FP64, 1e-5 FP32). It also checks the size limit is
rejected before any work. It lives in a file of its own, collected last.
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


@pytest.mark.parametrize("dtype,tol", [("c64", 1e-5), ("c128", 1e-10)])
def test_static_apply_matches_workspace_apply(ace, dtype, tol):
    n, L, nocc, nb = 24, 10.0, 13, 9
    s = synth.System(n=n, L=L, n_occ=nocc, n_bands=nb, kernel="erfc", omega=0.3)
    ecut = 0.3 * (math.pi * n / L) ** 2
    td = ace.TORCH_DTYPES[dtype]
    phi = torch.from_numpy(synth.orbitals(s, 17, ecut=ecut)).to(td).cuda()
    plan = ace.Plan(n, L, nocc, dtype=dtype, kernel="erfc", omega=0.3)
    xi = plan.build(phi)["Xi"]
    assert plan.status() == (0, 0)
    lib = ace.lib()
    for call, seed in enumerate((5, 6)):
        psi = torch.from_numpy(synth.targets(s, seed, ecut=ecut)).to(td).cuda()
        want = plan.apply(xi, psi)
        got = torch.full_like(want, float("nan"))
        code = lib.ace_apply_static(plan._h, ctypes.c_void_p(xi.data_ptr()), ctypes.c_void_p(psi.data_ptr()),
                                    nb, ctypes.c_void_p(got.data_ptr()),
                                    ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
        assert code == ace.ACE_OK, lib.ace_last_error()
        torch.cuda.synchronize()
        err = float(torch.linalg.vector_norm(got - want) / torch.linalg.vector_norm(want))
        assert err < tol, (call, err)


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
