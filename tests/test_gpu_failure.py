"""Failure detection on the GPU in forms that fault, trap or hang nothing.

* A bounded device wait that runs out: the persistent engine's waits on other
  blocks' work are bounded; the debug hook asks each wait for one finished task
  more than exists, so every dependent wait runs out after a short poll limit.
  The launch ends by itself with ACE_ERR_TIMEOUT in the plan's status word and
  the context stays usable: the next call with the hook off matches the oracle.
* An allocation that fails: each of the plan set-up's device allocations in
  turn is made to fail; plan creation returns ACE_ERR_CUDA, releases what it
  had allocated, and a plan made afterwards works.
"""
import math

import numpy as np
import pytest

import oracle
from paper_1601_07159_gb300 import synth
from tests.conftest import rel

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


def _host(t):
    return t.detach().cpu().numpy().astype(np.complex128)


@pytest.mark.parametrize("graphs", [False, True])
def test_engine_wait_runs_out_and_recovers(ace, graphs):
    n, L, N, nb = 24, 10.0, 21, 10
    s = synth.System(n=n, L=L, n_occ=N, n_bands=nb, kernel="erfc", omega=0.3)
    ecut = 0.3 * (math.pi * n / L) ** 2
    phi = synth.orbitals(s, 8, ecut=ecut)
    psi = synth.targets(s, 8, ecut=ecut)
    kern = oracle.coulomb_kernel((n, n, n), (L, L, L), "erfc", 0.3)
    plan = ace.Plan(n, L, N, dtype="c64", kernel="erfc", omega=0.3, tile=4, max_pairs=16,
                    engine=True, graphs=graphs)
    phi_d = torch.from_numpy(phi).to(torch.complex64).cuda()
    psi_d = torch.from_numpy(psi).to(torch.complex64).cuda()
    plan.debug_engine_wait(polls=1000, unreachable=True)
    plan.exchange_apply(phi_d, psi_d)
    code, task = plan.status()
    assert code == ace.ACE_ERR_TIMEOUT and task >= 0
    plan.build(phi_d)                                  # the build's Cholesky keeps the first failure
    assert plan.status()[0] == ace.ACE_ERR_TIMEOUT
    plan.debug_engine_wait()                           # back to the default limit
    y = plan.exchange_apply(phi_d, psi_d)
    out = plan.build(phi_d)
    assert plan.status() == (0, 0)
    assert rel(_host(y), oracle.exchange_apply(phi, psi, kern)) < 1e-6
    assert rel(_host(out["W"]), oracle.exchange_W(phi, kern)) < 1e-6


def test_plan_allocation_failures_are_reported_and_released(ace):
    n, L, N = 16, 8.0, 12
    ace.Plan(n, L, N).close()                          # warm the context and the module
    torch.cuda.synchronize()
    ace.debug_fail_alloc(0)
    p = ace.Plan(n, L, N)
    count = ace.debug_fail_alloc(0)                    # allocations of one plan set-up
    p.close()
    assert count >= 5
    free0 = torch.cuda.mem_get_info()[0]
    for k in range(1, count + 1):
        ace.debug_fail_alloc(k)
        try:
            with pytest.raises(ace.AceError) as ei:
                ace.Plan(n, L, N)
        finally:
            ace.debug_fail_alloc(0)
        assert ei.value.code == ace.ACE_ERR_CUDA and "out of memory" in str(ei.value), k
    torch.cuda.synchronize()
    assert abs(torch.cuda.mem_get_info()[0] - free0) <= (2 << 20)
    s = synth.System(n=n, L=L, n_occ=N, n_bands=1)
    phi = synth.orbitals(s, 3, ecut=0.3 * (math.pi * n / L) ** 2)
    plan = ace.Plan(n, L, N)
    out = plan.build(torch.from_numpy(phi).to(torch.complex64).cuda())
    assert plan.status() == (0, 0)
    kern = oracle.coulomb_kernel((n, n, n), (L, L, L), "bare", 0.0)
    assert rel(_host(out["W"]), oracle.exchange_W(phi, kern)) < 1e-6
