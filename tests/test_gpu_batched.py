"""Batched ACE construction (many uneven systems in one captured graph) and the
autotuner, through the C ABI, against single-system builds and the FP64
oracle."""
import math

import numpy as np
import pytest

import oracle
from paper_1601_07159_gb300 import synth
from tests.conftest import rel

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL_XI = {"c64": 1e-5, "c128": 1e-10, "r64": 1e-10}
TOL_E = {"c64": 1e-6, "c128": 1e-10, "r64": 1e-10}


@pytest.fixture(scope="module")
def ace():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1601_07159_gb300 import build_lib
    build_lib.build()
    from paper_1601_07159_gb300 import ace as mod
    return mod


def _ecut(n, L):
    return min(synth.ECUT_HA, 0.3 * (math.pi * n / L) ** 2)


def _host(t):
    return t.detach().cpu().numpy().astype(np.complex128 if t.is_complex() else np.float64)


# n, L, N, dtype, kernel, omega: edges, orbital counts, dtypes and kernels all differ
SYSTEMS = [(16, 6.0, 5, "c64", "bare", 0.0), (20, 8.0, 9, "c64", "erfc", 0.3),
           (24, 10.0, 13, "c64", "bare", 0.0), (32, 10.0, 8, "c64", "bare", 0.0),
           (16, 6.0, 6, "c128", "erfc", 0.5), (12, 5.0, 3, "r64", "bare", 0.0),
           (24, 9.0, 1, "c64", "bare", 0.0)]


def _system(i, n, L, N, dtype, kernel, omega, ace):
    s = synth.System(n=n, L=L, n_occ=N, n_bands=N, real=(dtype == "r64"), kernel=kernel, omega=omega)
    phi = synth.orbitals(s, 7000 + i, ecut=_ecut(n, L))
    plan = ace.Plan(n, L, N, dtype=dtype, kernel=kernel, omega=omega)
    return s, phi, plan, torch.from_numpy(phi).to(ace.TORCH_DTYPES[dtype]).cuda()


@pytest.mark.parametrize("chains", [1, 3])
def test_batched_matches_single_builds_and_oracle(ace, chains):
    """Every system of the batch gets bitwise the Xi and E_x of its own
    ace_build (same kernels, same schedule), on capture and on replay; the
    graph reads the inputs at replay time; and each system matches the FP64
    oracle (Eq. Wtilde, Eq. EX with psi = phi)."""
    sys_ = [_system(i, *c, ace) for i, c in enumerate(SYSTEMS)]
    plans = [t[2] for t in sys_]
    phis = [t[3] for t in sys_]
    batch = ace.Batch(plans, chains=chains)
    xis = [p.empty(p.n_occ) for p in plans]
    for rep in range(2):                                     # capture, then replay
        batch.build(phis, xis)
        ex = batch.ex.clone()
        for i, (p, phi) in enumerate(zip(plans, phis)):
            single = p.build(phi, want_w=False, want_m=False)
            assert torch.equal(single["Xi"], xis[i]), (rep, i)
            assert single["Ex"].item() == ex[i].item(), (rep, i)
            assert p.status() == (0, 0)
    for i, (s, phi_h, p, _) in enumerate(sys_):
        n, L, N, dtype, kernel, omega = SYSTEMS[i]
        kern = oracle.coulomb_kernel((n, n, n), (L, L, L), kernel, omega)
        ref = oracle.ace_build(phi_h, kern, s.dv)
        assert rel(_host(xis[i]), ref["Xi"]) < TOL_XI[dtype], i
        assert rel(ex[i].item(), ref["Ex"]) < TOL_E[dtype], i
    # new data behind the same pointers: the replayed graph sees it
    phis[2].copy_(torch.flip(phis[2], dims=[0]))
    batch.build(phis, xis)
    single = plans[2].build(phis[2], want_w=False, want_m=False)
    assert torch.equal(single["Xi"], xis[2])


def test_batched_reports_device_failure_per_system(ace):
    """A system whose -M is singular (a zero orbital) reports NOT_POSDEF in its
    own plan's status word; the other systems of the batch are unaffected."""
    sys_ = [_system(i, *c, ace) for i, c in enumerate(SYSTEMS[:3])]
    plans = [t[2] for t in sys_]
    phis = [t[3] for t in sys_]
    phis[1][3].zero_()
    batch = ace.Batch(plans, chains=2)
    xis, ex = batch.build(phis)
    assert plans[1].status() == (ace.ACE_ERR_NOT_POSDEF, 4)
    for i in (0, 2):
        assert plans[i].status() == (0, 0)
        assert torch.equal(plans[i].build(phis[i], want_w=False, want_m=False)["Xi"], xis[i])


def test_batched_rejects_bad_batches(ace):
    p = ace.Plan(16, 6.0, 4)
    phi = p.empty(4)
    with pytest.raises(ace.AceError) as e:
        ace.Batch([p, p]).build([phi, phi])
    assert e.value.code == ace.ACE_ERR_ARG


def test_config3_draw_first_systems(ace):
    """The first systems of the seeded config-3 draw (edges in {32..64}, N in
    [16, 128], bare kernel, c64) at full size in one batch: bitwise equal to
    single builds, and each satisfies dV Xi^* Phi = -L^* (upper triangular,
    Eq. ACEcond) and 1/2 tr M = -1/2 ||dV Xi^* Phi||_F^2 (Eq. EX_ACE)."""
    draw = synth.batched_systems()[:6]
    plans, phis = [], []
    for i, s in enumerate(draw):
        phi = synth.orbitals(s, synth.seed_for(3, i))
        plans.append(ace.Plan(s.n, s.L, s.n_occ, dtype="c64", kernel="bare"))
        phis.append(torch.from_numpy(phi).to(torch.complex64).cuda())
    batch = ace.Batch(plans)
    xis, ex = batch.build(phis)
    for i, (s, p) in enumerate(zip(draw, plans)):
        single = p.build(phis[i], want_w=False, want_m=False)
        assert torch.equal(single["Xi"], xis[i]) and single["Ex"].item() == ex[i].item()
        A = s.dv * (xis[i].reshape(s.n_occ, -1).to(torch.complex128).conj() @
                    phis[i].reshape(s.n_occ, -1).to(torch.complex128).T)
        low = torch.tril(A, diagonal=-1)
        assert float(torch.linalg.norm(low) / torch.linalg.norm(A)) < 1e-5, i
        e_ace = -0.5 * float(torch.linalg.norm(A) ** 2)
        assert abs(e_ace - ex[i].item()) < 1e-5 * abs(ex[i].item()), i


def test_autotune_and_tuning_table(ace, tmp_path):
    """The autotuner returns a valid schedule with a measured time; a plan made
    from the tuning table (and reloaded from its JSON file) matches the oracle."""
    n, L, N = 16, 6.0, 12
    t = ace.autotune(n, L, N, "c64", "bare")
    assert t["tile"] in (4, 6, 8) and t["max_pairs"] >= t["tile"] ** 2 and t["ms"] > 0
    assert t["radix"] in (0, 1)                      # radix order is one of the searched knobs
    path = str(tmp_path / "tune.json")
    tab = ace.TuningTable(path)
    plan = tab.plan(n, L, N, "c64", "bare")
    tab2 = ace.TuningTable(path)
    assert ace.TuningTable.key(n, N, "c64", "bare") in tab2.table
    s = synth.System(n=n, L=L, n_occ=N, n_bands=N)
    phi = synth.orbitals(s, 4242, ecut=_ecut(n, L))
    out = plan.build(torch.from_numpy(phi).to(torch.complex64).cuda())
    kern = oracle.coulomb_kernel((n, n, n), (L, L, L), "bare", 0.0)
    ref = oracle.ace_build(phi, kern, s.dv)
    assert rel(_host(out["W"]), ref["W"]) < 1e-6
    assert rel(_host(out["Xi"]), ref["Xi"]) < 1e-5
    # plan creation consults the registered tuned schedule (the last ace_autotune,
    # the one behind the table's entry, registered it)
    t2 = tab2.table[ace.TuningTable.key(n, N, "c64", "bare")]
    default = ace.Plan(n, L, N, "c64", "bare").effective_schedule()
    assert (default["tile"], default["max_pairs"], default["overlap"]) == (t2["tile"], t2["max_pairs"], t2["overlap"])
    assert ace.TuningTable.key((n, n, n), N, "c64", "bare") == ace.TuningTable.key(n, N, "c64", "bare")
    ace.tuning_clear()
    ace.tuning_register(n, L, N, "c64", "bare", tile=4, max_pairs=48, lanes=3, overlap=False, radix=1)
    e = ace.Plan(n, L, N, "c64", "bare").effective_schedule()
    assert (e["tile"], e["max_pairs"], e["lanes"], e["overlap"], e["radix"]) == (4, 48, 3, False, 1)
    assert ace.Plan(n, L, N, "c64", "bare", tile=8).effective_schedule()["tile"] == 8   # explicit knobs win
    ace.tuning_clear()
    assert ace.Plan(n, L, N, "c64", "bare").effective_schedule()["tile"] == 8
