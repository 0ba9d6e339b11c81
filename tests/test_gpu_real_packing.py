"""Real vectors (r64): two pair solves per complex FFT.

For real orbitals the pair densities rho_lr = phi_l phi_r are real and the
kernel K(G) is real and even, so V_lr = F^-1[K F rho_lr] is real: one complex
solve of rho_lr + i rho_lr2 gives V_lr and V_lr2 as its real and imaginary
parts (Sec. 2, the Gamma-point case). The schedule packs the pairs (l, r),
(l, r + 1) of a tile row into one scratch slot; on a diagonal tile the pair
(l, l) keeps a slot of its own, so the energy weights of a slot's pairs agree.
These tests run the packed path on every tile shape (full and ragged
diagonal and off-diagonal tiles, odd right-hand blocks, one-sided tiles with
odd target counts), in every launch mode, against the FP64 oracle, and check
that the real schedule needs half the batches of the complex one.
"""
import math

import numpy as np
import pytest

import oracle
from paper_1601_07159_gb300 import synth
from tests.conftest import rel

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-10


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
    return t.detach().cpu().numpy().astype(np.float64)


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(torch.float64).cuda()


# n, L, N, n_b, tile, max_pairs, engine, graphs
CASES = [
    (16, 7.0, 19, 7, 8, 0, False, True),     # tiles 8, 8, 3: full and ragged, odd n_r = 3
    (16, 7.0, 19, 7, 6, 40, False, False),   # tile 6 (18 and 15 slots), 7 = 6 + 1, eager
    (20, 8.0, 13, 5, 4, 0, True, True),      # persistent engine, tile 4
    (12, 6.0, 1, 1, 8, 0, False, True),      # one orbital: a single diagonal slot
    (12, 6.0, 2, 3, 8, 0, True, False),      # N = 2: the slot (0, 0) and the slot (0, 1) + (1, 1) apart
    (24, 10.0, 17, 9, 8, 64, False, True),   # two full off-diagonal tiles in one batch (32 slots each)
]


@pytest.mark.parametrize("n,L,nocc,nb,tile,max_pairs,engine,graphs", CASES)
def test_real_packed_matches_oracle(ace, n, L, nocc, nb, tile, max_pairs, engine, graphs):
    s = synth.System(n=n, L=L, n_occ=nocc, n_bands=nb, real=True, kernel="bare", omega=0.0)
    phi = synth.orbitals(s, 9100 + nocc, ecut=_ecut(n, L))
    psi = synth.targets(s, 9100 + nocc, ecut=_ecut(n, L))
    kern = oracle.coulomb_kernel((n, n, n), (L, L, L), "bare", 0.0)
    ref = oracle.ace_build(phi, kern, s.dv)
    plan = ace.Plan(n, L, nocc, dtype="r64", kernel="bare", tile=tile, max_pairs=max_pairs, engine=engine,
                    graphs=graphs)
    phi_d, psi_d = _dev(phi), _dev(psi)

    out = plan.build(phi_d)
    assert plan.status() == (0, 0)
    assert rel(_host(out["W"]), ref["W"].real) < TOL
    assert rel(_host(out["M"]), ref["M"].real) < TOL
    assert rel(_host(out["Xi"]), ref["Xi"].real) < TOL
    assert abs(out["Ex"].item() - ref["Ex"]) < TOL * abs(ref["Ex"])

    y = plan.exchange_apply(phi_d, psi_d)                     # one-sided tiles, n_b odd
    assert rel(_host(y), oracle.exchange_apply(phi, psi, kern).real) < TOL

    e_direct = oracle.energy_direct(phi, kern, s.volume)
    g_ref = oracle.energy_grad(phi, kern, s.dv).real
    ex, g = plan.energy_grad(phi_d, grad=True)
    assert abs(ex.item() - e_direct) < TOL * abs(e_direct)
    assert rel(_host(g), g_ref) < TOL
    ex_s, _ = plan.energy_grad(phi_d, grad=False, recompute=False)   # store the packed potentials
    ex_g, g_s = plan.energy_grad(phi_d, grad=True, recompute=False)  # gradient from the store
    assert abs(ex_s.item() - e_direct) < TOL * abs(e_direct)
    assert rel(_host(g_s), g_ref) < TOL


def test_real_schedule_halves_batches(ace):
    """32 orbitals, tile 8, 64 slots per batch: the complex schedule runs 10
    batches (6 off-diagonal tiles of 64 pairs, 4 diagonal tiles of 36), the
    real one 5 (two 32-slot off-diagonal tiles or two 24-slot diagonal tiles
    per batch)."""
    n, L, N = 12, 6.0, 32
    counts = {}
    for dtype in ("c128", "r64"):
        plan = ace.Plan(n, L, N, dtype=dtype, kernel="bare", tile=8, max_pairs=64, graphs=False)
        s = synth.System(n=n, L=L, n_occ=N, n_bands=N, real=(dtype == "r64"))
        phi = synth.orbitals(s, 77, ecut=_ecut(n, L))
        phi_d = torch.from_numpy(phi).to(ace.TORCH_DTYPES[dtype]).cuda()
        plan.build(phi_d)                                          # schedules and kernels warm
        plan.profile_begin()
        plan.build(phi_d, want_w=False, want_m=False)
        counts[dtype] = plan.profile_end()["batches"]
    assert counts == {"c128": 10, "r64": 5}, counts


def test_real_matches_complex_path(ace):
    """The same real orbitals through the packed real path and the complex
    FP64 path (one pair per solve) give the same W, Xi and E_x to 1e-12."""
    n, L, N = 16, 7.0, 11
    s = synth.System(n=n, L=L, n_occ=N, n_bands=N, real=True)
    phi = synth.orbitals(s, 31, ecut=_ecut(n, L))
    r = ace.Plan(n, L, N, dtype="r64", kernel="bare").build(_dev(phi))
    c = ace.Plan(n, L, N, dtype="c128", kernel="bare").build(torch.from_numpy(phi).to(torch.complex128).cuda())
    assert rel(_host(r["W"]), c["W"].cpu().numpy()) < 1e-12
    assert rel(_host(r["Xi"]), c["Xi"].cpu().numpy()) < 1e-12
    assert abs(r["Ex"].item() - c["Ex"].item()) < 1e-12 * abs(c["Ex"].item())
