"""Orthorhombic cells on n_x x n_y x n_z grids (Sec. 2: a plane-wave basis on
the grid of a periodic cell) through the C ABI against the FP64 oracle, which
builds K(G) and the Poisson solves per axis: the ACE build (W, M, Xi, E_x),
the exchange apply, the ACE apply, the direct energy and gradient, and the
Poisson entry, for non-square planes (12 x 16, 48 x 40, 24 x 16) and square
planes with another pencil length (16 x 16 x 64, 40 x 48 x 96), in every
dtype."""
import math

import numpy as np
import pytest

import oracle
from paper_1601_07159_gb300 import synth
from tests.conftest import rel

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = {"c128": dict(w=1e-10, m=1e-10, xi=1e-10, y=1e-10, e=1e-10, g=1e-10),
       "r64": dict(w=1e-10, m=1e-10, xi=1e-10, y=1e-10, e=1e-10, g=1e-10),
       "c64": dict(w=1e-6, m=1e-5, xi=1e-5, y=1e-6, e=1e-6, g=1e-5)}


@pytest.fixture(scope="module")
def ace():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1601_07159_gb300 import build_lib
    build_lib.build()
    from paper_1601_07159_gb300 import ace as mod
    return mod


def _host(t):
    return t.detach().cpu().numpy().astype(np.complex128 if t.is_complex() else np.float64)


CASES = [
    # grid (n_x, n_y, n_z), cell (L_x, L_y, L_z), N, n_b, dtype, kernel, omega
    ((12, 16, 20), (6.0, 8.0, 10.0), 7, 3, "c64", "erfc", 0.3),
    ((12, 16, 20), (6.0, 8.0, 10.0), 9, 2, "c128", "bare", 0.0),
    ((12, 16, 20), (6.0, 8.0, 10.0), 5, 2, "r64", "bare", 0.0),
    ((48, 40, 36), (20.5, 17.08, 15.375), 11, 3, "c64", "erfc", 0.106),
    ((48, 40, 36), (20.5, 17.08, 15.375), 3, 2, "c128", "erfc", 0.106),
    ((24, 16, 12), (10.0, 7.0, 5.0), 10, 4, "c64", "bare", 0.0),
    ((16, 16, 64), (7.0, 7.0, 27.3), 9, 2, "c64", "bare", 0.0),
    ((40, 48, 96), (17.08, 20.5, 41.0), 3, 2, "c64", "erfc", 0.106),
]


@pytest.mark.parametrize("grid,cell,nocc,nb,dtype,kernel,omega", CASES)
def test_orthorhombic_parity(ace, grid, cell, nocc, nb, dtype, kernel, omega):
    s = synth.System(n=0, L=0.0, n_occ=nocc, n_bands=nb, real=(dtype == "r64"), kernel=kernel, omega=omega,
                     grid=grid, cell=cell)
    ecut = min(synth.ECUT_HA, 0.3 * min((math.pi * n / l) ** 2 for n, l in zip(grid, cell)))
    seed = 5200 + sum(grid)
    phi = synth.orbitals(s, seed, ecut=ecut)
    psi = synth.targets(s, seed, ecut=ecut)
    kern = oracle.coulomb_kernel(s.shape, s.lengths, kernel, omega)
    ref = oracle.ace_build(phi, kern, s.dv)
    tol = TOL[dtype]
    assert ace.supported_grid(grid, dtype)
    plan = ace.Plan(grid, cell, nocc, dtype=dtype, kernel=kernel, omega=omega)
    td = ace.TORCH_DTYPES[dtype]
    phi_d = torch.from_numpy(phi).to(td).cuda()
    psi_d = torch.from_numpy(psi).to(td).cuda()
    out = plan.build(phi_d)
    assert plan.status() == (0, 0)
    assert rel(_host(out["W"]), ref["W"]) < tol["w"]
    m_ref = ref["M"].real if dtype == "r64" else ref["M"]
    assert rel(_host(out["M"]), m_ref) < tol["m"]
    assert rel(_host(out["Xi"]), ref["Xi"]) < tol["xi"]
    assert abs(out["Ex"].item() - ref["Ex"]) < tol["e"] * abs(ref["Ex"])
    y = plan.exchange_apply(phi_d, psi_d)
    assert rel(_host(y), oracle.exchange_apply(phi, psi, kern)) < tol["y"]
    ya = plan.apply(out["Xi"], psi_d)
    assert rel(_host(ya), oracle.ace_apply(ref["Xi"], psi, s.dv)) < tol["xi"]
    ex, g = plan.energy_grad(phi_d, grad=True)
    e_direct = oracle.energy_direct(phi, kern, s.volume)
    assert abs(ex.item() - e_direct) < tol["e"] * abs(e_direct)
    assert rel(_host(g), oracle.energy_grad(phi, kern, s.dv)) < tol["g"]
    v = plan.poisson(psi_d)
    v_ref = oracle.poisson(psi, kern)
    if dtype == "r64":
        v_ref = v_ref.real
    assert rel(_host(v), v_ref) < tol["w"]


def test_unlisted_plane_is_refused(ace):
    assert not ace.supported_grid((12, 20, 16), "c64")
    with pytest.raises(ace.AceError) as ei:
        ace.Plan((12, 20, 16), (6.0, 10.0, 8.0), 4)
    assert ei.value.code == ace.ACE_ERR_UNSUPPORTED
