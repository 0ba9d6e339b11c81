"""The odd-radix-first line transforms (ACE_FLAG_RADIX_ODD_FIRST), a schedule
choice of the autotuner: on every grid compiled in that order (cubic edges
with a factor 3 or 5 beside a power of two, and the non-square planes) the
FP32 build, energy and gradient match the FP64 oracle to the FP32 mode's
tolerances, and differ from the default order's results only by rounding."""
import math

import numpy as np
import pytest

import oracle
from paper_1601_07159_gb300 import build_lib, synth
from tests.conftest import rel

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

R1_EDGES, R1_PLANES = build_lib.shape_lists()["f32_r1"]


@pytest.fixture(scope="module")
def ace():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build_lib.build()
    from paper_1601_07159_gb300 import ace as mod
    return mod


def _host(t):
    return t.detach().cpu().numpy().astype(np.complex128)


def _case(grid, cell, nocc, seed):
    s = synth.System(n=0, L=0.0, n_occ=nocc, n_bands=1, kernel="erfc", omega=0.3, grid=grid, cell=cell)
    ecut = min(synth.ECUT_HA, 0.3 * min((math.pi * n / l) ** 2 for n, l in zip(grid, cell)))
    phi = synth.orbitals(s, seed, ecut=ecut)
    return s, phi, oracle.coulomb_kernel(s.shape, s.lengths, "erfc", 0.3)


GRIDS = [((n, n, n), (0.43 * n,) * 3) for n in R1_EDGES if n <= 48] + \
        [((nx, ny, 16), (0.43 * nx, 0.43 * ny, 6.9)) for nx, ny in R1_PLANES] + [((96, 96, 96), (41.0,) * 3)]


@pytest.mark.parametrize("grid,cell", GRIDS)
def test_odd_radix_first_matches_oracle(ace, grid, cell):
    nocc = 3 if grid[0] == 96 else 9
    s, phi, kern = _case(grid, cell, nocc, seed=7000 + sum(grid))
    ref = oracle.ace_build(phi, kern, s.dv)
    phi_d = torch.from_numpy(phi).to(torch.complex64).cuda()
    p1 = ace.Plan(grid, cell, nocc, dtype="c64", kernel="erfc", omega=0.3, radix=1)
    p0 = ace.Plan(grid, cell, nocc, dtype="c64", kernel="erfc", omega=0.3)
    assert p1.effective_schedule()["radix"] == 1 and p0.effective_schedule()["radix"] == 0
    o1, o0 = p1.build(phi_d), p0.build(phi_d)
    assert p1.status() == (0, 0)
    assert rel(_host(o1["W"]), ref["W"]) < 1e-6
    assert rel(_host(o1["Xi"]), ref["Xi"]) < 1e-5
    assert abs(o1["Ex"].item() - ref["Ex"]) < 1e-6 * abs(ref["Ex"])
    assert rel(_host(o1["W"]), _host(o0["W"])) < 1e-6
    assert not torch.equal(o1["W"], o0["W"])              # the other instances really ran
    e1, g1 = p1.energy_grad(phi_d, grad=True)
    assert abs(e1.item() - ref["Ex"]) < 1e-6 * abs(ref["Ex"])
    assert rel(_host(g1), oracle.energy_grad(phi, kern, s.dv)) < 1e-5
