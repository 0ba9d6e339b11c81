"""Full-size parity at the workload shapes, through the C ABI, against the FP64
oracle and against FP64 runs of the CUDA path.

* 64^3, L = 27.33, N = 256, bare kernel (the differentiation workload): the
  FP32 gradient of E_x (Eq. EX) from the hand-written adjoint behind the
  autograd Function, against central differences of FP64 GPU energies along
  32 seeded directions (h = 1e-4), against the FP64 GPU gradient on the whole
  array, and the FP64 gradient's columns against the oracle.
* 48^3, L = 20.5, N = 128, 192 bands, screened kernel: every output of the
  build (W, M, Xi, E_x) and the apply against a full oracle build.
* The whole 64-system uneven batch in one ace_build_batched: every system
  bitwise equal to its own ace_build, sampled W columns of every system and
  E_x of the cheapest systems against the oracle.

Tolerances (Frobenius-relative) are those of the FP32 mode: 1e-6 on W and E_x,
1e-5 on M, Xi, the apply and the gradient (and the gradient within 1e-5 of the
finite differences); 1e-10 for FP64 storage.
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
    return t.detach().cpu().numpy().astype(np.complex128 if t.is_complex() else np.float64)


def _w_column(phi, i, kern):
    """W_i = -sum_j phi_j Poisson[conj(phi_j) phi_i] (Eq. W), one column."""
    return oracle.exchange_apply(phi, phi[i][None], kern)[0]


def test_diff64_gradient_against_fd_and_fp64(ace):
    s = synth.DIFF_64
    phi = synth.orbitals(s, synth.seed_for(4))
    kern = oracle.coulomb_kernel((s.n,) * 3, (s.L,) * 3, s.kernel, s.omega)
    plan32 = ace.Plan(s.n, s.L, s.n_occ, dtype="c64", kernel=s.kernel)
    plan64 = ace.Plan(s.n, s.L, s.n_occ, dtype="c128", kernel=s.kernel)
    phi64 = torch.from_numpy(phi).cuda()
    # FP32 forward + hand-written adjoint through the autograd Function
    p32 = phi64.to(torch.complex64).requires_grad_(True)
    e32 = ace.exchange_energy(p32, plan32)
    e32.backward()
    g32 = p32.grad.detach()
    assert plan32.status() == (0, 0)
    e64, g64 = plan64.energy_grad(phi64, grad=True)
    assert plan64.status() == (0, 0)
    assert abs(e32.item() - e64.item()) < 1e-6 * abs(e64.item())
    assert float(torch.linalg.vector_norm(g32.to(torch.complex128) - g64) / torch.linalg.vector_norm(g64)) < 1e-5
    G64 = _host(g64)
    for i in (0, 255):
        assert rel(G64[i], 2.0 * s.dv * _w_column(phi, i, kern)) < 1e-10, i
    # central differences of FP64 energies along 32 seeded directions with dV ||D||^2 = 1
    gen = torch.Generator(device="cuda").manual_seed(synth.seed_for(4, 77))
    h = 1e-4
    g32d = g32.to(torch.complex128)
    errs = []
    for _ in range(32):
        d = torch.complex(torch.randn(phi64.shape, generator=gen, device="cuda", dtype=torch.float64),
                          torch.randn(phi64.shape, generator=gen, device="cuda", dtype=torch.float64))
        d /= torch.sqrt(s.dv * torch.sum(torch.abs(d) ** 2))
        ep = plan64.energy_grad(phi64 + h * d)[0].item()
        em = plan64.energy_grad(phi64 - h * d)[0].item()
        fd = (ep - em) / (2 * h)
        an = float(torch.sum(g32d.conj() * d).real)
        errs.append(abs(fd - an) / abs(an))
        del d
    print(f"64^3 N=256: max FD rel error over 32 directions {max(errs):.3e}")
    assert max(errs) < 1e-5


def test_si64_full_size_against_full_oracle_build(ace):
    """The 48^3 workload in the launch configuration the bench times."""
    s = synth.SI64_48
    seed = synth.seed_for(2)
    phi = synth.orbitals(s, seed)
    psi = synth.targets(s, seed)
    kern = oracle.coulomb_kernel((s.n,) * 3, (s.L,) * 3, s.kernel, s.omega)
    ref = oracle.ace_build(phi, kern, s.dv)
    plan = ace.Plan(s.n, s.L, s.n_occ, dtype="c64", kernel=s.kernel, omega=s.omega)
    phi_d = torch.from_numpy(phi).to(torch.complex64).cuda()
    psi_d = torch.from_numpy(psi).to(torch.complex64).cuda()
    out = plan.build(phi_d)
    y = plan.apply(out["Xi"], psi_d)
    assert plan.status() == (0, 0)
    W = _host(out["W"])
    col = [rel(W[i], ref["W"][i]) for i in range(s.n_occ)]
    print(f"48^3 N=128: W columns max rel {max(col):.3e}")
    assert max(col) < 1e-6
    assert rel(W, ref["W"]) < 1e-6
    assert rel(_host(out["M"]), ref["M"]) < 1e-5
    assert rel(_host(out["Xi"]), ref["Xi"]) < 1e-5
    assert abs(out["Ex"].item() - ref["Ex"]) < 1e-6 * abs(ref["Ex"])
    assert rel(_host(y), oracle.ace_apply(ref["Xi"], psi, s.dv)) < 1e-5


def test_batched_full_draw(ace):
    """All 64 systems of the seeded uneven draw (edges in {32..64}, N in
    [16, 128], bare kernel, c64) in one ace_build_batched (Alg. 2 steps 2-3
    per system)."""
    draw = synth.batched_systems()
    assert len(draw) == 64
    phis_h, plans, phis = [], [], []
    for i, s in enumerate(draw):
        phi = synth.orbitals(s, synth.seed_for(3, i))
        phis_h.append(phi)
        plans.append(ace.Plan(s.n, s.L, s.n_occ, dtype="c64", kernel="bare"))
        phis.append(torch.from_numpy(phi).to(torch.complex64).cuda())
    batch = ace.Batch(plans)
    xis, ex = batch.build(phis)
    ex = ex.clone()
    for p in plans:
        assert p.status() == (0, 0)
    kerns = {}
    for i, (s, p) in enumerate(zip(draw, plans)):
        single = p.build(phis[i], want_m=False)
        assert torch.equal(single["Xi"], xis[i]), i
        assert single["Ex"].item() == ex[i].item(), i
        key = (s.n, s.L)
        if key not in kerns:
            kerns[key] = oracle.coulomb_kernel((s.n,) * 3, (s.L,) * 3, "bare", 0.0)
        W = single["W"]
        for c in (0, s.n_occ - 1):
            assert rel(_host(W[c]), _w_column(phis_h[i], c, kerns[key])) < 1e-6, (i, c)
        vphi = p.apply(xis[i], phis[i])                       # Eq. ACEcond
        assert float(torch.linalg.vector_norm(vphi - W) / torch.linalg.vector_norm(W)) < 1e-5, i
        del single, W, vphi
    cost = sorted(range(64), key=lambda i: draw[i].n_occ ** 2 * draw[i].ng)
    for i in cost[:8]:
        s = draw[i]
        ref_e = 0.5 * float(np.real(np.trace(oracle.overlap_M(
            phis_h[i], oracle.exchange_W(phis_h[i], kerns[(s.n, s.L)]), s.dv))))
        assert abs(ex[i].item() - ref_e) < 1e-6 * abs(ref_e), i
