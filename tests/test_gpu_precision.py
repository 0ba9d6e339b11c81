"""Dense-step precision modes and the vector stride, through the C ABI.

* Xi = W L^{-*} (Eq. Wtilde) to FP64 accuracy in the FP32 mode: the FP16
  tensor-core slice product (ACE_PREC_XI_FP64, the C64 default) against plain
  FP64 arithmetic on CUDA cores (ACE_PREC_XI_FP64_SIMT) with the same W and
  L^{-*}: within one FP32 rounding of each other when stored in FP32, and
  within 1e-10 (relative) in FP64 output; both against the FP64 oracle. On an
  ill-conditioned -M the TF32-split product (ACE_PREC_SPLIT_TF32) drifts from
  the FP64 product while the slice product does not.
* ACE_PREC_SPLIT_BF16: M and the apply on BF16 tensor cores (hi/lo split),
  against the oracle with their measured error.
* ACE_PREC_FP32 is the CUDA-core FP32 path (bitwise the legacy flag).
* A leading dimension ld > N_g: every entry point gives bitwise the packed
  results, and the elements between N_g and ld are never touched.
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


def _inputs(n, L, nocc, nb, kernel, omega, seed):
    s = synth.System(n=n, L=L, n_occ=nocc, n_bands=nb, kernel=kernel, omega=omega)
    ecut = min(synth.ECUT_HA, 0.3 * (math.pi * n / L) ** 2)
    return s, synth.orbitals(s, seed, ecut=ecut), synth.targets(s, seed, ecut=ecut)


def _ulp_close(a, b):
    """Two FP32 roundings of FP64-accurate values: |a - b| <= 2^-23 |b| (one
    rounding each) + 2^-26 s_g, s_g the largest |b| at the element's grid
    point (the slice product is FP64-accurate relative to the size of the
    terms it sums, about the magnitude of Xi at that point)."""
    a64, b64 = a.to(torch.complex128), b.to(torch.complex128)
    d = torch.abs(a64 - b64)
    scale = torch.abs(b64).amax(dim=0, keepdim=True)
    bound = 2.0 ** -23 * torch.abs(b64) + 2.0 ** -26 * scale
    return bool(torch.all(d <= bound)), float((d / (torch.abs(b64) + 1e-30)).max())


@pytest.mark.parametrize("n,L,nocc,kernel,omega", [(24, 10.0, 13, "erfc", 0.3), (48, 20.5, 128, "erfc", 0.106),
                                                   (16, 8.0, 150, "bare", 0.0)])
def test_xi_fp64_modes(ace, n, L, nocc, kernel, omega):
    s, phi, psi = _inputs(n, L, nocc, 4, kernel, omega, seed=4100 + n)
    kern = oracle.coulomb_kernel((n,) * 3, (L,) * 3, kernel, omega)
    ref = oracle.ace_build(phi, kern, s.dv)
    phi_d = torch.from_numpy(phi).to(torch.complex64).cuda()
    out = {}
    plans = {}
    for prec in ("split_tf32", "default", "xi_fp64", "xi_fp64_simt"):
        plans[prec] = ace.Plan(n, L, nocc, dtype="c64", kernel=kernel, omega=omega, prec=prec)
        out[prec] = plans[prec].build(phi_d)
        assert plans[prec].status() == (0, 0), prec
    assert torch.equal(out["default"]["Xi"], out["xi_fp64"]["Xi"])      # the C64 default
    for prec in ("split_tf32", "xi_fp64", "xi_fp64_simt"):
        assert torch.equal(out[prec]["W"], out["default"]["W"])
        assert torch.equal(out[prec]["M"], out["default"]["M"])
        assert rel(_host(out[prec]["Xi"]), ref["Xi"]) < 1e-5
    ok, worst = _ulp_close(out["xi_fp64"]["Xi"], out["xi_fp64_simt"]["Xi"])
    print(f"{n}^3 N={nocc}: slice vs FP64 Xi, max elementwise rel diff {worst:.2e}")
    assert ok
    # FP64 output of the two products from the same W and L^{-*}
    p = plans["xi_fp64"]
    a = p.debug_xi_product(out["xi_fp64"]["W"], 1)
    b = p.debug_xi_product(out["xi_fp64"]["W"], 2)
    e = float(torch.linalg.vector_norm(a - b) / torch.linalg.vector_norm(b))
    print(f"{n}^3 N={nocc}: FP64-output slice product vs FP64 CUDA cores: {e:.2e}")
    assert e < 1e-10
    assert p.status() == (0, 0)
    # the apply of the FP64-accurate Xi
    psi_d = torch.from_numpy(psi).to(torch.complex64).cuda()
    y = plans["xi_fp64"].apply(out["xi_fp64"]["Xi"], psi_d)
    assert rel(_host(y), oracle.ace_apply(ref["Xi"], psi, s.dv)) < 1e-5


def test_xi_fp64_on_an_ill_conditioned_m(ace):
    """Orbitals scaled over three decades make -M ill-conditioned (its eigenvalues
    spread over about six decades),
    so the entries of L^{-*} are large: the FP64-accurate slice product stays
    within one FP32 rounding of the plain FP64 product, the TF32-split product
    does not."""
    n, L, nocc = 16, 8.0, 24
    s, phi, _ = _inputs(n, L, nocc, 1, "bare", 0.0, seed=77)
    phi = phi * np.logspace(0, -3, nocc)[:, None, None, None]
    phi_d = torch.from_numpy(phi).to(torch.complex64).cuda()
    res = {}
    for prec in ("split_tf32", "xi_fp64", "xi_fp64_simt"):
        plan = ace.Plan(n, L, nocc, dtype="c64", prec=prec)
        res[prec] = plan.build(phi_d)["Xi"]
        assert plan.status() == (0, 0), prec
    ok, worst = _ulp_close(res["xi_fp64"], res["xi_fp64_simt"])
    d_tf32 = float(torch.linalg.vector_norm(res["split_tf32"] - res["xi_fp64_simt"]) /
                   torch.linalg.vector_norm(res["xi_fp64_simt"]))
    d_oz = float(torch.linalg.vector_norm(res["xi_fp64"] - res["xi_fp64_simt"]) /
                 torch.linalg.vector_norm(res["xi_fp64_simt"]))
    print(f"ill-conditioned: TF32 split vs FP64 {d_tf32:.2e}, slices vs FP64 {d_oz:.2e} (max elementwise {worst:.2e})")
    assert ok and d_oz < 1e-7 and d_oz < d_tf32


@pytest.mark.parametrize("n,L,nocc,nb,kernel,omega", [(24, 10.0, 13, 5, "erfc", 0.3),
                                                      (48, 20.5, 128, 150, "erfc", 0.106),
                                                      (20, 8.0, 40, 128, "bare", 0.0)])
def test_split_bf16(ace, n, L, nocc, nb, kernel, omega):
    """ACE_PREC_SPLIT_BF16: M = dV Phi^* W and the apply on BF16 tensor cores
    with the hi/lo split (MMA widths 128, 192 and 256 by n_b and N). W is the
    default plan's (same pair path), E_x is within FP32 rounding (the diagonal
    of M is summed from FP32 products), and M, Xi and V_ACE psi stay within
    1e-4 of the FP64 oracle (measured errors printed: about 2^-16 per product,
    averaged over the N_g terms of each sum)."""
    s, phi, psi = _inputs(n, L, nocc, nb, kernel, omega, seed=5200 + n)
    kern = oracle.coulomb_kernel((n,) * 3, (L,) * 3, kernel, omega)
    ref = oracle.ace_build(phi, kern, s.dv)
    phi_d = torch.from_numpy(phi).to(torch.complex64).cuda()
    psi_d = torch.from_numpy(psi).to(torch.complex64).cuda()
    bf = ace.Plan(n, L, nocc, dtype="c64", kernel=kernel, omega=omega, prec="split_bf16")
    tf = ace.Plan(n, L, nocc, dtype="c64", kernel=kernel, omega=omega)
    ob, ot = bf.build(phi_d), tf.build(phi_d)
    assert bf.status() == (0, 0)
    assert torch.equal(ob["W"], ot["W"])
    assert abs(ob["Ex"].item() - ref["Ex"]) < 1e-6 * abs(ref["Ex"])
    e_m = rel(_host(ob["M"]), ref["M"])
    e_xi = rel(_host(ob["Xi"]), ref["Xi"])
    y = bf.apply(ob["Xi"], psi_d)
    e_y = rel(_host(y), oracle.ace_apply(ref["Xi"], psi, s.dv))
    e_m_tf = rel(_host(ot["M"]), ref["M"])
    print(f"{n}^3 N={nocc} n_b={nb}: split_bf16 M {e_m:.2e} (TF32 split {e_m_tf:.2e}), Xi {e_xi:.2e}, "
          f"apply {e_y:.2e}")
    assert e_m < 1e-4 and e_xi < 1e-4 and e_y < 1e-4
    assert e_m > e_m_tf                                  # BF16 really ran: coarser than TF32


def test_prec_fp32_is_the_cuda_core_path(ace):
    n, L, nocc = 20, 8.0, 9
    s, phi, psi = _inputs(n, L, nocc, 5, "bare", 0.0, seed=12)
    phi_d = torch.from_numpy(phi).to(torch.complex64).cuda()
    psi_d = torch.from_numpy(psi).to(torch.complex64).cuda()
    a = ace.Plan(n, L, nocc, prec="fp32")
    b = ace.Plan(n, L, nocc, tensor_cores=False)
    oa, ob = a.build(phi_d), b.build(phi_d)
    assert torch.equal(oa["Xi"], ob["Xi"]) and torch.equal(oa["M"], ob["M"])
    assert torch.equal(a.apply(oa["Xi"], psi_d), b.apply(ob["Xi"], psi_d))


@pytest.mark.parametrize("dtype", ["c64", "c128", "r64"])
def test_leading_dimension(ace, dtype):
    n, L, nocc, nb = 16, 8.0, 7, 5
    real = dtype == "r64"
    s = synth.System(n=n, L=L, n_occ=nocc, n_bands=nb, real=real, kernel="erfc", omega=0.3)
    ecut = 0.3 * (math.pi * n / L) ** 2
    phi = synth.orbitals(s, 31, ecut=ecut)
    psi = synth.targets(s, 31, ecut=ecut)
    td = ace.TORCH_DTYPES[dtype]
    packed = ace.Plan(n, L, nocc, dtype=dtype, kernel="erfc", omega=0.3)
    ld = n ** 3 + 96
    strided = ace.Plan(n, L, nocc, dtype=dtype, kernel="erfc", omega=0.3, ld=ld)
    sentinel = 12345.0

    def put(a):
        t = strided.empty(a.shape[0])
        t.as_strided((a.shape[0], ld), (ld, 1)).fill_(sentinel)
        t.copy_(torch.from_numpy(a).to(td))
        return t

    def gaps_intact(t):
        flat = t.as_strided((t.shape[0], ld), (ld, 1))
        return bool(torch.all(flat[:, n ** 3:] == sentinel))

    phi_p = torch.from_numpy(phi).to(td).cuda()
    psi_p = torch.from_numpy(psi).to(td).cuda()
    phi_s, psi_s = put(phi), put(psi)
    xi_s, w_s = put(np.zeros_like(phi)), put(np.zeros_like(phi))
    a = packed.build(phi_p)
    b = strided.build(phi_s, xi=xi_s, w=w_s)
    assert packed.status() == (0, 0) and strided.status() == (0, 0)
    assert torch.equal(a["W"], b["W"]) and torch.equal(a["Xi"], b["Xi"]) and torch.equal(a["M"], b["M"])
    y_s = put(np.zeros_like(psi))
    assert torch.equal(packed.apply(a["Xi"], psi_p), strided.apply(xi_s, psi_s, out=y_s))
    y2_s = put(np.zeros_like(psi))
    assert torch.equal(packed.exchange_apply(phi_p, psi_p), strided.exchange_apply(phi_s, psi_s, out=y2_s))
    g_s = put(np.zeros_like(phi))
    ea, ga = packed.energy_grad(phi_p, grad=True, grad_scale=0.5)
    eb, gb = strided.energy_grad(phi_s, grad=True, grad_scale=0.5, out=g_s)
    assert ea.item() == eb.item() and torch.equal(ga, gb)
    for t in (phi_s, psi_s, xi_s, w_s, y_s, y2_s, g_s):
        assert gaps_intact(t)
