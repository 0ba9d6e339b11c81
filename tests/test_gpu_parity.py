"""GPU parity: the CUDA path through the C ABI against the FP64 oracle.

Tolerances (Frobenius-relative, ||x - x_ref|| / ||x_ref||):
* FP64 storage (r64, c128): 1e-10 on every output;
* FP32 storage (c64): 1e-6 on W, V_X psi, E_x (FFT path in FP32 with FP64
  twiddles; the bound is the one the FP32 mode is specified to meet), 1e-5 on
  M, Xi and V_ACE psi (FP32 GEMMs over N_g ~ 1e5 terms; Xi also carries the
  conditioning of L), 1e-5 on the gradient.
"""
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


def _ecut(n, L):
    # sphere well inside the grid's Nyquist box: |G|^2/2 <= 0.3 (pi n / L)^2
    return min(synth.ECUT_HA, 0.3 * (math.pi * n / L) ** 2)


def _inputs(n, L, nocc, nb, dtype, kernel, omega, seed):
    s = synth.System(n=n, L=L, n_occ=nocc, n_bands=nb, real=(dtype == "r64"), kernel=kernel, omega=omega)
    phi = synth.orbitals(s, seed, ecut=_ecut(n, L))
    psi = synth.targets(s, seed, ecut=_ecut(n, L))
    kern = oracle.coulomb_kernel((n, n, n), (L, L, L), kernel, omega)
    return s, phi, psi, kern


def _dev(a, dtype, ace):
    return torch.from_numpy(np.ascontiguousarray(a)).to(ace.TORCH_DTYPES[dtype]).cuda()


def _host(t):
    return t.detach().cpu().numpy().astype(np.complex128 if t.is_complex() else np.float64)


CASES = [
    # n, L, N, nb, dtype, kernel, omega
    (8, 6.0, 5, 3, "c128", "erfc", 0.5),
    (12, 7.0, 11, 7, "c128", "bare", 0.0),       # N = 8 + 3: ragged tile
    (16, 8.0, 9, 4, "c64", "erfc", 0.3),
    (20, 8.0, 6, 5, "c64", "bare", 0.0),         # radix 5
    (24, 10.0, 8, 16, "r64", "bare", 0.0),       # the real Gamma-point 24^3 workload
    (32, 11.0, 13, 9, "c64", "erfc", 0.106),
    (36, 12.0, 10, 6, "c64", "erfc", 0.106),     # radix 3 x 3
    (40, 14.0, 7, 3, "c128", "bare", 0.0),
    (48, 20.5, 17, 5, "c64", "erfc", 0.106),     # the 48^3 edge, ragged N
    (64, 27.3, 12, 4, "c64", "bare", 0.0),
    (96, 41.0, 5, 3, "c64", "erfc", 0.106),      # the 96^3 edge (Si512-like cell, h = 0.427)
    (64, 27.3, 6, 3, "c128", "bare", 0.0),       # FP64 two-lane line transforms
    (64, 27.3, 5, 2, "r64", "bare", 0.0),
    (96, 41.0, 3, 2, "c128", "erfc", 0.106),
]


@pytest.mark.parametrize("n,L,nocc,nb,dtype,kernel,omega", CASES)
def test_build_apply_energy_parity(ace, n, L, nocc, nb, dtype, kernel, omega):
    s, phi, psi, kern = _inputs(n, L, nocc, nb, dtype, kernel, omega, seed=1000 + n)
    ref = oracle.ace_build(phi, kern, s.dv)
    tol = TOL[dtype]
    plan = ace.Plan(n, L, nocc, dtype=dtype, kernel=kernel, omega=omega)
    phi_d, psi_d = _dev(phi, dtype, ace), _dev(psi, dtype, ace)

    out = plan.build(phi_d)
    code, piv = plan.status()
    assert code == 0, (code, piv)
    assert rel(_host(out["W"]), ref["W"]) < tol["w"]
    m_ref = ref["M"].real if dtype == "r64" else ref["M"]
    assert rel(_host(out["M"]), m_ref) < tol["m"]
    assert rel(_host(out["Xi"]), ref["Xi"]) < tol["xi"]
    assert abs(out["Ex"].item() - ref["Ex"]) < tol["e"] * abs(ref["Ex"])

    y = plan.exchange_apply(phi_d, psi_d)
    assert rel(_host(y), oracle.exchange_apply(phi, psi, kern)) < tol["y"]

    ya = plan.apply(out["Xi"], psi_d)
    assert rel(_host(ya), oracle.ace_apply(ref["Xi"], psi, s.dv)) < tol["xi"]

    e_direct = oracle.energy_direct(phi, kern, s.volume)
    ex, g = plan.energy_grad(phi_d, grad=True, grad_scale=0.75)
    assert abs(ex.item() - e_direct) < tol["e"] * abs(e_direct)
    assert rel(_host(g), 0.75 * oracle.energy_grad(phi, kern, s.dv)) < tol["g"]
    ex_only, none = plan.energy_grad(phi_d, grad=False)
    assert none is None and abs(ex_only.item() - ex.item()) <= 1e-12 * abs(ex.item())


def test_bitwise_reproducible(ace):
    s, phi, psi, kern = _inputs(24, 10.0, 19, 5, "c64", "erfc", 0.3, seed=5)
    plan = ace.Plan(24, 10.0, 19, dtype="c64", kernel="erfc", omega=0.3, max_pairs=100, tile=4)
    phi_d = _dev(phi, "c64", ace)
    a = plan.build(phi_d)
    b = plan.build(phi_d)
    assert torch.equal(a["W"], b["W"]) and torch.equal(a["Xi"], b["Xi"])
    # a different tile / batch schedule gives the same W to rounding
    plan2 = ace.Plan(24, 10.0, 19, dtype="c64", kernel="erfc", omega=0.3, max_pairs=64, tile=8)
    c = plan2.build(phi_d)
    ref = oracle.exchange_W(phi, kern)
    assert rel(_host(c["W"]), ref) < 1e-6 and rel(_host(a["W"]), ref) < 1e-6


@pytest.mark.parametrize("engine,lanes,graphs,overlap", [(True, 1, True, False), (True, 1, False, False),
                                                        (False, 3, True, False), (False, 0, True, True)])
def test_schedules_match_bitwise(ace, engine, lanes, graphs, overlap):
    """Every way of running the four-kernel pair schedule gives the same bits
    as eager launches: replayed from a graph with a round's batches spread
    over lanes, and the two-stream schedule in which pass A of a batch
    overlaps pass D of the previous one. Each output element is written by one
    tile per round and rounds run in order; new pointers capture a new graph.
    The persistent engine accumulates a full off-diagonal tile with one thread
    per point (the four-kernel pass D splits it over two), so it agrees to
    rounding, and is bitwise stable from call to call."""
    s, phi, psi, kern = _inputs(24, 10.0, 21, 10, "c64", "erfc", 0.3, seed=8)
    eager = ace.Plan(24, 10.0, 21, dtype="c64", kernel="erfc", omega=0.3, tile=4, max_pairs=16,
                     graphs=False)
    graph = ace.Plan(24, 10.0, 21, dtype="c64", kernel="erfc", omega=0.3, tile=4, max_pairs=16,
                     lanes=lanes, graphs=graphs, engine=engine, overlap=overlap)
    phi_d = _dev(phi, "c64", ace)
    psi_d = _dev(psi, "c64", ace)

    def same(x, y, tol):
        if engine:
            return float(torch.linalg.vector_norm(x - y) / torch.linalg.vector_norm(x)) < tol
        return torch.equal(x, y)

    a = eager.build(phi_d)
    first = None
    for _ in range(2):                       # capture, then replay
        b = graph.build(phi_d)
        assert same(a["W"], b["W"], 1e-6) and same(a["Xi"], b["Xi"], 1e-5)
        if first is None:
            first = b["W"].clone()
        assert torch.equal(first, b["W"])
    phi2 = phi_d.clone()
    c = graph.build(phi2)                    # new pointer -> new graph
    assert torch.equal(first, c["W"])
    # one-sided tiles: the runtime-length loop may contract multiply-adds
    # differently in the two kernels, so modes agree to rounding, and each
    # mode is bitwise stable from call to call
    ya = eager.exchange_apply(phi_d, psi_d)
    yb1 = graph.exchange_apply(phi_d, psi_d).clone()
    yb2 = graph.exchange_apply(phi_d, psi_d)
    assert torch.equal(yb1, yb2)
    d = float(torch.linalg.vector_norm(ya - yb2) / torch.linalg.vector_norm(ya))
    print(f"exchange apply, engine={engine} lanes={lanes} graphs={graphs} overlap={overlap}: "
          f"rel diff to eager {d:.3e}")
    assert d < 1e-6
    ea, ga = eager.energy_grad(phi_d, grad=True, grad_scale=-1.5)
    eb, gb = graph.energy_grad(phi_d, grad=True, grad_scale=-1.5)
    assert same(ga, gb, 1e-6) and abs(ea.item() - eb.item()) <= 1e-13 * abs(ea.item())
    assert graph.status() == (0, 0)
    assert rel(_host(gb), -1.5 * oracle.energy_grad(phi, kern, s.dv)) < 1e-5


@pytest.mark.parametrize("n,L,nocc,nb", [(20, 8.0, 13, 70), (24, 10.0, 130, 9)])
def test_tensor_core_gemms_match_cuda_cores(ace, n, L, nocc, nb):
    """tcgen05 TF32 3-term-split GEMMs (M, Xi, apply) against the FP32 CUDA-core
    ones and the FP64 oracle, on shapes with partial row (N not a multiple of
    128), column (n_b not a multiple of 64) and grid-point (8000 points) tiles."""
    s, phi, psi, kern = _inputs(n, L, nocc, nb, "c64", "erfc", 0.3, seed=31)
    ref = oracle.ace_build(phi, kern, s.dv)
    phi_d, psi_d = _dev(phi, "c64", ace), _dev(psi, "c64", ace)
    tc = ace.Plan(n, L, nocc, dtype="c64", kernel="erfc", omega=0.3)
    simt = ace.Plan(n, L, nocc, dtype="c64", kernel="erfc", omega=0.3, tensor_cores=False)
    a, b = tc.build(phi_d), simt.build(phi_d)
    assert tc.status() == (0, 0) and simt.status() == (0, 0)
    assert torch.equal(a["W"], b["W"])
    m_ref = ref["M"]
    assert rel(_host(a["M"]), m_ref) < 1e-5 and rel(_host(b["M"]), m_ref) < 1e-5
    assert rel(_host(a["Xi"]), ref["Xi"]) < 1e-5
    ya = tc.apply(a["Xi"], psi_d)
    yb = simt.apply(b["Xi"], psi_d)
    y_ref = oracle.ace_apply(ref["Xi"], psi, s.dv)
    assert rel(_host(ya), y_ref) < 1e-5 and rel(_host(yb), y_ref) < 1e-5
    assert tc.status() == (0, 0)


@pytest.mark.parametrize("nocc,nb", [(100, 64), (20, 96), (20, 128), (150, 150), (20, 200), (20, 257)])
def test_tensor_core_tile_widths(ace, nocc, nb):
    """The tensor-core GEMMs pick an MMA width of 128, 192 or 256 columns per
    call (tiles of 64, 96 or 128 complex columns): n_b = 64 -> 128, 96 and 150
    and 257 -> 192, 128 and 200 -> 256, N = 100 -> 256 and N = 150 -> 192 for
    M and Xi, full and partial last tiles. M, Xi and the apply against the FP64
    oracle and the CUDA-core GEMMs."""
    n, L = 16, 8.0
    s, phi, psi, kern = _inputs(n, L, nocc, nb, "c64", "bare", 0.0, seed=57)
    ref = oracle.ace_build(phi, kern, s.dv)
    phi_d, psi_d = _dev(phi, "c64", ace), _dev(psi, "c64", ace)
    tc = ace.Plan(n, L, nocc, dtype="c64", kernel="bare")
    simt = ace.Plan(n, L, nocc, dtype="c64", kernel="bare", tensor_cores=False)
    a, b = tc.build(phi_d), simt.build(phi_d)
    assert tc.status() == (0, 0) and simt.status() == (0, 0)
    assert rel(_host(a["M"]), ref["M"]) < 1e-5
    assert rel(_host(a["Xi"]), ref["Xi"]) < 1e-5
    assert rel(_host(a["Xi"]), _host(b["Xi"])) < 1e-5
    xi_ref = _dev(ref["Xi"], "c64", ace)
    y = tc.apply(xi_ref, psi_d)
    y_simt = simt.apply(xi_ref, psi_d)
    y_ref = oracle.ace_apply(ref["Xi"], psi, s.dv)
    assert rel(_host(y), y_ref) < 1e-5
    assert rel(_host(y), _host(y_simt)) < 1e-5
    assert tc.status() == (0, 0)


def test_single_orbital_and_empty(ace):
    s, phi, psi, kern = _inputs(16, 8.0, 1, 2, "c128", "erfc", 0.4, seed=9)
    plan = ace.Plan(16, 8.0, 1, dtype="c128", kernel="erfc", omega=0.4)
    phi_d = _dev(phi, "c128", ace)
    out = plan.build(phi_d)
    assert rel(_host(out["W"]), oracle.exchange_W(phi, kern)) < 1e-10
    empty = torch.empty((0, 16, 16, 16), dtype=torch.complex128, device="cuda")
    y = plan.exchange_apply(phi_d, empty)
    assert y.shape[0] == 0
    assert plan.apply(out["Xi"], empty).shape[0] == 0


def test_errors_reported(ace):
    n, L = 16, 8.0
    s, phi, psi, kern = _inputs(n, L, 4, 2, "c128", "bare", 0.0, seed=3)
    plan = ace.Plan(n, L, 4, dtype="c128")
    phi_d = _dev(phi, "c128", ace)
    # workspace too small
    lib = ace.lib()
    import ctypes
    y = plan.empty(2)
    tiny = torch.empty(256, dtype=torch.uint8, device="cuda")
    code = lib.ace_exchange_apply(plan._h, ctypes.c_void_p(phi_d.data_ptr()), ctypes.c_void_p(phi_d.data_ptr()),
                                  2, ctypes.c_void_p(y.data_ptr()), ctypes.c_void_p(tiny.data_ptr()), 256, None)
    assert code == ace.ACE_ERR_WORKSPACE
    # aliasing output
    with pytest.raises(ace.AceError) as ei:
        plan.exchange_apply(phi_d, phi_d[:2].contiguous(), out=phi_d[:2])
    assert ei.value.code in (ace.ACE_ERR_ARG,)
    # -M singular: a zero orbital makes row/column 4 of M exactly zero, so the
    # 4th pivot is exactly 0 -> reported on the status word (two equal orbitals
    # would only give a rounding-level pivot of either sign)
    dup = phi.copy()
    dup[3] = 0.0
    plan.build(_dev(dup, "c128", ace))
    code, piv = plan.status()
    assert code == ace.ACE_ERR_NOT_POSDEF and piv == 4
    # non-finite input -> non-finite pivot
    bad = phi.copy()
    bad[0, 0, 0, 0] = np.nan
    plan.build(_dev(bad, "c128", ace))
    code, piv = plan.status()
    assert code == ace.ACE_ERR_NONFINITE and piv == 1
    # status clears after a good build
    plan.build(phi_d)
    assert plan.status() == (0, 0)


def test_autograd_gradient_fd(ace):
    """Gradient of E_x through the autograd Function: against the oracle and
    against central differences of FP64 GPU energies (h = 1e-4)."""
    n, L = 16, 8.0
    s, phi, psi, kern = _inputs(n, L, 3, 1, "c128", "bare", 0.0, seed=21)
    plan = ace.Plan(n, L, 3, dtype="c128")
    phi_d = _dev(phi, "c128", ace).requires_grad_(True)
    e = ace.exchange_energy(phi_d, plan)
    (2.5 * e).backward()
    g = _host(phi_d.grad)
    assert rel(g, 2.5 * oracle.energy_grad(phi, kern, s.dv)) < 1e-10
    h = 1e-4
    errs = []
    for d in synth.directions(phi.shape, 8, 77, s.dv):
        dd = _dev(d, "c128", ace)
        ep = plan.energy_grad(phi_d.detach() + h * dd)[0].item()
        em = plan.energy_grad(phi_d.detach() - h * dd)[0].item()
        fd = 2.5 * (ep - em) / (2 * h)
        an = float(np.real(np.vdot(g, d)))
        errs.append(abs(fd - an) / max(abs(an), 1e-12))
    assert max(errs) < 1e-5


def test_si64_full_size_sampled(ace):
    """The 48^3, N = 128, 192-band screened workload in the launch
    configuration the bench times (default plan): W, M on sampled orbitals
    against the oracle; V_ACE Phi = W, E_x(1/2 tr M) = E_x(Parseval), and the
    exchange apply on sampled bands."""
    s = synth.SI64_48
    seed = synth.seed_for(2)
    phi = synth.orbitals(s, seed)
    kern = oracle.coulomb_kernel((s.n,) * 3, (s.L,) * 3, s.kernel, s.omega)
    plan = ace.Plan(s.n, s.L, s.n_occ, dtype="c64", kernel=s.kernel, omega=s.omega)
    phi_d = _dev(phi, "c64", ace)
    out = plan.build(phi_d)
    assert plan.status() == (0, 0)
    W = _host(out["W"])
    M = _host(out["M"])
    for i in (0, 37, 127):
        w_ref = -np.sum(phi * oracle.poisson(np.conj(phi) * phi[i][None], kern), axis=0)
        assert rel(W[i], w_ref) < 1e-6
        m_col = s.dv * (np.conj(phi.reshape(s.n_occ, -1)) @ w_ref.ravel())
        assert rel(M[:, i], m_col) < 1e-5
    # Eq. ACEcond on the GPU's own outputs
    vphi = plan.apply(out["Xi"], phi_d)
    assert rel(_host(vphi), W) < 1e-5
    ex, _ = plan.energy_grad(phi_d)
    assert abs(ex.item() - out["Ex"].item()) < 2e-6 * abs(ex.item())
    psi = synth.targets(s, seed, count=4)
    y = plan.exchange_apply(phi_d, _dev(psi, "c64", ace))
    assert rel(_host(y), oracle.exchange_apply(phi, psi, kern)) < 1e-6


def test_diff64_full_size_sampled(ace):
    """The differentiation workload at full size (64^3, L = 27.33, N = 256,
    bare kernel, FP32): the hand-written adjoint gives grad = 2 dV W (Eq. EX,
    Wirtinger derivative in the torch convention) on sampled orbitals against
    the oracle's W columns; E_x from the Parseval sum equals 1/2 tr M of the
    build; the autograd Function returns the same gradient."""
    s = synth.DIFF_64
    seed = synth.seed_for(4)
    phi = synth.orbitals(s, seed)
    kern = oracle.coulomb_kernel((s.n,) * 3, (s.L,) * 3, s.kernel, s.omega)
    plan = ace.Plan(s.n, s.L, s.n_occ, dtype="c64", kernel=s.kernel)
    phi_d = _dev(phi, "c64", ace)
    ex, g = plan.energy_grad(phi_d, grad=True)
    assert plan.status() == (0, 0)
    G = _host(g)
    for i in (0, 131, 255):
        w_ref = -np.sum(phi * oracle.poisson(np.conj(phi) * phi[i][None], kern), axis=0)
        assert rel(G[i], 2.0 * s.dv * w_ref) < 1e-5, i
    out = plan.build(phi_d, want_w=False, want_m=False)
    assert abs(ex.item() - out["Ex"].item()) < 2e-6 * abs(ex.item())
    p = phi_d.clone().requires_grad_(True)
    e = ace.exchange_energy(p, plan)
    e.backward()
    assert torch.equal(p.grad, g)


@pytest.mark.parametrize("n,L,ne,nphi,dtype,kernel,omega", [
    (16, 8.0, 5, 9, "c64", "erfc", 0.3),
    (20, 8.0, 8, 21, "c128", "bare", 0.0),       # N_phi - N_e = 13: two one-sided blocks, ragged
    (12, 6.0, 3, 6, "r64", "bare", 0.0),
    (48, 20.5, 16, 24, "c64", "erfc", 0.106),    # the 48^3 cell, r = 1.5
])
def test_oversampled_build_parity(ace, n, L, ne, nphi, dtype, kernel, omega):
    """ACE with oversampling (Sec. 3): W_i = V_X[Phi_occ] Phi_i for all N_phi
    orbitals, M, Xi over N_phi, E_x of the occupied block, against the oracle;
    the oversampled V_ACE reproduces W on all N_phi orbitals (Eq. ACEcond on
    the larger subspace)."""
    s = synth.System(n=n, L=L, n_occ=nphi, n_bands=1, real=(dtype == "r64"), kernel=kernel, omega=omega)
    phi = synth.orbitals(s, 3300 + n, ecut=_ecut(n, L))
    kern = oracle.coulomb_kernel((n, n, n), (L, L, L), kernel, omega)
    ref = oracle.ace_build_oversampled(phi, ne, kern, s.dv)
    tol = TOL[dtype]
    plan = ace.Plan(n, L, ne, dtype=dtype, kernel=kernel, omega=omega)
    phi_d = _dev(phi, dtype, ace)
    out = plan.build_oversampled(phi_d)
    assert plan.status() == (0, 0)
    assert rel(_host(out["W"]), ref["W"]) < tol["w"]
    m_ref = ref["M"].real if dtype == "r64" else ref["M"]
    assert rel(_host(out["M"]), m_ref) < tol["m"]
    assert rel(_host(out["Xi"]), ref["Xi"]) < tol["xi"]
    assert abs(out["Ex"].item() - ref["Ex"]) < tol["e"] * abs(ref["Ex"])
    full = ace.Plan(n, L, nphi, dtype=dtype, kernel=kernel, omega=omega)   # applies N_phi vectors of Xi
    vphi = full.apply(out["Xi"], phi_d)
    assert rel(_host(vphi), _host(out["W"])) < tol["xi"]
    second = plan.build_oversampled(phi_d)                                # graph replay
    assert torch.equal(second["W"], out["W"]) and torch.equal(second["Xi"], out["Xi"])


def test_oversampled_without_extra_orbitals_is_the_build(ace):
    s, phi, psi, kern = _inputs(24, 10.0, 11, 4, "c64", "erfc", 0.3, seed=9)
    plan = ace.Plan(24, 10.0, 11, dtype="c64", kernel="erfc", omega=0.3)
    phi_d = _dev(phi, "c64", ace)
    a = plan.build(phi_d)
    b = plan.build_oversampled(phi_d)
    for k in ("W", "Xi", "M"):
        assert torch.equal(a[k], b[k]), k
    assert a["Ex"].item() == b["Ex"].item()
    with pytest.raises(ValueError):
        plan.build_oversampled(phi_d[:10])
    ws = plan.workspace(ace.OP_BUILD_OVERSAMPLED, 11)
    xi = plan.empty(11)
    code = ace.lib().ace_build_oversampled(plan._h, ace._ptr(phi_d), 10, None, ace._ptr(xi), None, None,
                                           ace._ptr(ws), ws.numel(), ace._stream())
    assert code == ace.ACE_ERR_ARG


@pytest.mark.parametrize("n,L,dtype,kernel,omega", [(16, 8.0, "c64", "bare", 0.0), (20, 9.0, "r64", "bare", 0.0),
                                                    (24, 10.0, "c128", "erfc", 0.3), (48, 20.5, "c64", "bare", 0.0)])
def test_poisson_hartree_parity(ace, n, L, dtype, kernel, omega):
    """Periodic Poisson solves through the pair passes against the oracle's
    FFT Poisson (pinned to the dense DFT): the Hartree potential V_H[rho] of
    Eq. HF for the electron density rho = sum_i |phi_i|^2 (bare kernel), plus
    more densities than one batch holds."""
    s = synth.System(n=n, L=L, n_occ=6, n_bands=1, real=(dtype == "r64"), kernel=kernel, omega=omega)
    phi = synth.orbitals(s, 4400 + n, ecut=_ecut(n, L))
    rho = np.sum(np.abs(phi) ** 2, axis=0)[None]
    extra = synth.targets(s, 4400 + n, count=11, ecut=_ecut(n, L))
    if dtype == "r64":
        extra = extra.real
    dens = np.concatenate([rho, extra], axis=0)
    kern = oracle.coulomb_kernel((n, n, n), (L, L, L), kernel, omega)
    plan = ace.Plan(n, L, 6, dtype=dtype, kernel=kernel, omega=omega, max_pairs=0)
    v = plan.poisson(_dev(dens, dtype, ace))
    ref = oracle.poisson(dens, kern)
    if dtype == "r64":
        ref = ref.real
    assert rel(_host(v), ref) < TOL[dtype]["w"]
    # Hartree energy 1/2 dV sum rho V_H > 0 for the density (bare kernel)
    if kernel == "bare":
        eh = 0.5 * s.dv * float(np.real(np.sum(np.conj(rho[0]) * _host(v)[0])))
        assert eh > 0


def test_si512_full_size(ace):
    """The large workload at full size (96^3, L = 41, N = 1024, screened
    kernel, FP32 pairs, TF32 3-term GEMMs, FP64 Cholesky), default plan:
    properties that hold at any size -- V_ACE Phi = W (Eq. ACEcond),
    dV Xi^* Phi = -L^* (upper triangular), 1/2 tr M = -1/2 ||dV Xi^* Phi||^2
    (Eq. EX_ACE) -- sampled W and M columns, and sampled single pair solves on
    the full grid, against the FP64 oracle."""
    s = synth.SI512_96
    phi = synth.orbitals_device(s, synth.seed_for(5))
    plan = ace.Plan(s.n, s.L, s.n_occ, dtype="c64", kernel=s.kernel, omega=s.omega)
    out = plan.build(phi)
    assert plan.status() == (0, 0)
    cols = (0, 1023)
    w_gpu = {i: _host(out["W"][i]) for i in cols}
    m_gpu = {i: _host(out["M"][:, i]) for i in cols}
    vphi = plan.apply(out["Xi"], phi)
    assert float(torch.linalg.vector_norm(vphi - out["W"]) / torch.linalg.vector_norm(out["W"])) < 1e-5
    del vphi
    a = s.dv * (out["Xi"].reshape(s.n_occ, -1).conj() @ phi.reshape(s.n_occ, -1).T).to(torch.complex128)
    assert float(torch.linalg.norm(torch.tril(a, -1)) / torch.linalg.norm(a)) < 1e-5
    ex = out["Ex"].item()
    assert abs(-0.5 * float(torch.linalg.norm(a) ** 2) - ex) < 1e-5 * abs(ex)
    assert ex < 0
    del out, a
    torch.cuda.empty_cache()
    kern = oracle.coulomb_kernel((s.n,) * 3, (s.L,) * 3, s.kernel, s.omega)
    # sampled W columns (Eq. W), all 1024 pair solves each, and the matching M
    # columns; V_X[Phi] is a sum over orbitals, so the oracle runs on chunks of Phi
    w_ref = {i: np.zeros((s.n,) * 3, dtype=np.complex128) for i in cols}
    m_ref = {i: np.zeros(s.n_occ, dtype=np.complex128) for i in cols}
    targets = {i: phi[i].cpu().numpy().astype(np.complex128)[None] for i in cols}
    for c in range(0, s.n_occ, 128):
        chunk = phi[c:c + 128].cpu().numpy().astype(np.complex128)
        for i in cols:
            w_ref[i] += oracle.exchange_apply(chunk, targets[i], kern)[0]
    for c in range(0, s.n_occ, 128):
        chunk = phi[c:c + 128].cpu().numpy().astype(np.complex128).reshape(-1, s.n ** 3)
        for i in cols:
            m_ref[i][c:c + 128] = s.dv * (np.conj(chunk) @ w_ref[i].ravel())
    for i in cols:
        assert rel(w_gpu[i], w_ref[i]) < 1e-6, i            # measured 1.9e-7
        assert rel(m_gpu[i], m_ref[i]) < 1e-6, i            # measured 1.9e-7
    one = ace.Plan(s.n, s.L, 1, dtype="c64", kernel=s.kernel, omega=s.omega)
    for i, j in ((0, 1), (517, 1023), (900, 900)):
        y = one.exchange_apply(phi[i:i + 1].contiguous(), phi[j:j + 1].contiguous())
        pi = phi[i].cpu().numpy().astype(np.complex128)
        pj = phi[j].cpu().numpy().astype(np.complex128)
        ref = -pi * oracle.poisson((np.conj(pi) * pj)[None], kern)[0]
        assert rel(_host(y)[0], ref) < 1e-6, (i, j)


@pytest.mark.parametrize("dtype,graphs,overlap", [("c64", True, True), ("c64", True, False), ("c64", False, True),
                                                  ("c128", True, True), ("r64", True, True)])
def test_stored_pair_potentials(ace, dtype, graphs, overlap):
    """ace_exchange_energy_grad with recompute = 0: the energy call keeps every
    unique pair potential in the workspace, the gradient call only accumulates
    (Eq. EX and its gradient 2 dV W); energies and gradients are bitwise those
    of the recomputing sweep, on every schedule, and through the autograd
    Function with and without the store."""
    s, phi, psi, kern = _inputs(24, 10.0, 21, 1, dtype, "erfc", 0.3, seed=61)
    plan = ace.Plan(24, 10.0, 21, dtype=dtype, kernel="erfc", omega=0.3, tile=4, max_pairs=16,
                    graphs=graphs, overlap=overlap)
    phi_d = _dev(phi, dtype, ace)
    e1, g1 = plan.energy_grad(phi_d, grad=True, grad_scale=0.5)
    e0, _ = plan.energy_grad(phi_d)
    for _ in range(2):                                   # capture, then replay
        e2, none = plan.energy_grad(phi_d, recompute=False)
        e3, g3 = plan.energy_grad(phi_d, grad=True, grad_scale=0.5, recompute=False)
        assert none is None and plan.status() == (0, 0)
        assert e3.item() == e2.item()                    # the stored energy sums, reduced again
        assert abs(e2.item() - e0.item()) <= 1e-13 * abs(e0.item())
        assert abs(e1.item() - e0.item()) <= 1e-13 * abs(e0.item())
        assert torch.equal(g3, g1)
    assert rel(_host(g3), 0.5 * oracle.energy_grad(phi, kern, s.dv)) < TOL[dtype]["g"]
    need = plan.workspace_size(ace.OP_ENERGY_GRAD_STORE)
    pairs, slot = 21 * 22 // 2, 24 ** 3 * (8 if dtype == "c64" else 16)
    if dtype == "r64":      # two real pair potentials per complex slot
        assert (pairs + 1) // 2 * slot <= need < pairs * slot
    else:
        assert need >= pairs * slot
    grads = []
    for store in (True, False):
        p = phi_d.clone().requires_grad_(True)
        e = ace.exchange_energy(p, plan, store=store)
        (3.0 * e).backward()
        grads.append(p.grad)
    assert torch.equal(grads[0], grads[1]) and torch.equal(grads[0], 6.0 * g1)
