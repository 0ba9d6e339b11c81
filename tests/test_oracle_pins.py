"""Pins of the FP64 oracle to facts other than itself.

Each test fixes one part of the oracle against a closed form, a brute-force
sum, an invariant stated in the paper, or a textbook identity, so that a
dropped term, a wrong sign or conjugate, a transposed operand or a wrong
normalisation fails at least one of them:

* plane-wave orbitals: V_X e^{ik.r} = -sum_i K(k - k_i)/Omega e^{ik.r} and
  E_x = -1/2 sum_ij K(k_i - k_j)/Omega, with K evaluated here from the
  formula (bare 4 pi/q^2, screened (4 pi/q^2)(1 - e^{-q^2/4w^2}));
* the screened kernel against a radial quadrature of erfc(w r)/r;
* FFT Poisson vs. an explicit O(N_g^2) DFT sum on 8^3 grids;
* V_X vs. the dense Hadamard-product matrix of Eq. VXkernel, Hermitian and
  negative semidefinite;
* V_ACE phi_i = W_i and symmetry (Eq. ACEcond), rank N (Eq. ACE),
  Xi* Phi = -L*, agreement on span(Phi);
* E_x from Eq. EX, from 1/2 tr M and from Eq. EX_ACE agree;
* gradient: Euler identity of the quartic energy and central differences.
"""
import math

import numpy as np
import pytest
import scipy.integrate
import scipy.special

import oracle
from paper_1601_07159_gb300 import synth
from tests.conftest import rel


def _fftfreq_index(q, n):
    """Wrap an integer wavevector index onto the FFT grid (|q| <= n/2)."""
    q = q % n
    return q - n if q > n // 2 else q


def _k_formula(q2, kind, omega, g0):
    if q2 == 0.0:
        return g0
    if kind == "bare":
        return 4.0 * math.pi / q2
    return 4.0 * math.pi / q2 * (1.0 - math.exp(-q2 / (4.0 * omega * omega)))


def _small_system(n=8, L=6.0, nocc=4, real=False, kernel="bare", omega=0.0, seed=7):
    s = synth.System(n=n, L=L, n_occ=nocc, n_bands=3, real=real, kernel=kernel, omega=omega)
    phi = synth.orbitals(s, seed, ecut=6.0)
    psi = synth.targets(s, seed, ecut=6.0)
    kern = oracle.coulomb_kernel((n, n, n), (L, L, L), kernel, omega)
    return s, phi, psi, kern


# --------------------------------------------------------------------------- (a)
@pytest.mark.parametrize("kind,omega", [("bare", 0.0), ("erfc", 0.3), ("erfc", 0.106)])
def test_plane_wave_closed_form(kind, omega):
    n, L = 8, 7.0
    vol = L ** 3
    m_occ = [(0, 0, 0), (1, 0, 0), (0, -1, 2), (3, 1, -1), (-2, 2, 1)]
    m_tgt = (1, 2, -3)
    g0 = 0.0 if kind == "bare" else math.pi / omega ** 2
    phi = synth.plane_wave_orbitals(n, L, m_occ)
    psi = synth.plane_wave_orbitals(n, L, [m_tgt]) * math.sqrt(vol)   # e^{ik.r}
    kern = oracle.coulomb_kernel((n, n, n), (L, L, L), kind, omega)

    def kq(ma, mb):
        q = [_fftfreq_index(ma[d] - mb[d], n) for d in range(3)]
        q2 = sum((2 * math.pi * qd / L) ** 2 for qd in q)
        return _k_formula(q2, kind, omega, g0)

    lam = -sum(kq(m_tgt, mi) for mi in m_occ) / vol
    y = oracle.exchange_apply(phi, psi, kern)
    assert rel(y, lam * psi) < 1e-12

    e_closed = -0.5 * sum(kq(mi, mj) for mi in m_occ for mj in m_occ) / vol
    assert abs(oracle.energy_direct(phi, kern, vol) - e_closed) < 1e-12 * abs(e_closed)
    out = oracle.ace_build(phi, kern, vol / n ** 3) if kind != "bare" else None
    if out is not None:   # bare K(0)=0 makes -M singular only if a K vanishes; erfc is SPD
        assert abs(out["Ex"] - e_closed) < 1e-12 * abs(e_closed)


def test_screened_kernel_radial_quadrature():
    """(4 pi/G^2)(1 - e^{-G^2/4w^2}) is the 3-D transform of erfc(w r)/r:
    (4 pi/G) int_0^inf erfc(w r) sin(G r) dr."""
    omega = 0.106
    for g in (0.3, 0.9, 2.5):
        val, _ = scipy.integrate.quad(lambda r: scipy.special.erfc(omega * r),
                                      0, 60.0 / omega, weight="sin", wvar=g, limit=400)
        ft = 4.0 * math.pi / g * val
        kern = oracle.coulomb_kernel((4, 4, 4), (2 * math.pi / g * 1.0,) * 3, "erfc", omega)
        # index (1,0,0) of a cell with Lx = 2 pi/g has |G| = g
        assert abs(kern[0, 0, 1] - ft) < 1e-8 * ft


def test_screened_kernel_limits():
    shape, lengths = (6, 6, 6), (5.0, 5.0, 5.0)
    bare = oracle.coulomb_kernel(shape, lengths, "bare")
    wide = oracle.coulomb_kernel(shape, lengths, "erfc", 1e-4)
    sharp = oracle.coulomb_kernel(shape, lengths, "erfc", 1e4)
    nz = bare > 0
    assert np.allclose(wide[nz], bare[nz], rtol=1e-12)
    assert np.max(np.abs(sharp[nz])) < 1e-6
    assert wide[0, 0, 0] == pytest.approx(math.pi / 1e-8)


# --------------------------------------------------------------------------- (b)
@pytest.mark.parametrize("kind,omega", [("bare", 0.0), ("erfc", 0.4)])
def test_poisson_vs_dense_dft(kind, omega):
    rng = np.random.default_rng(3)
    shape = (8, 6, 5)          # non-cubic, mixed radix, odd edge
    lengths = (4.0, 5.0, 6.5)
    rho = rng.standard_normal(shape) + 1j * rng.standard_normal(shape)
    kern = oracle.coulomb_kernel(shape, lengths, kind, omega)
    assert rel(oracle.poisson(rho, kern), oracle.poisson_bruteforce(rho, kern)) < 1e-12


@pytest.mark.parametrize("real", [False, True])
def test_exchange_vs_dense_matrix(real):
    s, phi, psi, kern = _small_system(real=real, kernel="erfc", omega=0.5)
    vx = oracle.vx_matrix(phi, kern)
    y_dense = (vx @ psi.reshape(psi.shape[0], -1).T).T.reshape(psi.shape)
    assert rel(oracle.exchange_apply(phi, psi, kern), y_dense) < 1e-12


# --------------------------------------------------------------------------- (c)
@pytest.mark.parametrize("kind", ["bare", "erfc"])
def test_vx_hermitian_nsd(kind):
    s, phi, psi, kern = _small_system(kernel=kind, omega=0.5)
    vx = oracle.vx_matrix(phi, kern)
    scale = np.linalg.norm(vx, 2)
    assert np.linalg.norm(vx - vx.conj().T) < 1e-13 * scale * vx.shape[0]
    ev = np.linalg.eigvalsh(0.5 * (vx + vx.conj().T))
    assert ev.max() <= 1e-13 * scale
    assert ev.min() < -1e-3 * scale      # nontrivial


@pytest.mark.parametrize("real", [False, True])
def test_ace_conditions(real):
    s, phi, psi, kern = _small_system(nocc=5, real=real, kernel="erfc", omega=0.5)
    out = oracle.ace_build(phi, kern, s.dv)
    W, M, L, Xi = out["W"], out["M"], out["L"], out["Xi"]
    # Eq. ACEcond: V_ACE phi_i = W_i
    assert rel(oracle.ace_apply(Xi, phi, s.dv), W) < 1e-12
    # M Hermitian negative definite, L its Cholesky factor (lower, positive diagonal)
    assert np.linalg.eigvalsh(M).max() < 0
    assert np.allclose(np.triu(L, 1), 0) and np.all(np.real(np.diag(L)) > 0)
    assert rel(L @ L.conj().T, -M) < 1e-13
    # Xi* Phi dV = -L*
    c = s.dv * (Xi.reshape(s.n_occ, -1).conj() @ phi.reshape(s.n_occ, -1).T)
    assert rel(c, -L.conj().T) < 1e-12
    # agreement on span(Phi), not outside it
    coef = np.random.default_rng(1).standard_normal((s.n_occ, 2)) + 1j
    inspan = np.tensordot(coef.T, phi, axes=1)
    assert rel(oracle.ace_apply(Xi, inspan, s.dv), oracle.exchange_apply(phi, inspan, kern)) < 1e-12
    assert rel(oracle.ace_apply(Xi, psi, s.dv), oracle.exchange_apply(phi, psi, kern)) > 1e-3
    # Eq. ACE: V_ACE Hermitian, negative semidefinite, strict rank N
    dense = np.stack([oracle.ace_apply(Xi, e.reshape(1, *phi.shape[1:]), s.dv).ravel()
                      for e in np.eye(phi[0].size)], axis=1)
    assert np.linalg.norm(dense - dense.conj().T) < 1e-12 * np.linalg.norm(dense)
    ev = np.linalg.eigvalsh(0.5 * (dense + dense.conj().T))
    assert ev.max() < 1e-12 * abs(ev.min())
    assert np.linalg.matrix_rank(dense, tol=1e-10 * abs(ev.min())) == s.n_occ
    if real:
        assert np.max(np.abs(W.imag)) < 1e-13 * np.max(np.abs(W))


# --------------------------------------------------------------------------- (d)
@pytest.mark.parametrize("kind", ["bare", "erfc"])
def test_energies_agree(kind):
    s, phi, psi, kern = _small_system(n=10, L=7.0, nocc=6, kernel=kind, omega=0.3)
    out = oracle.ace_build(phi, kern, s.dv)
    e_direct = oracle.energy_direct(phi, kern, s.volume)
    e_ace = oracle.energy_ace(out["Xi"], phi, s.dv)
    assert e_direct < 0
    assert abs(out["Ex"] - e_direct) < 1e-12 * abs(e_direct)
    assert abs(e_ace - e_direct) < 1e-12 * abs(e_direct)


def test_unitary_invariance():
    s, phi, psi, kern = _small_system(nocc=4, kernel="erfc", omega=0.5)
    u = synth.random_unitary(s.n_occ, 11)
    phiu = np.tensordot(u.T, phi, axes=1)        # (Phi U)_k = sum_i phi_i U_ik
    W = oracle.exchange_W(phi, kern)
    Wu = oracle.exchange_W(phiu, kern)
    assert rel(Wu, np.tensordot(u.T, W, axes=1)) < 1e-12
    assert rel(oracle.exchange_apply(phiu, psi, kern), oracle.exchange_apply(phi, psi, kern)) < 1e-12
    xi = oracle.ace_build(phi, kern, s.dv)["Xi"]
    xiu = oracle.ace_build(phiu, kern, s.dv)["Xi"]
    assert rel(oracle.ace_apply(xiu, psi, s.dv), oracle.ace_apply(xi, psi, s.dv)) < 1e-12


def test_single_uniform_orbital():
    """N = 1, phi = 1/sqrt(Omega): rho is constant, only G = 0 survives, so
    W = -K(0)/Omega phi."""
    n, L, omega = 6, 5.0, 0.7
    phi = np.full((1, n, n, n), 1.0 / math.sqrt(L ** 3), dtype=np.complex128)
    kern = oracle.coulomb_kernel((n, n, n), (L, L, L), "erfc", omega)
    W = oracle.exchange_W(phi, kern)
    assert rel(W, -(math.pi / omega ** 2) / L ** 3 * phi) < 1e-13
    kb = oracle.coulomb_kernel((n, n, n), (L, L, L), "bare")
    assert np.max(np.abs(oracle.exchange_W(phi, kb))) < 1e-15


# --------------------------------------------------------------------------- gradient
def test_gradient_euler_and_fd():
    s, phi, psi, kern = _small_system(n=8, L=6.0, nocc=3, kernel="bare")
    g = oracle.energy_grad(phi, kern, s.dv)
    e0 = oracle.energy_direct(phi, kern, s.volume)
    # quartic in Phi: sum Re(conj(g) phi) = 4 E
    assert abs(float(np.real(np.vdot(g, phi))) - 4 * e0) < 1e-12 * abs(e0)
    h = 1e-4
    for d in synth.directions(phi.shape, 4, 99, s.dv):
        ep = oracle.energy_direct(phi + h * d, kern, s.volume)
        em = oracle.energy_direct(phi - h * d, kern, s.volume)
        fd = (ep - em) / (2 * h)
        an = float(np.real(np.vdot(g, d)))
        assert abs(fd - an) < 1e-7 * max(abs(an), 1e-3)


# --------------------------------------------------------------------------- generator
def test_generator_orthonormal_and_real():
    s = synth.GAMMA_24
    phi = synth.orbitals(s, synth.seed_for(1))
    assert phi.dtype == np.float64 and phi.shape == (8, 24, 24, 24)
    gram = s.dv * phi.reshape(8, -1) @ phi.reshape(8, -1).T
    assert np.allclose(gram, np.eye(8), atol=1e-13)
    psi = synth.targets(s, synth.seed_for(1))
    assert psi.shape == (16, 24, 24, 24)
    assert np.allclose(s.dv * np.sum(psi ** 2, axis=(1, 2, 3)), 1.0)


def test_generator_sphere_counts():
    """The coefficient sphere |G|^2/2 <= E_cut on the FFT grid holds exactly
    the integer vectors m with (2 pi/L)^2 |m|^2 / 2 <= E_cut (the sphere fits
    inside the grid's Nyquist box at both sizes)."""
    for n, L in ((24, 10.0), (48, 20.5)):
        g2 = synth.wavevector_sq(n, L)
        r = int(math.ceil(math.sqrt(2 * synth.ECUT_HA) * L / (2 * math.pi)))
        assert r < n // 2
        m = np.arange(-r, r + 1)
        mx, my, mz = np.meshgrid(m, m, m, indexing="ij")
        want = int(np.sum(0.5 * (2 * math.pi / L) ** 2 * (mx ** 2 + my ** 2 + mz ** 2) <= synth.ECUT_HA))
        assert int(np.sum(0.5 * g2 <= synth.ECUT_HA)) == want


# --------------------------------------------------------------------------- oversampling
@pytest.mark.parametrize("real", [False, True])
def test_oversampled_ace(real):
    """Oversampling r = N_phi/N_e > 1 (Sec. 3): V_X stays that of the N_e occupied
    orbitals, and V_ACE built on the N_phi orbitals reproduces it on all of
    them -- checked against the dense V_X matrix of Eq. VXkernel -- while the
    r = 1 operator misses the extra ones; N_phi = N_e reduces to ace_build; E_x
    is that of the occupied block (Eq. EX)."""
    s, phi, psi, kern = _small_system(nocc=7, real=real, kernel="erfc", omega=0.5)
    ne = 4
    out = oracle.ace_build_oversampled(phi, ne, kern, s.dv)
    vx = oracle.vx_matrix(phi[:ne], kern)
    flat = phi.reshape(phi.shape[0], -1)
    w_dense = (vx @ flat.T).T.reshape(phi.shape)
    assert rel(out["W"], w_dense) < 1e-12
    assert rel(oracle.ace_apply(out["Xi"], phi, s.dv), w_dense) < 1e-12
    r1 = oracle.ace_build(phi[:ne], kern, s.dv)
    assert rel(oracle.ace_apply(r1["Xi"], phi[ne:], s.dv), w_dense[ne:]) > 1e-3
    assert rel(out["L"] @ out["L"].conj().T, -out["M"]) < 1e-13
    assert abs(out["Ex"] - oracle.energy_direct(phi[:ne], kern, s.volume)) < 1e-12 * abs(out["Ex"])
    same = oracle.ace_build_oversampled(phi[:ne], ne, kern, s.dv)
    for k in ("W", "M", "Xi"):
        assert rel(same[k], r1[k]) < 1e-14
    assert abs(same["Ex"] - r1["Ex"]) < 1e-14 * abs(r1["Ex"])


def test_kinetic_kernel_plane_waves():
    """The kinetic table |G|^2/2 with the FFT Poisson step applies -1/2 Laplacian:
    a plane wave e^{ik.r} (k on the grid) is an eigenvector with eigenvalue
    |k|^2/2, computed here from the integer wavevector."""
    n, L = 10, 7.0
    kin = oracle.kinetic_kernel((n, n, n), (L, L, L))
    for m in [(0, 0, 0), (1, 0, 0), (2, -3, 1), (-4, 4, 2), (5, 0, -5)]:
        pw = synth.plane_wave_orbitals(n, L, [m])[0]
        k2 = sum((2.0 * math.pi * mi / L) ** 2 for mi in m)
        t = oracle.poisson(pw[None], kin)[0]
        if k2 == 0.0:
            assert np.max(np.abs(t)) < 1e-13
        else:
            assert rel(t, 0.5 * k2 * pw) < 1e-12


@pytest.mark.parametrize("shape,lengths", [((8, 8, 8), (6.0, 6.0, 6.0)), ((8, 6, 5), (6.0, 5.0, 4.5))])
def test_kernel_tables_reflection_symmetric(shape, lengths):
    """Every kernel here depends on |G|^2 only, and the wrapped frequency of
    index n - k is -(that of k), so each table is unchanged by k -> (n - k) mod n
    on every axis, the Nyquist index included: the reading that lets the CUDA
    path store the table over indices 0..n/2 per axis only."""
    tables = [oracle.coulomb_kernel(shape, lengths, "bare"), oracle.coulomb_kernel(shape, lengths, "erfc", 0.4),
              oracle.kinetic_kernel(shape, lengths)]
    for k in tables:
        for axis, n in enumerate(k.shape):
            idx = (-np.arange(n)) % n
            assert np.array_equal(np.take(k, idx, axis=axis), k)
    # and the folded indices cover every value: min(k, n - k) reaches each class once
    n = shape[0]
    assert sorted({min(i, n - i) for i in range(n)}) == list(range(n // 2 + 1))


# ---------------------------------------------------------------- model SCF (Eq. HF, Alg. 1/2)
def _wells(shape, lengths, depth=3.0, width=0.8):
    nz, ny, nx = shape
    lx, ly, lz = lengths
    z, y, x = np.meshgrid(np.arange(nz) * lz / nz, np.arange(ny) * ly / ny, np.arange(nx) * lx / nx, indexing="ij")
    v = np.zeros(shape)
    for c in ((0.25, 0.25, 0.25), (0.75, 0.75, 0.25), (0.75, 0.25, 0.75), (0.25, 0.75, 0.75)):
        dx = (x - c[0] * lx + lx / 2) % lx - lx / 2
        dy = (y - c[1] * ly + ly / 2) % ly - ly / 2
        dz = (z - c[2] * lz + lz / 2) % lz - lz / 2
        v -= depth * np.exp(-(dx * dx + dy * dy + dz * dz) / (2 * width * width))
    return v


def test_model_scf_free_electron():
    """No external potential, one electron: the ground state is the constant
    orbital (G = 0, kinetic energy 0), and its Hartree and exchange potentials
    cancel exactly (spinless HF is free of self-interaction), so the
    eigenvalue is 0 and E_x = -E_H of the uniform density (0 with K(0) = 0)."""
    shape, lengths = (6, 6, 6), (5.0, 5.0, 5.0)
    r = oracle.model_scf(np.zeros(shape), lengths, 1, real=True)
    assert abs(r["eigenvalues"][0]) < 1e-10
    phi = r["psi"][0]
    assert np.allclose(np.abs(phi), np.abs(phi).mean(), rtol=1e-8)
    assert abs(r["ex"]) < 1e-10


def test_model_scf_one_electron_is_the_bare_ground_state():
    """One orbital in a potential well: V_H[|phi|^2] phi + V_X[phi] phi = 0
    exactly, so the self-consistent orbital and eigenvalue are those of
    T + V_loc alone (the lowest eigenpair, by inverse iteration here) and E_x
    equals -1/2 <phi, V_H phi>."""
    shape, lengths = (8, 8, 8), (6.0, 6.0, 6.0)
    v = _wells(shape, lengths)
    r = oracle.model_scf(v, lengths, 1, real=True)
    ng = v.size
    dv = np.prod(lengths) / ng
    kin = oracle.kinetic_kernel(shape, lengths)
    # lowest eigenpair of T + V_loc by inverse iteration with matrix-free solves (CG on H - sigma)
    import scipy.sparse.linalg as sla
    h = sla.LinearOperator((ng, ng), matvec=lambda x: np.real(oracle.poisson(x.reshape(shape), kin)).ravel()
                           + v.ravel() * x, dtype=np.float64)
    w0, u0 = sla.eigsh(h, k=1, which="SA", tol=1e-13)
    assert abs(r["eigenvalues"][0] - w0[0]) < 1e-9
    phi = r["psi"][0].ravel()
    assert abs(abs(np.dot(phi, u0[:, 0])) * np.sqrt(dv) - 1.0) < 1e-9
    bare = oracle.coulomb_kernel(shape, lengths, "bare")
    vh = np.real(oracle.poisson((phi * phi).reshape(shape), bare)).ravel()
    assert abs(r["ex"] + 0.5 * dv * np.sum(phi * vh * phi)) < 1e-10


def test_model_scf_fixed_point_satisfies_hf_equations():
    """At the returned fixed point the orbitals solve H[rho, phi] phi_i =
    eps_i phi_i with H applied matrix-free through the pinned Poisson solve and
    exchange apply (Eq. applyVX2), not the dense matrices the loop used; E_x
    equals the direct pair sum (Eq. EX)."""
    shape, lengths = (8, 8, 8), (6.0, 6.0, 6.0)
    v = _wells(shape, lengths)
    r = oracle.model_scf(v, lengths, 4)
    phi = r["psi"]
    kin = oracle.kinetic_kernel(shape, lengths)
    bare = oracle.coulomb_kernel(shape, lengths, "bare")
    rho = np.sum(np.abs(phi) ** 2, axis=0)
    vh = np.real(oracle.poisson(rho, bare))
    hphi = oracle.poisson(phi, kin) + (v + vh)[None] * phi + oracle.exchange_apply(phi, phi, kern=bare)
    res = hphi - r["eigenvalues"][:, None, None, None] * phi
    assert np.linalg.norm(res) < 1e-8 * np.linalg.norm(hphi)
    assert abs(r["ex"] - oracle.energy_direct(phi, bare, np.prod(lengths))) < 1e-10 * abs(r["ex"])
