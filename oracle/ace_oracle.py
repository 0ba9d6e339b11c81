"""FP64 CPU oracle for the exchange / ACE hot path (L. Lin, "Adaptively
Compressed Exchange Operator", arXiv:1601.07159).

TEST INFRASTRUCTURE ONLY. Nothing in the product path may import or call this
module: only the tests, the smoke check and the CPU-baseline leg of the bench
use it. It shares no code with the CUDA path (no kernels, headers, tables or
helpers); it reads the same seeded inputs as the GPU side, nothing more.

Every function is the plain definition, written for a reader to check against
the paper by eye: library primitives (numpy FFTs, matmul, LAPACK Cholesky and
triangular solve) are steps; nothing is fused, blocked or reordered, and the
i<->j pair symmetry that the CUDA path exploits is NOT used here.

Conventions (the readings of the paper this oracle takes):

* Arrays are [orbital][z][y][x]; the grid has N_g = n0*n1*n2 points, cell
  volume Omega, dV = Omega/N_g.  Inner products <f, g> = dV sum conj(f) g
  (the discrete form of the integrals in Eq. HF, Eq. ACEconstruct2).
* Poisson-type solve of Eq. applyVX with a periodic G-space kernel K(G):
  rho_hat(G) = N_g^-1 sum_r rho(r) e^{-iG.r},  v(r) = sum_G K(G) rho_hat(G) e^{iG.r}.
  With numpy's conventions that is exactly v = ifftn(K * fftn(rho)).
* K(G) = 4 pi/|G|^2 (bare Coulomb, Eq. VXkernel) or the short-range
  erfc(omega r)/r kernel of Eq. EXSR, whose transform is
  (4 pi/|G|^2)(1 - exp(-|G|^2 / (4 omega^2))).  G = 0: bare K(0) = 0 (no
  divergence correction is mentioned in the paper); screened K(0) = pi/omega^2
  (the analytic limit), both overridable.  alpha scales the whole kernel
  (1/4 for the PBE0/HSE fractions of Eq. ExPBE0/ExHSE; default 1).
* Complex orbitals (the paper writes real ones): V_X(r,r') = -sum_j phi_j(r)
  conj(phi_j(r')) K(r-r'); pair density conj(phi_j) psi; M_kl = <phi_k, W_l>;
  -M = L L^*; Xi = W L^{-*}; V_ACE = -Xi Xi^* (with the dV of the inner
  product).  For real orbitals these reduce to the paper's formulas.

Parity pins live in tests/test_oracle_*.py (closed forms, brute-force dense
DFT, invariants, finite differences); no function here is unpinned.
"""
from __future__ import annotations

import math
import os

import numpy as np
import scipy.fft
import scipy.linalg

_WORKERS = os.cpu_count() or 1


# --------------------------------------------------------------------------
# Kernel in reciprocal space (Eq. applyVX with 1/|r-r'|; Eq. EXSR with erfc)
# --------------------------------------------------------------------------
def reciprocal_sq(shape, lengths) -> np.ndarray:
    """|G|^2 on the wrapped FFT index grid; shape = (n2, n1, n0) = (z, y, x),
    lengths = (Lx, Ly, Lz)."""
    n2, n1, n0 = shape
    lx, ly, lz = lengths
    gx = 2.0 * math.pi * np.fft.fftfreq(n0, d=1.0 / n0) / lx
    gy = 2.0 * math.pi * np.fft.fftfreq(n1, d=1.0 / n1) / ly
    gz = 2.0 * math.pi * np.fft.fftfreq(n2, d=1.0 / n2) / lz
    z, y, x = np.meshgrid(gz, gy, gx, indexing="ij")
    return x * x + y * y + z * z


def coulomb_kernel(shape, lengths, kind="bare", omega=0.0, g0=None, alpha=1.0):
    """K(G): bare 4 pi/G^2 (Eq. VXkernel) or (4 pi/G^2)(1 - e^{-G^2/4 w^2})
    (transform of erfc(w r)/r, Eq. EXSR)."""
    g2 = reciprocal_sq(shape, lengths)
    k = np.zeros_like(g2)
    nz = g2 > 0
    if kind == "bare":
        k[nz] = 4.0 * math.pi / g2[nz]
        k0 = 0.0 if g0 is None else g0
    elif kind == "erfc":
        k[nz] = 4.0 * math.pi / g2[nz] * (1.0 - np.exp(-g2[nz] / (4.0 * omega * omega)))
        k0 = math.pi / (omega * omega) if g0 is None else g0
    else:
        raise ValueError(kind)
    k[~nz] = k0
    return alpha * k


# --------------------------------------------------------------------------
# Poisson solve and the exchange operator (Eq. applyVX, applyVX2, W)
# --------------------------------------------------------------------------
def kinetic_kernel(shape, lengths, alpha=1.0):
    """alpha |G|^2 / 2 on the wrapped grid: with poisson() below it applies the
    kinetic-energy operator -1/2 Laplacian of Eq. HF spectrally."""
    return alpha * 0.5 * reciprocal_sq(shape, lengths)


def poisson(rho: np.ndarray, kern: np.ndarray) -> np.ndarray:
    """v = sum_G K(G) rho_hat(G) e^{iG.r}; rho may carry leading batch axes."""
    axes = (-3, -2, -1)
    rho_hat = scipy.fft.fftn(rho, axes=axes, workers=_WORKERS)
    return scipy.fft.ifftn(kern * rho_hat, axes=axes, workers=_WORKERS)


def exchange_apply(phi: np.ndarray, psi: np.ndarray, kern: np.ndarray) -> np.ndarray:
    """(V_X[phi] psi_b)(r) = -sum_j phi_j(r) Poisson[conj(phi_j) psi_b](r)
    (Eq. applyVX2), all N x N_b pair solves, no pair symmetry used."""
    phi = np.asarray(phi, dtype=np.complex128)
    psi = np.asarray(psi, dtype=np.complex128)
    out = np.empty(psi.shape, dtype=np.complex128)
    for b in range(psi.shape[0]):
        rho = np.conj(phi) * psi[b][None]          # N pair densities
        v = poisson(rho, kern)
        out[b] = -np.sum(phi * v, axis=0)
    return out


def exchange_W(phi: np.ndarray, kern: np.ndarray) -> np.ndarray:
    """W_i = V_X[phi] phi_i (Eq. W)."""
    return exchange_apply(phi, phi, kern)


# --------------------------------------------------------------------------
# ACE construction (Eq. ACEconstruct1-2, the Cholesky step, Eq. Wtilde, ACE)
# --------------------------------------------------------------------------
def _mat(a: np.ndarray) -> np.ndarray:
    """[count][grid] -> N_g x count matrix (columns = orbitals)."""
    return a.reshape(a.shape[0], -1).T


def _unmat(m: np.ndarray, shape) -> np.ndarray:
    return np.ascontiguousarray(m.T).reshape(shape)


def overlap_M(phi: np.ndarray, W: np.ndarray, dv: float) -> np.ndarray:
    """M_kl = <phi_k, W_l> = dV sum_r conj(phi_k) W_l, then the Hermitian part
    (M is Hermitian negative semidefinite in exact arithmetic)."""
    m = dv * (_mat(phi).conj().T @ _mat(W))
    return 0.5 * (m + m.conj().T)


def cholesky_neg(M: np.ndarray) -> np.ndarray:
    """Lower-triangular L with -M = L L^* (LAPACK potrf)."""
    return scipy.linalg.cholesky(-M, lower=True)


def xi_from(W: np.ndarray, L: np.ndarray) -> np.ndarray:
    """Xi = W L^{-*}, i.e. xi_k = sum_i W_i (L^{-*})_ik (Eq. Wtilde), computed
    as Xi^* = L^{-1} W^* by a triangular solve."""
    xih = scipy.linalg.solve_triangular(L, _mat(W).conj().T, lower=True)
    return _unmat(xih.conj().T, W.shape)


def ace_build(phi: np.ndarray, kern: np.ndarray, dv: float) -> dict:
    """Alg. 2 steps 2-3: W, M, L, Xi, and E_x = 1/2 Re tr M."""
    W = exchange_W(phi, kern)
    M = overlap_M(phi, W, dv)
    L = cholesky_neg(M)
    Xi = xi_from(W, L)
    return {"W": W, "M": M, "L": L, "Xi": Xi, "Ex": 0.5 * float(np.real(np.trace(M)))}


def ace_build_oversampled(phi: np.ndarray, n_occ: int, kern: np.ndarray, dv: float) -> dict:
    """ACE with oversampling r = N_phi / N_e > 1 (Sec. 3, last paragraph): the
    exchange operator is that of the N_e = n_occ occupied orbitals phi[:n_occ],
    W_i = V_X[phi_occ] phi_i for all N_phi orbitals, then M, L, Xi over the N_phi
    columns as in ace_build. E_x = 1/2 Re tr of the occupied block of M."""
    phi = np.asarray(phi, dtype=np.complex128)
    W = exchange_apply(phi[:n_occ], phi, kern)
    M = overlap_M(phi, W, dv)
    L = cholesky_neg(M)
    Xi = xi_from(W, L)
    ex = 0.5 * float(np.real(np.trace(M[:n_occ, :n_occ])))
    return {"W": W, "M": M, "L": L, "Xi": Xi, "Ex": ex}


def ace_apply(xi: np.ndarray, psi: np.ndarray, dv: float) -> np.ndarray:
    """V_ACE psi = -sum_k xi_k <xi_k, psi> (Eq. ACE)."""
    c = dv * (_mat(xi).conj().T @ _mat(np.asarray(psi, dtype=np.complex128)))
    return _unmat(-(_mat(xi) @ c), psi.shape)


# --------------------------------------------------------------------------
# Exchange energy (Eq. EX, Eq. EX_ACE) and its gradient
# --------------------------------------------------------------------------
def energy_direct(phi: np.ndarray, kern: np.ndarray, volume: float) -> float:
    """E_x = -1/2 sum_ij <rho_ij, Poisson rho_ij> = -1/2 sum_ij Omega sum_G
    K(G) |rho_hat_ij(G)|^2 (Eq. EX by Parseval), all ordered pairs."""
    phi = np.asarray(phi, dtype=np.complex128)
    ng = phi[0].size
    total = 0.0
    for i in range(phi.shape[0]):
        rho = np.conj(phi) * phi[i][None]
        rho_hat = scipy.fft.fftn(rho, axes=(-3, -2, -1), workers=_WORKERS) / ng
        total += float(np.sum(kern[None] * np.abs(rho_hat) ** 2))
    return -0.5 * volume * total


def energy_ace(xi: np.ndarray, phi: np.ndarray, dv: float) -> float:
    """E_x = -1/2 sum_ik |<xi_k, phi_i>|^2 (Eq. EX_ACE)."""
    c = dv * (_mat(xi).conj().T @ _mat(np.asarray(phi, dtype=np.complex128)))
    return -0.5 * float(np.sum(np.abs(c) ** 2))


def energy_grad(phi: np.ndarray, kern: np.ndarray, dv: float) -> np.ndarray:
    """Gradient of E_x in the torch convention dE/dRe + i dE/dIm: each orbital
    enters E four times and K is symmetric, so g_k(r) = 2 dV W_k(r)."""
    return 2.0 * dv * exchange_W(phi, kern)


# --------------------------------------------------------------------------
# Brute force (no FFT library): dense DFT sums and the explicit V_X matrix
# --------------------------------------------------------------------------
def dft_matrix(n: int, sign: int) -> np.ndarray:
    j = np.arange(n)
    return np.exp(sign * 2j * math.pi * np.outer(j, j) / n)


def poisson_bruteforce(rho: np.ndarray, kern: np.ndarray) -> np.ndarray:
    """v(r) = sum_G K(G) [N_g^-1 sum_r' rho(r') e^{-iG.r'}] e^{iG.r} by explicit
    summation over all grid points and wavevectors (O(N_g^2))."""
    n2, n1, n0 = rho.shape
    ng = rho.size
    # explicit phase matrix e^{-iG.r} over flattened (G, r) index pairs
    iz, iy, ix = np.meshgrid(np.arange(n2), np.arange(n1), np.arange(n0), indexing="ij")
    r = np.stack([ix.ravel() / n0, iy.ravel() / n1, iz.ravel() / n2], axis=1)   # fractional
    mz, my, mx = np.meshgrid(np.fft.fftfreq(n2, 1.0 / n2), np.fft.fftfreq(n1, 1.0 / n1),
                             np.fft.fftfreq(n0, 1.0 / n0), indexing="ij")
    m = np.stack([mx.ravel(), my.ravel(), mz.ravel()], axis=1)
    phase = np.exp(-2j * math.pi * (m @ r.T))          # [G][r]
    rho_hat = phase @ rho.ravel() / ng
    v = phase.conj().T @ (kern.ravel() * rho_hat)
    return v.reshape(rho.shape)


def kernel_realspace(kern: np.ndarray) -> np.ndarray:
    """K_r(d) = N_g^-1 sum_G K(G) e^{iG.d}: the periodic real-space kernel, so
    that Poisson[rho](r) = sum_r' K_r(r - r') rho(r'). Explicit sum."""
    return poisson_bruteforce(_delta(kern.shape), kern)


def _delta(shape) -> np.ndarray:
    d = np.zeros(shape, dtype=np.complex128)
    d[0, 0, 0] = 1.0
    return d


def kernel_matrix(kern: np.ndarray) -> np.ndarray:
    """K_mat[r, r'] = K_r(r - r') over all pairs of grid points (periodic)."""
    n2, n1, n0 = kern.shape
    kr = kernel_realspace(kern)
    iz, iy, ix = np.meshgrid(np.arange(n2), np.arange(n1), np.arange(n0), indexing="ij")
    iz, iy, ix = iz.ravel(), iy.ravel(), ix.ravel()
    return kr[(iz[:, None] - iz[None, :]) % n2,
              (iy[:, None] - iy[None, :]) % n1,
              (ix[:, None] - ix[None, :]) % n0]


def vx_matrix(phi: np.ndarray, kern: np.ndarray) -> np.ndarray:
    """Dense V_X on the grid from Eq. VXkernel: V_X(r, r') = -Gamma(r, r')
    K_r(r - r'), the Hadamard product of the density matrix
    Gamma(r,r') = sum_j phi_j(r) conj(phi_j(r')) with the Coulomb kernel.
    Acts on grid vectors as (V_X psi)(r) = sum_r' V_X(r, r') psi(r')."""
    p = _mat(np.asarray(phi, dtype=np.complex128))
    gamma = p @ p.conj().T
    return -gamma * kernel_matrix(kern)


# --------------------------------------------------------------------------
# Self-consistent field of a model Hamiltonian (Eq. HF; the loops of Alg. 1/2)
# --------------------------------------------------------------------------
def model_scf(v_loc: np.ndarray, lengths, n_occ: int, mix: float = 0.5, tol: float = 1e-11,
              max_iter: int = 300, real: bool = False) -> dict:
    """Ground state of the spinless Hartree-Fock model H = -1/2 Laplacian +
    V_loc + V_H[rho] + V_X[Gamma] (Eq. HF) on the grid of v_loc, by dense
    diagonalisation: every iteration builds H as a dense N_g x N_g matrix
    (the kinetic and Hartree parts from the periodic G-space kernels, V_X from
    Eq. VXkernel with the current density matrix Gamma), takes its n_occ
    lowest eigenvectors, and mixes Gamma linearly with the new one, until the
    new Gamma equals the old to `tol`. The fixed point is the self-consistent
    solution that Alg. 1 and Alg. 2 reach by their inner and outer loops.
    Returns the orbitals [n_occ][grid] (dV sum |phi|^2 = 1), the n_occ lowest
    eigenvalues of the final H, E_x = 1/2 dV sum_i <phi_i, V_X phi_i> and the
    iteration count. Small grids only (N_g^2 dense matrices)."""
    shape = v_loc.shape
    ng = v_loc.size
    vol = float(np.prod(lengths))
    dv = vol / ng
    kin = kinetic_kernel(shape, lengths)
    bare = coulomb_kernel(shape, lengths, "bare")
    unit = np.eye(ng).reshape((ng,) + shape)
    t_mat = _mat(poisson(unit, kin))                 # column j = T e_j
    k_mat = kernel_matrix(bare)
    dtype = np.float64 if real else np.complex128

    def hamiltonian(gamma):
        rho = np.real(np.diag(gamma))
        v_h = np.real(poisson(rho.reshape(shape), bare)).ravel()
        h = t_mat + np.diag(v_loc.ravel() + v_h) - gamma * k_mat
        h = 0.5 * (h + h.conj().T)
        return (h.real if real else h).astype(dtype)

    def occupied(h):
        w, u = scipy.linalg.eigh(h)
        phi = u[:, :n_occ] / math.sqrt(dv)           # dV sum |phi|^2 = 1
        return w, phi, phi @ phi.conj().T

    w, phi, gamma = occupied((t_mat + np.diag(v_loc.ravel())).real if real else t_mat + np.diag(v_loc.ravel()))
    it = 0
    for it in range(1, max_iter + 1):
        w, phi, g_out = occupied(hamiltonian(gamma))
        change = np.linalg.norm(g_out - gamma) / np.linalg.norm(g_out)
        gamma = (1.0 - mix) * gamma + mix * g_out
        if change < tol:
            break
    w, phi, gamma = occupied(hamiltonian(g_out))
    vx_phi = -(gamma * k_mat) @ phi
    ex = 0.5 * dv * float(np.real(np.sum(np.conj(phi) * vx_phi)))
    orbitals = np.ascontiguousarray(phi.T).reshape((n_occ,) + shape)
    return {"psi": orbitals, "eigenvalues": w[:n_occ], "ex": ex, "iterations": it}
