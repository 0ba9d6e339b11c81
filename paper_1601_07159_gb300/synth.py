"""Seeded synthetic inputs: orbitals and target vectors on a periodic grid.

This module builds *inputs* only. It holds none of the exchange / ACE
arithmetic, imports nothing else from this package and nothing from the
oracle, so the oracle (test infrastructure) and the CUDA path can both be fed
from it without sharing method code.

Workloads are shaped like the silicon runs of Sec. 4 (Si8/Si64/Si216/Si512,
Gamma-point, plane-wave basis):

* cubic cell of edge ``L`` (bohr) sampled on an ``n^3`` grid, x fastest (or an
  orthorhombic cell L_x x L_y x L_z on an n_x x n_y x n_z grid);
* reciprocal vectors G = 2*pi*m/L per axis with the wrapped FFT index m;
* orbital coefficients c(G) = (a + i b)/sqrt(2) * exp(-|G|^2 / (2 E_cut)) on
  the sphere |G|^2/2 <= E_cut (E_cut = 10 Ha), zero outside, a, b ~ N(0, 1);
* real Gamma-point orbitals enforce c(-G) = conj c(G) and a real c(0);
* phi(r) = sum_G c(G) exp(i G.r), then a QR factorisation of sqrt(dV)*Phi
  with diag(R) > 0 makes the columns orthonormal in the discrete inner
  product <f, g> = dV sum_r conj(f) g (the orthonormality of Eq. HF);
* target vectors psi use the same recipe with seed + 500, normalised but not
  orthogonalised against Phi.

Arrays are numpy, shape (count, n_z, n_y, n_x) = [orbital][z][y][x], FP64
(complex128, or float64 for real Gamma-point systems).
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

ECUT_HA = 10.0
SEED_BASE = 1601071590
SHAPE_SEED_BATCHED = 1601074590


@dataclasses.dataclass(frozen=True)
class System:
    """Shape of one periodic system: a cubic cell of edge L on an n^3 grid, or
    an orthorhombic cell `cell` = (L_x, L_y, L_z) on a `grid` = (n_x, n_y, n_z)
    grid (then n and L are not used)."""

    n: int                 # grid points per edge
    L: float               # cell edge (bohr)
    n_occ: int             # exchange orbitals N
    n_bands: int           # target vectors psi
    real: bool = False     # real Gamma-point orbitals
    kernel: str = "bare"   # "bare" or "erfc"
    omega: float = 0.0     # screening parameter (bohr^-1) for "erfc"
    grid: tuple | None = None   # (n_x, n_y, n_z) of a non-cubic grid
    cell: tuple | None = None   # (L_x, L_y, L_z) of a non-cubic cell

    @property
    def nxyz(self) -> tuple:
        return tuple(self.grid) if self.grid else (self.n,) * 3

    @property
    def lengths(self) -> tuple:
        return tuple(self.cell) if self.cell else (self.L,) * 3

    @property
    def shape(self) -> tuple:
        """Array shape of one vector: (n_z, n_y, n_x)."""
        nx, ny, nz = self.nxyz
        return (nz, ny, nx)

    @property
    def ng(self) -> int:
        nx, ny, nz = self.nxyz
        return nx * ny * nz

    @property
    def volume(self) -> float:
        lx, ly, lz = self.lengths
        return lx * ly * lz

    @property
    def dv(self) -> float:
        return self.volume / self.ng


# The five workloads, sizes per the silicon runs of Sec. 4 (Eq. numbering of
# the paper is used in docstrings elsewhere).
GAMMA_24 = System(n=24, L=10.0, n_occ=8, n_bands=16, real=True, kernel="bare")
SI64_48 = System(n=48, L=20.5, n_occ=128, n_bands=192, kernel="erfc", omega=0.106)
DIFF_64 = System(n=64, L=20.5 * 64 / 48, n_occ=256, n_bands=384, kernel="bare")
SI512_96 = System(n=96, L=41.0, n_occ=1024, n_bands=1536, kernel="erfc", omega=0.106)

WORKLOADS = {
    "gamma24_n8_fp64": (1, GAMMA_24),
    "si64_48cube_n128": (2, SI64_48),
    "diff_64cube_n256": (4, DIFF_64),
    "si512_96cube_n1024": (5, SI512_96),
}


def batched_systems(count: int = 64, seed: int = SHAPE_SEED_BATCHED):
    """Uneven batch: edges uniform in {32,36,40,48,64}, N uniform in [16,128],
    bands = floor(1.5 N), L scaled so the grid spacing matches the 48^3 cell."""
    rng = np.random.Generator(np.random.PCG64(seed))
    edges = np.array([32, 36, 40, 48, 64])
    out = []
    for _ in range(count):
        n = int(edges[rng.integers(0, len(edges))])
        nocc = int(rng.integers(16, 129))
        out.append(System(n=n, L=20.5 * n / 48, n_occ=nocc,
                          n_bands=(3 * nocc) // 2, kernel="bare"))
    return out


def seed_for(config_index: int, system_index: int = 0) -> int:
    return SEED_BASE + 1000 * config_index + system_index


def wavevector_sq(n: int, L: float) -> np.ndarray:
    """|G|^2 on the wrapped n^3 index grid, array [z][y][x]."""
    m = np.fft.fftfreq(n, d=1.0 / n)
    g = 2.0 * math.pi * m / L
    gz, gy, gx = np.meshgrid(g, g, g, indexing="ij")
    return gx * gx + gy * gy + gz * gz


def wavevector_sq3(shape, lengths) -> np.ndarray:
    """|G|^2 on the wrapped index grid of shape (n_z, n_y, n_x), cell (L_x, L_y, L_z)."""
    nz, ny, nx = shape
    lx, ly, lz = lengths
    gx = 2.0 * math.pi * np.fft.fftfreq(nx, d=1.0 / nx) / lx
    gy = 2.0 * math.pi * np.fft.fftfreq(ny, d=1.0 / ny) / ly
    gz = 2.0 * math.pi * np.fft.fftfreq(nz, d=1.0 / nz) / lz
    z, y, x = np.meshgrid(gz, gy, gx, indexing="ij")
    return x * x + y * y + z * z


def _coefficients(rng, sysm: System, count: int, ecut: float) -> np.ndarray:
    shape = sysm.shape
    g2 = wavevector_sq3(shape, sysm.lengths)
    sphere = 0.5 * g2 <= ecut
    decay = np.where(sphere, np.exp(-g2 / (2.0 * ecut)), 0.0)
    a = rng.standard_normal((count,) + shape)
    b = rng.standard_normal((count,) + shape)
    c = (a + 1j * b) / math.sqrt(2.0) * decay
    if sysm.real:
        # Hermitian symmetry c(-G) = conj c(G): average with the mirrored conjugate.
        iz, iy, ix = ((-np.arange(m)) % m for m in shape)
        mirror = np.conj(c[:, iz][:, :, iy][:, :, :, ix])
        c = 0.5 * (c + mirror)
        c[:, 0, 0, 0] = c[:, 0, 0, 0].real
    return c


def _to_real_space(c: np.ndarray) -> np.ndarray:
    ng = c.shape[1] * c.shape[2] * c.shape[3]
    return np.fft.ifftn(c, axes=(1, 2, 3)) * ng


def orbitals(sysm: System, seed: int, ecut: float = ECUT_HA) -> np.ndarray:
    """Orthonormal exchange orbitals Phi, shape (N, n, n, n)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    phi = _to_real_space(_coefficients(rng, sysm, sysm.n_occ, ecut))
    if sysm.real:
        phi = phi.real
    a = math.sqrt(sysm.dv) * phi.reshape(sysm.n_occ, -1).T
    q, r = np.linalg.qr(a)
    sgn = np.sign(np.real(np.diag(r)))
    sgn[sgn == 0] = 1.0
    q = q * sgn[None, :]
    out = (q.T / math.sqrt(sysm.dv)).reshape((sysm.n_occ,) + sysm.shape)
    return np.ascontiguousarray(out)


def targets(sysm: System, seed: int, count: int | None = None,
            ecut: float = ECUT_HA) -> np.ndarray:
    """Target vectors psi (bands), each normalised, shape (count, n, n, n)."""
    count = sysm.n_bands if count is None else count
    rng = np.random.Generator(np.random.PCG64(seed + 500))
    psi = _to_real_space(_coefficients(rng, sysm, count, ecut))
    if sysm.real:
        psi = psi.real
    nrm = np.sqrt(sysm.dv * np.sum(np.abs(psi) ** 2, axis=(1, 2, 3)))
    return np.ascontiguousarray(psi / nrm[:, None, None, None])


def plane_wave_orbitals(n: int, L: float, mvecs) -> np.ndarray:
    """phi_i(r) = exp(i k_i.r)/sqrt(Omega) for integer wavevector indices m_i
    (k_i = 2*pi*m_i/L), shape (len(mvecs), n, n, n)."""
    x = np.arange(n) * (L / n)
    z3, y3, x3 = np.meshgrid(x, x, x, indexing="ij")
    out = []
    for (mx, my, mz) in mvecs:
        k = 2.0 * math.pi / L
        out.append(np.exp(1j * k * (mx * x3 + my * y3 + mz * z3)))
    return np.array(out) / math.sqrt(L ** 3)


def random_unitary(count: int, seed: int) -> np.ndarray:
    rng = np.random.Generator(np.random.PCG64(seed))
    a = rng.standard_normal((count, count)) + 1j * rng.standard_normal((count, count))
    q, r = np.linalg.qr(a)
    return q * (np.diag(r) / np.abs(np.diag(r)))[None, :]


def directions(shape, count: int, seed: int, dv: float) -> np.ndarray:
    """Seeded complex Gaussian directions D normalised to dV ||D||^2 = 1."""
    rng = np.random.Generator(np.random.PCG64(seed))
    d = rng.standard_normal((count,) + tuple(shape)) + 1j * rng.standard_normal((count,) + tuple(shape))
    nrm = np.sqrt(dv * np.sum(np.abs(d) ** 2, axis=tuple(range(1, d.ndim))))
    return d / nrm.reshape((count,) + (1,) * len(shape))


# --------------------------------------------------------------------------
# The same recipe on a CUDA device (torch), for workloads whose host QR and
# host arrays are too large to build per run (96^3 x 1024 orbitals: 14.5 GB in
# FP64, a 884736 x 1024 QR). The random stream is torch's, so these arrays are
# not the host ones above; the distribution and structure are the same.
# --------------------------------------------------------------------------
def _device_coefficients(sysm: System, count: int, gen, ecut: float, device):
    import torch
    n = sysm.n
    m = torch.fft.fftfreq(n, d=1.0 / n, device=device, dtype=torch.float64) * (2 * math.pi / sysm.L)
    g2 = m[:, None, None] ** 2 + m[None, :, None] ** 2 + m[None, None, :] ** 2
    decay = torch.where(0.5 * g2 <= ecut, torch.exp(-g2 / (2 * ecut)), torch.zeros_like(g2)).to(torch.float32)
    out = torch.empty((count, n, n, n), dtype=torch.complex64, device=device)
    for i in range(0, count, 64):
        k = min(64, count - i)
        c = torch.complex(torch.randn((k, n, n, n), generator=gen, device=device),
                          torch.randn((k, n, n, n), generator=gen, device=device)) / math.sqrt(2.0)
        out[i:i + k] = torch.fft.ifftn(c * decay, dim=(1, 2, 3)) * n ** 3
    return out


def orbitals_device(sysm: System, seed: int, device="cuda", ecut: float = ECUT_HA):
    """Orthonormal complex orbitals (N, n, n, n) complex64 on `device`: the
    recipe of orbitals() with torch's generator and a QR on the device."""
    import torch
    gen = torch.Generator(device=device).manual_seed(seed)
    phi = _device_coefficients(sysm, sysm.n_occ, gen, ecut, device)
    q, r = torch.linalg.qr(math.sqrt(sysm.dv) * phi.reshape(sysm.n_occ, -1).T)
    q = q * torch.sgn(torch.diagonal(r).real)[None, :]
    del phi, r
    return (q.T / math.sqrt(sysm.dv)).contiguous().reshape(sysm.n_occ, sysm.n, sysm.n, sysm.n)


def targets_device(sysm: System, seed: int, count: int | None = None, device="cuda", ecut: float = ECUT_HA):
    """Target vectors (count, n, n, n) complex64 on `device`, each normalised,
    not orthogonalised: the recipe of targets() with torch's generator."""
    import torch
    count = sysm.n_bands if count is None else count
    gen = torch.Generator(device=device).manual_seed(seed + 500)
    psi = _device_coefficients(sysm, count, gen, ecut, device)
    for i in range(0, count, 64):
        blk = psi[i:i + 64]
        nrm = torch.sqrt(sysm.dv * torch.sum(torch.abs(blk) ** 2, dim=(1, 2, 3)))
        blk /= nrm[:, None, None, None]
    return psi
