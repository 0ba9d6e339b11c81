"""ACE inside the self-consistent iterations of Alg. 2, on a model Hamiltonian.

    H[rho, phi] = -1/2 Laplacian + V_loc + V_H[rho] + V_X[phi]      (Eq. HF, spinless)

on a periodic cell, with a fixed local potential V_loc standing in for the
ions (no pseudopotentials). Alg. 2: each outer iteration builds the ACE
operator once from the current orbitals phi (ace_build: W, M, Cholesky, Xi);
the inner iterations then converge the electron density rho with V_X replaced
by V_ACE = -Xi Xi^* (ace_apply), and the exchange energy comes from Eq. EX_ACE
without a Poisson solve. With ace=False every application of H applies
V_X[phi] through all the pair solves instead (ace_exchange_apply, the inner
loop of Alg. 1): the same fixed point, at a Poisson-solve cost per H
application rather than per outer iteration (Sec. 3).

The inner eigensolver is Chebyshev-filtered subspace iteration: a polynomial
filter in H (only H applications) damps the unwanted part of the spectrum,
then the block is orthonormalised and rotated by Rayleigh-Ritz; the density is
mixed linearly. Every application of -1/2 Laplacian (the kinetic table), of
V_H (the bare Poisson solve) and of V_X / V_ACE runs in this library's kernels;
the eigensolver's small dense algebra (QR, projected eigenproblems, block
combinations) and the products with the local potential use torch.
"""
from __future__ import annotations

import math

import torch

from . import ace


class ModelHF:
    """Plans and operators of the model Hamiltonian on an n^3 grid of a cubic
    cell L. v_loc: real [n, n, n] tensor on the device (Hartree)."""

    def __init__(self, n: int, L: float, n_occ: int, v_loc: torch.Tensor, dtype: str = "c128",
                 kernel: str = "bare", omega: float = 0.0, alpha: float = 1.0, hartree: bool = True):
        self.n, self.L, self.n_occ = n, float(L), n_occ
        # eager launches: the solver's blocks are fresh tensors on every call, so
        # pointer-keyed graph capture would not be reused
        self.x = ace.Plan(n, L, n_occ, dtype=dtype, kernel=kernel, omega=omega, alpha=alpha, graphs=False)
        self.h = ace.Plan(n, L, 1, dtype=dtype, kernel="bare", graphs=False)
        self.t = ace.Plan(n, L, 1, dtype=dtype, kernel="kinetic", graphs=False)
        self.with_hartree = hartree
        self.dtype = dtype
        self.tdtype = ace.TORCH_DTYPES[dtype]
        self.rdtype = torch.float64 if dtype != "c64" else torch.float32
        self.dv = self.x.dv
        self.v_loc = v_loc.to(self.rdtype)
        self.counts = {"build": 0, "ace_apply": 0, "exchange_apply": 0, "h_apply": 0}
        # upper bound of the spectrum: T <= 3 (pi n / L)^2 / 2 on the grid, V_X <= 0
        self.t_max = 1.5 * (math.pi * n / self.L) ** 2

    # ------------------------------------------------------------------ operators
    def density(self, psi: torch.Tensor) -> torch.Tensor:
        """rho = sum_i |psi_i|^2 (Eq. HF)."""
        return torch.sum(psi.real ** 2 + psi.imag ** 2, dim=0) if psi.is_complex() else torch.sum(psi ** 2, dim=0)

    def hartree(self, rho: torch.Tensor) -> torch.Tensor:
        """V_H[rho] (Eq. HF), bare periodic Poisson solve with K(0) = 0 (zero
        when the model leaves the Hartree term out)."""
        if not self.with_hartree:
            return torch.zeros_like(rho)
        v = self.h.poisson(rho.to(self.tdtype)[None].contiguous())[0]
        return v.real if v.is_complex() else v

    def apply(self, psi: torch.Tensor, v_eff: torch.Tensor, xi=None, phi=None) -> torch.Tensor:
        """H psi with V_X replaced by V_ACE (xi given) or applied directly (phi)."""
        out = self.t.poisson(psi)
        out += v_eff[None] * psi
        if xi is not None:
            out += self.x.apply(xi, psi)
            self.counts["ace_apply"] += 1
        else:
            out += self.x.exchange_apply(phi, psi)
            self.counts["exchange_apply"] += 1
        self.counts["h_apply"] += 1
        return out

    # ------------------------------------------------------------------ dense helpers
    def _mat(self, a: torch.Tensor) -> torch.Tensor:
        return a.reshape(a.shape[0], -1)

    def inner(self, a: torch.Tensor, b: torch.Tensor) -> torch.Tensor:
        """Gram matrix dV a^* b over the grid."""
        return self.dv * (self._mat(a).conj() @ self._mat(b).T)

    def orthonormalize(self, s: torch.Tensor) -> torch.Tensor:
        q, _ = torch.linalg.qr(math.sqrt(self.dv) * self._mat(s).T)
        return (q.T / math.sqrt(self.dv)).reshape(s.shape).contiguous()

    # ------------------------------------------------------------------ solver
    def chebyshev(self, x, v_eff, xi, phi, degree, lo, hi, lowest):
        """Chebyshev filter of `degree` in H, damping [lo, hi], scaled at `lowest`."""
        e = 0.5 * (hi - lo)
        c = 0.5 * (hi + lo)
        sigma = e / (lowest - c)
        tau = 2.0 / sigma
        y = (self.apply(x, v_eff, xi, phi) - c * x) * (sigma / e)
        for _ in range(2, degree + 1):
            sigma_new = 1.0 / (tau - sigma)
            y_new = (self.apply(y, v_eff, xi, phi) - c * y) * (2.0 * sigma_new / e) - (sigma * sigma_new) * x
            x, y, sigma = y, y_new, sigma_new
        return y

    def rayleigh_ritz(self, s, v_eff, xi, phi):
        hs = self.apply(s, v_eff, xi, phi)
        h = self.inner(s, hs)
        w, u = torch.linalg.eigh(0.5 * (h + h.conj().T))
        x = torch.tensordot(u.T.to(s.dtype), s, dims=1).contiguous()
        hx = torch.tensordot(u.T.to(s.dtype), hs, dims=1).contiguous()
        return w, x, hx

    def scf(self, psi0: torch.Tensor, use_ace: bool = True, block: int | None = None, degree: int = 10,
            mix: float = 0.4, inner_tol: float = 1e-10, outer_tol: float = 1e-10, max_inner: int = 60,
            max_outer: int = 40) -> dict:
        """Alg. 2 (use_ace) or its V_X-direct counterpart from initial orbitals
        psi0 (n_occ orthonormal vectors). Returns the orbitals, the n_occ lowest
        eigenvalues, E_x per outer iteration, and the operator counts."""
        N = self.n_occ
        k = block or (N + max(2, N // 2))
        gen = torch.Generator(device=psi0.device).manual_seed(5)
        extra = torch.randn((k - N,) + tuple(psi0.shape[1:]), generator=gen, device=psi0.device,
                            dtype=self.rdtype).to(self.tdtype)
        x = self.orthonormalize(torch.cat([psi0.to(self.tdtype), extra]))
        phi = x[:N].contiguous()
        rho = self.density(phi)
        ex_hist = []
        w = None
        for outer in range(max_outer):
            xi = None
            if use_ace:                                   # ACE built once per outer iteration
                xi = self.x.build(phi, want_w=False, want_m=False)["Xi"]
                self.counts["build"] += 1
            for it in range(max_inner):
                v_eff = self.v_loc + self.hartree(rho)
                if w is None:
                    w, x, _ = self.rayleigh_ritz(x, v_eff, xi, None if use_ace else phi)
                hi = self.t_max + float(v_eff.max()) + 1.0
                y = self.chebyshev(x, v_eff, xi, None if use_ace else phi, degree, float(w[-1]), hi, float(w[0]))
                w, x, _ = self.rayleigh_ritz(self.orthonormalize(y), v_eff, xi, None if use_ace else phi)
                rho_out = self.density(x[:N])
                drho = float(torch.sum(torch.abs(rho_out - rho))) * self.dv
                rho = (1.0 - mix) * rho + mix * rho_out
                if drho < inner_tol:
                    break
            psi = x[:N].contiguous()
            # exchange energy of the new orbitals with the operator of this outer
            # iteration: Eq. EX_ACE (V_ACE) or its V_X[phi] counterpart
            vx = self.x.apply(xi, psi) if use_ace else self.x.exchange_apply(phi, psi)
            ex = 0.5 * self.dv * float(torch.sum((psi.conj() * vx).real))
            ex_hist.append(ex)
            phi = psi
            if len(ex_hist) > 1 and abs(ex_hist[-1] - ex_hist[-2]) < outer_tol * abs(ex_hist[-1]):
                break
        return {"psi": phi, "eigenvalues": w[:N].clone(), "ex_history": ex_hist, "outer": len(ex_hist),
                "counts": dict(self.counts)}
