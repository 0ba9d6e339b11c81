"""Run a few ACE builds (and applies) of one workload for an external profiler.

    python -m paper_1601_07159_gb300.profile_run [--n 96] [--L 41] [--n-occ 1024]
        [--bands 0] [--builds 2] [--eager] [--kernel erfc] [--omega 0.106]

Each build is ace_build (W, M, Cholesky, Xi) followed, with --bands > 0, by
ace_apply on that many bands. The orbitals are seeded complex Gaussian values
on the device, scaled to dV sum |phi|^2 ~ 1 but not orthogonalised (the time of
every kernel is independent of the values; -M stays positive definite), so no
host or device QR runs inside the profiled process. --eager launches every
pair pass separately (graphs off), so a profiler sees and names each kernel of
a pair batch; by default the pair section runs from captured graphs as in the
benchmark. Prints the plan's status word at the end (0 = no device-side
failure).
"""
from __future__ import annotations

import argparse


def main(argv=None) -> int:
    ap = argparse.ArgumentParser()
    ap.add_argument("--n", type=int, default=96)
    ap.add_argument("--L", type=float, default=41.0)
    ap.add_argument("--n-occ", type=int, default=1024)
    ap.add_argument("--bands", type=int, default=0)
    ap.add_argument("--builds", type=int, default=2)
    ap.add_argument("--eager", action="store_true")
    ap.add_argument("--kernel", default="erfc")
    ap.add_argument("--omega", type=float, default=0.106)
    ap.add_argument("--seed", type=int, default=5)
    args = ap.parse_args(argv)

    import torch
    from . import build_lib
    build_lib.build()
    from . import ace

    torch.cuda.set_device(0)
    n, N = args.n, args.n_occ
    dv = args.L ** 3 / n ** 3
    scale = (2.0 * n ** 3 * dv) ** -0.5
    g = torch.Generator(device="cuda").manual_seed(args.seed)

    def vectors(count):
        shape = (count, n, n, n)
        return torch.complex(torch.randn(shape, generator=g, device="cuda"),
                             torch.randn(shape, generator=g, device="cuda")) * scale

    phi = vectors(N)
    psi = vectors(args.bands) if args.bands > 0 else None
    plan = ace.Plan(n, args.L, N, dtype="c64", kernel=args.kernel, omega=args.omega, graphs=not args.eager)
    xi = plan.empty(N)
    y = plan.empty(args.bands) if psi is not None else None
    for _ in range(args.builds):
        plan.build(phi, want_w=False, want_m=False, xi=xi)
        if psi is not None:
            plan.apply(xi, psi, out=y)
    torch.cuda.synchronize()
    code, info = plan.status()
    print("status", code, info)
    return 0 if code == 0 else 1


if __name__ == "__main__":
    raise SystemExit(main())
