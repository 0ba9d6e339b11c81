#!/usr/bin/env python3
"""Benchmark of the ACE hot path on one GB300 (or N independent replicas).

Workloads (--workload; seeded synthetic orbitals shaped like the silicon runs):

* si512_96cube_n1024 (default): 96^3 grid, L = 41 bohr, N = 1024 orbitals,
  1536 bands, complex, screened kernel omega = 0.106 (Si512-like). A step is
  ace_build (W over the 524,800 unique pair FFT-Poisson solves, M = dV Phi^* W,
  FP64 Cholesky and L^{-1}, Xi = W L^{-*}, E_x) followed by ace_apply on the
  1536 bands.
* si64_48cube_n128: the same step at 48^3, L = 20.5, N = 128, 192 bands
  (Si64-like), 8256 unique pairs.
* batched64_uneven: one ace_build_batched of 64 uneven systems per step.

The metric is unique pair FFT-Poisson solves per second of whole steps.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--workload NAME]

Under torchrun each rank runs an independent replica (its own system): the
work is partitioned into independent problems, no data-path collective;
value = pairs over all ranks / max-over-ranks time ("scaling": "weak").

Besides the contract keys the default line carries: ms per build and per
apply; the pair pipeline's roofline; the end-to-end rate through pinned host
buffers; the oracle on a bounded sample of the same workload (cpu_baseline);
and, on one GPU, extra keys for the 48^3 workload (with its plain-FP64 build,
a cuFFT/torch W build, the direct-energy and Poisson entry points and an
oversampled build) and for the 64-system batch. The --no-* flags skip extras.

--impl reference times the FP64 CPU oracle on this host (rank 0 only), each
step a bounded sample of the same workload, extrapolated to a whole step.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_1601_07159_gb300 import synth  # noqa: E402

LARGE = "si512_96cube_n1024"
SI64 = "si64_48cube_n128"
BATCHED = "batched64_uneven"
SINGLE = {LARGE: (5, synth.SI512_96), SI64: (2, synth.SI64_48)}
METRIC = "pair FFT-Poisson solves/s"
UNIT = "pair-solves/s"
# DRAM bytes (read + write) of passes A-D per ace_build from an ncu capture of
# the current kernels on the default schedule, scaled from the captured pair
# batches to a whole build (workload -> (bytes, how it was taken)).
TRAFFIC = {
    LARGE: (25.80e12, "ncu dram__bytes_read.sum + dram__bytes_write.sum (--cache-control none) of passes A-D "
                      "on one off-diagonal 64-pair batch of the 96^3 grid (3146 MB; profile_run --n 96 --n-occ 24 "
                      "--eager, second batch), x 8200 batch equivalents (524,800 pairs / 64)"),
    SI64: (12.07e9, "ncu dram__bytes_read.sum + dram__bytes_write.sum (--cache-control none) of passes A-D "
                    "on the second off-diagonal 64-pair batch at 48^3 (93.5 MB; profile_run --n 48 --n-occ 128 "
                    "--eager), x 129 batch equivalents (8256 pairs / 64)"),
}


def parse(argv=None):
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=5)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", choices=["ours", "reference"], default="ours")
    p.add_argument("--workload", choices=[LARGE, SI64, BATCHED], default=LARGE)
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-extras", action="store_true", help="skip the 48^3 and batched extra keys")
    p.add_argument("--no-fp64", action="store_true")
    p.add_argument("--no-cufft", action="store_true", help="skip the cuFFT comparison")
    p.add_argument("--no-oversampled", action="store_true", help="skip the oversampled-build timing")
    p.add_argument("--no-entries", action="store_true",
                   help="skip the timings of the direct-energy and Poisson entry points")
    p.add_argument("--max-pairs", type=int, default=0, help="pair solves per batch (0 = plan default)")
    p.add_argument("--tile", type=int, default=0, help="orbitals per tile side (0 = plan default)")
    p.add_argument("--lanes", type=int, default=0, help="concurrent batch streams (0 = plan default)")
    p.add_argument("--eager", action="store_true",
                   help="four kernels per batch, launched eagerly (per-pass timings)")
    p.add_argument("--engine", action="store_true", help="persistent pair engine")
    p.add_argument("--no-pdl", action="store_true", help="no programmatic dependent launch")
    p.add_argument("--no-overlap", action="store_true",
                   help="spread a round's batches over lanes instead of overlapping pass A with pass D")
    p.add_argument("--chains", type=int, default=0, help="concurrent stream chains of a batch (0 = default)")
    p.add_argument("--radix", type=int, default=0, choices=[0, 1],
                   help="FFT radix order: 0 radix 4 first (default), 1 odd radix first")
    p.add_argument("--systems", type=int, default=64, help="systems of the batched workload")
    return p.parse_args(argv)


def default_schedule(args):
    return (args.max_pairs, args.tile, args.lanes, args.eager, args.engine, args.no_pdl, args.no_overlap,
            args.radix) == (0, 0, 0, False, False, False, False, 0)


def workload_config(name, s):
    return {"workload": name, "grid": f"{s.n}^3", "L_bohr": s.L, "n_occ": s.n_occ,
            "n_bands": s.n_bands, "kernel": f"erfc omega={s.omega}" if s.kernel == "erfc" else "bare",
            "orbitals": "seeded Gaussian-decaying plane waves |G|^2/2<=10 Ha, QR-orthonormal",
            "precision": "fp32 pair/FFT path, TF32 3-term-split M and apply, fp64 Cholesky and L^-1, "
                         "Xi = W L^-* to fp64 accuracy (fp16 tensor-core slices)",
            "l2": "working set > L2 every step (no flush needed)"}


def unique_pairs(n):
    return n * (n + 1) // 2


def pair_model_bytes(s):
    """Algorithmic bytes of one W build: 32 B per grid point per unique pair
    (two global transposes of the spectrum) + the Phi read and the W write."""
    return 32.0 * s.ng * unique_pairs(s.n_occ) + 2.0 * s.n_occ * s.ng * 8


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


# ----------------------------------------------------------------------------- clocks
class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.idx = gpu_index
        self.proc = None
        self.file = None

    def start(self):
        try:
            self.file = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.idx), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=self.file, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.file.flush()
        self.file.seek(0)
        rows = [r.strip().split(",") for r in self.file.read().splitlines() if r.strip()]
        os.unlink(self.file.name)
        sm, mx, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            try:
                sm.append(float(r[0]))
                mx = max(mx, float(r[1]))
                for k, nm in enumerate(names):
                    if r[4 + k].strip().lower() == "active":
                        reasons.add(nm)
            except (ValueError, IndexError):
                continue
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def physical_gpu_index(local_rank):
    vis = os.environ.get("CUDA_VISIBLE_DEVICES")
    if vis:
        items = [v.strip() for v in vis.split(",") if v.strip()]
        if local_rank < len(items) and items[local_rank].isdigit():
            return int(items[local_rank])
    return local_rank


# ----------------------------------------------------------------------------- oracle
def oracle_sample(s, seed, pair_budget_s=12.0, rows_div=None, min_pairs=2):
    """Time the FP64 oracle on a bounded sample of one step of workload `s` and
    extrapolate to the whole step.

    Pair section: ordered FFT-Poisson solves of Eq. applyVX2 (the oracle uses
    no pair symmetry, so a W build is N^2 of them) on seeded host orbitals of
    the workload's grid (16 orbitals; an FFT's cost does not depend on the
    values), as many as fit in about `pair_budget_s`. Dense section (M = dV
    Phi^* W, Cholesky, Xi = W L^{-*}, apply to the bands): the same oracle
    calls on a 1/rows_div sample of the grid rows with all N orbitals and bands
    (seeded Gaussian stand-ins, W = -Phi so that -M is positive definite),
    scaled by rows_div; the N x N Cholesky is timed once, unscaled.
    Returns (seconds actually spent, estimated seconds of a whole step, detail)."""
    import oracle
    small = synth.System(n=s.n, L=s.L, n_occ=16, n_bands=1, kernel=s.kernel, omega=s.omega)
    phi = synth.orbitals(small, seed)
    kern = oracle.coulomb_kernel((s.n,) * 3, (s.L,) * 3, s.kernel, s.omega)
    spent = 0.0
    t0 = time.perf_counter()
    oracle.exchange_apply(phi[:2], phi[:1], kern)
    per = (time.perf_counter() - t0) / 2
    spent += per * 2
    targets = int(max(1, min(16, pair_budget_s / max(per, 1e-6) / 16)))
    n_pairs = 16 * targets
    if pair_budget_s / max(per, 1e-6) < 16:            # fewer than one full target fits
        n_pairs = int(max(min_pairs, min(16, pair_budget_s / max(per, 1e-6))))
        t0 = time.perf_counter()
        oracle.exchange_apply(phi[:n_pairs], phi[:1], kern)
    else:
        t0 = time.perf_counter()
        oracle.exchange_apply(phi, phi[:targets], kern)
    t_pairs = time.perf_counter() - t0
    spent += t_pairs
    per_pair = t_pairs / n_pairs
    t_w = per_pair * s.n_occ * s.n_occ
    # dense part on a row sample
    if rows_div is None:
        rows_div = max(1, s.ng // 16384)
    rows = max(s.n_occ, s.ng // rows_div)
    rows_div = s.ng / rows
    rng = np.random.Generator(np.random.PCG64(seed + 7))
    a = rng.standard_normal((s.n_occ, rows)) + 1j * rng.standard_normal((s.n_occ, rows))
    b = rng.standard_normal((s.n_bands, rows)) + 1j * rng.standard_normal((s.n_bands, rows))
    t0 = time.perf_counter()
    M = oracle.overlap_M(a, -a, s.dv)
    t_m = time.perf_counter() - t0
    t0 = time.perf_counter()
    Lc = oracle.cholesky_neg(M)
    t_chol = time.perf_counter() - t0
    t0 = time.perf_counter()
    xi = oracle.xi_from(-a, Lc)
    t_xi = time.perf_counter() - t0
    t0 = time.perf_counter()
    oracle.ace_apply(xi, b, s.dv)
    t_apply = time.perf_counter() - t0
    spent += t_m + t_chol + t_xi + t_apply
    full = t_w + (t_m + t_xi + t_apply) * rows_div + t_chol
    detail = {"ordered_pair_solves_timed": n_pairs, "s_per_ordered_pair_solve": per_pair,
              "t_w_est_s": t_w, "grid_rows_timed": rows, "rows_scale": rows_div,
              "t_dense_est_s": (t_m + t_xi) * rows_div + t_chol, "t_apply_est_s": t_apply * rows_div,
              "t_step_est_s": full, "t_spent_s": spent}
    return spent, full, detail


def input_seed(rank, workload=LARGE):
    """Seed of rank `rank`'s replica: every rank solves its own system."""
    cfg = SINGLE[workload][0] if workload in SINGLE else 3
    return synth.seed_for(cfg, rank)


def max_over_ranks(ms, dist, device):
    """The slowest rank's time (ms); the time itself without a process group."""
    if dist is None:
        return ms
    import torch
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_step, steps, world, ms):
    """Units processed by all ranks per second of the slowest rank's time."""
    return units_per_step * steps * world / (ms / 1e3)


def run_reference(args):
    """The FP64 oracle on this host's cores, each step a bounded sample of the
    chosen workload (pair solves and a row sample of the dense part), with the
    whole step's time extrapolated from it."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    workload = getattr(args, "workload", LARGE)
    if workload not in SINGLE:
        workload = LARGE
    cfg, s = SINGLE[workload]
    seed = input_seed(0, workload)
    budget = 1.0 if s.n >= 96 else 0.5
    for _ in range(args.warmup):
        oracle_sample(s, seed, pair_budget_s=budget)
    spent, full, last = 0.0, 0.0, None
    for _ in range(args.steps):
        sp, fu, last = oracle_sample(s, seed, pair_budget_s=budget)
        spent += sp
        full += fu
    pairs = unique_pairs(s.n_occ)
    value = pairs * args.steps / full
    cores = os.cpu_count()
    sample = (f"per step: {last['ordered_pair_solves_timed']} ordered FFT-Poisson solves on the "
              f"{s.n}^3 grid (of the {s.n_occ ** 2} of a W build) and the dense part on "
              f"{last['grid_rows_timed']} of {s.ng} grid rows, extrapolated to a whole step "
              f"(build + apply of {s.n_bands} bands)")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * spent / max(args.steps, 1),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": workload_config(workload, s),
            "extrapolation": {"full_step_ms_est": 1e3 * full / max(args.steps, 1),
                              "factor": full / max(spent, 1e-12), "extrapolated": True},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": sample, "extrapolated": True},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ----------------------------------------------------------------------------- cuFFT comparison
def cufft_baseline(phi_d, s, w_ours, reps=2):
    """The same W build (unique pairs, both accumulations) written with cuFFT
    (torch.fft) and torch elementwise kernels: a library comparison, timed
    only. Row l of the pair triangle is one batch: rho = conj(phi_l) phi_r for
    r >= l, v = IFFT(K FFT(rho)), W_r -= phi_l v, W_l -= sum_{r>l} phi_r conj(v)."""
    import torch
    n = s.n
    m = np.fft.fftfreq(n, d=1.0 / n)
    g = 2.0 * math.pi * m / s.L
    g2 = g[:, None, None] ** 2 + g[None, :, None] ** 2 + g[None, None, :] ** 2
    with np.errstate(divide="ignore", invalid="ignore"):
        k = 4.0 * math.pi / g2
        if s.kernel == "erfc":
            k = k * (1.0 - np.exp(-g2 / (4.0 * s.omega ** 2)))
    k[0, 0, 0] = math.pi / s.omega ** 2 if s.kernel == "erfc" else 0.0
    kt = torch.from_numpy(k).to(torch.float32).cuda()
    N = s.n_occ
    w = torch.zeros_like(phi_d)

    def build():
        w.zero_()
        for l in range(N):
            rho = torch.conj(phi_d[l])[None] * phi_d[l:]
            v = torch.fft.ifftn(torch.fft.fftn(rho, dim=(1, 2, 3)) * kt, dim=(1, 2, 3))
            w[l:] -= phi_d[l][None] * v
            if l + 1 < N:
                w[l] -= torch.sum(phi_d[l + 1:] * torch.conj(v[1:]), dim=0)

    build()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        build()
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / reps
    diff = float(torch.linalg.vector_norm(w - w_ours) / torch.linalg.vector_norm(w_ours))
    return {"value": unique_pairs(N) / (ms / 1e3), "unit": UNIT, "ms_per_w_build": ms,
            "what": "unique-pair W build with torch.fft (cuFFT) + torch elementwise, one triangle row per batch",
            "rel_diff_W_vs_ours": diff}


# ----------------------------------------------------------------------------- GPU arm
def init_dist():
    import torch
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    from paper_1601_07159_gb300 import build_lib
    if rank == 0 or world == 1:
        build_lib.build()
    if dist:
        dist.barrier()
    return rank, world, local, dist


def make_plan(ace, s, args):
    return ace.Plan(s.n, s.L, s.n_occ, dtype="c64", kernel=s.kernel, omega=s.omega,
                    max_pairs=args.max_pairs, tile=args.tile, lanes=args.lanes,
                    graphs=not args.eager, engine=args.engine and not args.eager,
                    pdl=not args.no_pdl, overlap=not args.no_overlap, radix=args.radix)


def device_inputs(s, seed):
    """Phi and Psi (complex64) on the current device: host-generated for the
    smaller grids, generated on the device for the 96^3 workload."""
    import torch
    if s.n >= 96:
        return synth.orbitals_device(s, seed), synth.targets_device(s, seed)
    phi = torch.from_numpy(synth.orbitals(s, seed)).to(torch.complex64).cuda()
    psi = torch.from_numpy(synth.targets(s, seed)).to(torch.complex64).cuda()
    return phi, psi


def time_steps(plan, phi_d, psi_d, xi_d, y_d, K, warmup, dist, local, clocks=True):
    """W untimed warm-up steps, then exactly K steps (ace_build + ace_apply)
    between CUDA events on the launching stream, bracketed by a barrier and a
    synchronize; the pair section's duration comes from the plan's profile
    events around it."""
    import torch
    stream = torch.cuda.current_stream()
    for _ in range(max(warmup, 3)):
        plan.build(phi_d, want_w=False, want_m=False, xi=xi_d)
        plan.apply(xi_d, psi_d, out=y_d)
    code, piv = plan.status()
    if code != 0:
        raise RuntimeError(f"ace_build status {code} (pivot {piv})")
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True),
           torch.cuda.Event(enable_timing=True)) for _ in range(K)]
    plan.profile_begin(max_events=5 * (K + 1) * 64)
    sampler = ClockSampler(physical_gpu_index(local)) if clocks else None
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    if sampler:
        sampler.start()
    t_start = torch.cuda.Event(enable_timing=True)
    t_end = torch.cuda.Event(enable_timing=True)
    t_start.record(stream)
    for k in range(K):
        ev[k][0].record(stream)
        plan.build(phi_d, want_w=False, want_m=False, xi=xi_d)
        ev[k][1].record(stream)
        plan.apply(xi_d, psi_d, out=y_d)
        ev[k][2].record(stream)
    t_end.record(stream)
    torch.cuda.synchronize()
    clk = sampler.stop() if sampler else None
    prof = plan.profile_end()
    code, piv = plan.status()
    if code != 0:
        raise RuntimeError(f"ace_build status {code} (pivot {piv}) in the timed steps")
    return {"elapsed_ms": t_start.elapsed_time(t_end),
            "build_ms": statistics.mean(e[0].elapsed_time(e[1]) for e in ev),
            "apply_ms": statistics.mean(e[1].elapsed_time(e[2]) for e in ev),
            "prof": prof, "clocks": clk}


def time_e2e(plan, phi_d, psi_d, xi_d, y_d, Ke, dist):
    """End to end through the public API: every step copies its inputs (Phi,
    Psi) from pinned host memory and its results (Y, E_x) back. Streamed the
    way a caller feeding a sequence of systems would: two device buffers per
    input, the inputs of step i+1 uploaded and the results of step i
    downloaded on copy streams while step i+1 computes. Returns (ms, bytes
    up, bytes down) per Ke steps."""
    import torch
    stream = torch.cuda.current_stream()
    phi_h = phi_d.cpu().pin_memory()
    psi_h = psi_d.cpu().pin_memory()
    y_h = torch.empty(y_d.shape, dtype=y_d.dtype).pin_memory()      # downloads are serialised on d2h_s
    ex_h = torch.empty((), dtype=torch.float64).pin_memory()
    h2d_s, d2h_s = torch.cuda.Stream(), torch.cuda.Stream()
    phi_b = [phi_d, torch.empty_like(phi_d)]
    psi_b = [psi_d, torch.empty_like(psi_d)]
    y_b = [y_d, torch.empty_like(y_d)]
    ev_in = [torch.cuda.Event(), torch.cuda.Event()]
    ev_done = [torch.cuda.Event(), torch.cuda.Event()]
    ev_out = [torch.cuda.Event(), torch.cuda.Event()]
    for b in range(2):     # graphs for both buffer sets, outside the timed region
        plan.build(phi_b[b], want_w=False, want_m=False, xi=xi_d)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    h2d_s.wait_event(e0)
    with torch.cuda.stream(h2d_s):
        phi_b[0].copy_(phi_h, non_blocking=True)
        psi_b[0].copy_(psi_h, non_blocking=True)
    ev_in[0].record(h2d_s)
    for i in range(Ke):
        b = i & 1
        stream.wait_event(ev_in[b])
        out = plan.build(phi_b[b], want_w=False, want_m=False, xi=xi_d)
        if i >= 2:
            stream.wait_event(ev_out[b])              # y_b[b] downloaded two steps ago
        plan.apply(xi_d, psi_b[b], out=y_b[b])
        ev_done[b].record(stream)
        d2h_s.wait_event(ev_done[b])
        out["Ex"].record_stream(d2h_s)                # read on the download stream
        with torch.cuda.stream(d2h_s):
            y_h.copy_(y_b[b], non_blocking=True)
            ex_h.copy_(out["Ex"], non_blocking=True)
        ev_out[b].record(d2h_s)
        if i + 1 < Ke:                                # inputs of the next step
            h2d_s.wait_event(ev_done[1 - b] if i >= 1 else e0)
            with torch.cuda.stream(h2d_s):
                phi_b[1 - b].copy_(phi_h, non_blocking=True)
                psi_b[1 - b].copy_(psi_h, non_blocking=True)
            ev_in[1 - b].record(h2d_s)
    stream.wait_event(ev_out[(Ke - 1) & 1])
    stream.wait_event(ev_out[Ke & 1])
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    h2d = phi_h.numel() * phi_h.element_size() + psi_h.numel() * psi_h.element_size()
    d2h = y_h.numel() * y_h.element_size() + 8
    del phi_b[1], psi_b[1], y_b[1]
    return ms, h2d, d2h


def roofline(s, pair_ms, traffic):
    hbm, peak_kind = peaks()
    alg = pair_model_bytes(s)
    achieved = alg / (pair_ms / 1e3) / 1e9
    out = {"kernel": "pair FFT-Poisson pipeline (passes A-D, per ace_build)", "bound": "hbm",
           "achieved": achieved, "peak": hbm, "unit": "GB/s", "frac": achieved / hbm,
           "peak_kind": peak_kind, "alg_bytes_per_launch": alg,
           "alg_model": "32 B/point/unique pair + Phi read + W write", "ms_per_launch": pair_ms,
           "traffic": traffic[0] if traffic else None}
    if traffic:
        out["traffic_source"] = traffic[1]
    return out


def run_single(args):
    import torch
    rank, world, local, dist = init_dist()
    from paper_1601_07159_gb300 import ace

    name = args.workload
    cfg, s = SINGLE[name]
    phi_d, psi_d = device_inputs(s, input_seed(rank, name))
    plan = make_plan(ace, s, args)
    xi_d = plan.empty(s.n_occ)
    y_d = plan.empty(s.n_bands)
    K = args.steps
    t = time_steps(plan, phi_d, psi_d, xi_d, y_d, K, args.warmup, dist, local)
    elapsed_ms = max_over_ranks(t["elapsed_ms"], dist, "cuda")
    pairs = unique_pairs(s.n_occ)
    value = whole_job_rate(pairs, K, world, elapsed_ms)
    pair_ms = t["prof"]["pair_ms"] / K
    traffic = TRAFFIC.get(name) if default_schedule(args) else None
    roof = roofline(s, pair_ms, traffic)

    Ke = max(3, K // 4)
    e2e_ms, h2d, d2h = time_e2e(plan, phi_d, psi_d, xi_d, y_d, Ke, dist)
    e2e_ms = max_over_ranks(e2e_ms, dist, "cuda")
    e2e_value = whole_job_rate(pairs, Ke, world, e2e_ms)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        spent, full, det = oracle_sample(s, input_seed(0, name), pair_budget_s=12.0)
        cpu = {"value": pairs / full, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
               "extrapolated": True, "scale_factor": full / spent,
               "sample": f"{det['ordered_pair_solves_timed']} ordered FFT-Poisson solves of the {s.n}^3 grid "
                         f"(of the {s.n_occ ** 2} of a W build) and the dense part (M, Cholesky, Xi, apply) on "
                         f"{det['grid_rows_timed']} of {s.ng} grid rows, scaled to a whole step",
               "detail": det}

    line = None
    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": K,
                "warmup": args.warmup, "ms_per_step": elapsed_ms / K, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": workload_config(name, s),
                "ms_per_build": t["build_ms"], "ms_per_apply": t["apply_ms"],
                "roofline": roof, "cpu_baseline": cpu,
                "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d,
                        "d2h_bytes_per_step": d2h, "steps": Ke},
                "gpu_launches": t["prof"]["launches"], "clocks": t["clocks"]}
    if rank == 0 and world == 1 and not args.no_extras:
        del xi_d, y_d, plan
        torch.cuda.empty_cache()
        line["xi_variants"] = xi_variants(ace, s, phi_d, reps=1, warm=s.n < 96)
        line["gemm_variants"] = gemm_variants(ace, s, phi_d, psi_d, reps=1, warm=s.n < 96)
    del phi_d, psi_d
    torch.cuda.empty_cache()
    if rank == 0 and world == 1 and not args.no_extras:
        if name != SI64:
            line[SI64] = si64_extra(ace, args)
            torch.cuda.empty_cache()
        line[BATCHED] = batched_extra(ace, args)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist:
        dist.barrier()
        dist.destroy_process_group()
    return 0


def xi_variants(ace, s, phi_d, reps, warm=True):
    """Xi = W L^{-*} (Eq. Wtilde) three ways on the same W and L^{-*}: the
    default FP64-accurate FP16-tensor-core slice product, the TF32 3-term-split
    product and plain FP64 on CUDA cores; ms per whole ace_build with each, and
    each Xi's relative difference to the plain-FP64 one. Without `warm` the
    timed build also captures its graphs (a few ms, for seconds-long builds)."""
    import torch
    stream = torch.cuda.current_stream()
    out, xis = {}, {}
    for key, prec in (("fp64_slices", "xi_fp64"), ("tf32_split", "split_tf32"), ("fp64_cuda_cores", "xi_fp64_simt")):
        plan = ace.Plan(s.n, s.L, s.n_occ, dtype="c64", kernel=s.kernel, omega=s.omega, prec=prec)
        xi = plan.empty(s.n_occ)
        if warm:
            plan.build(phi_d, want_w=False, want_m=False, xi=xi)
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(reps):
            plan.build(phi_d, want_w=False, want_m=False, xi=xi)
        b.record(stream)
        torch.cuda.synchronize()
        out[key] = {"prec": prec, "ms_per_build": a.elapsed_time(b) / reps, "status": plan.status()[0]}
        xis[key] = xi
        del plan
    ref = xis["fp64_cuda_cores"]
    for key in out:
        out[key]["xi_rel_diff_vs_fp64"] = float(torch.linalg.vector_norm(xis[key] - ref) / torch.linalg.vector_norm(ref))
    del xis, ref
    torch.cuda.empty_cache()
    return out


def gemm_variants(ace, s, phi_d, psi_d, reps, warm=True):
    """The dense products (M = dV Phi^* W, the apply) with the TF32 split (the
    default) and the BF16 split (ACE_PREC_SPLIT_BF16): ms per ace_build and per
    ace_apply with each, and the BF16 results' relative difference to the TF32
    ones (M, V_ACE psi)."""
    import torch
    stream = torch.cuda.current_stream()
    out, res = {}, {}
    for key, prec in (("tf32_split", "default"), ("bf16_split", "split_bf16")):
        plan = ace.Plan(s.n, s.L, s.n_occ, dtype="c64", kernel=s.kernel, omega=s.omega, prec=prec)
        xi = plan.empty(s.n_occ)
        y = plan.empty(s.n_bands)
        if warm:
            plan.build(phi_d, want_w=False, want_m=False, xi=xi)
            plan.apply(xi, psi_d, out=y)
        torch.cuda.synchronize()
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
        tb = ta = 0.0
        for _ in range(reps):
            ev[0].record(stream)
            o = plan.build(phi_d, want_w=False, want_m=True, xi=xi)
            ev[1].record(stream)
            plan.apply(xi, psi_d, out=y)
            ev[2].record(stream)
            torch.cuda.synchronize()
            tb += ev[0].elapsed_time(ev[1])
            ta += ev[1].elapsed_time(ev[2])
        out[key] = {"prec": prec, "ms_per_build": tb / reps, "ms_per_apply": ta / reps, "status": plan.status()[0]}
        res[key] = (o["M"], y)
        del plan, xi
    for i, name in enumerate(("m", "apply")):
        a, b = res["bf16_split"][i], res["tf32_split"][i]
        out["bf16_split"][f"{name}_rel_diff_vs_tf32"] = float(torch.linalg.vector_norm(a - b) /
                                                              torch.linalg.vector_norm(b))
    del res
    torch.cuda.empty_cache()
    return out


def si64_extra(ace, args, K=20):
    """The 48^3 workload: K timed steps, its pair-pipeline roofline, and the
    plain-FP64, cuFFT, entry-point and oversampled comparisons."""
    import torch
    cfg, s = SINGLE[SI64]
    phi_d, psi_d = device_inputs(s, input_seed(0, SI64))
    plan = make_plan(ace, s, args)
    xi_d = plan.empty(s.n_occ)
    y_d = plan.empty(s.n_bands)
    t = time_steps(plan, phi_d, psi_d, xi_d, y_d, K, 3, None, 0, clocks=False)
    pairs = unique_pairs(s.n_occ)
    traffic = TRAFFIC.get(SI64) if default_schedule(args) else None
    out = {"value": pairs * K / (t["elapsed_ms"] / 1e3), "unit": UNIT, "steps": K,
           "ms_per_step": t["elapsed_ms"] / K, "ms_per_build": t["build_ms"], "ms_per_apply": t["apply_ms"],
           "roofline": roofline(s, t["prof"]["pair_ms"] / K, traffic)}
    stream = torch.cuda.current_stream()

    def timed(f, reps=5):
        f()
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(reps):
            f()
        b.record(stream)
        torch.cuda.synchronize()
        return a.elapsed_time(b) / reps

    out["xi_variants"] = xi_variants(ace, s, phi_d, reps=3)
    out["gemm_variants"] = gemm_variants(ace, s, phi_d, psi_d, reps=3)
    if not args.no_fp64:
        # plain-FP64 form of the same build: the denominator of the mixed-vs-FP64 ratio
        plan64 = ace.Plan(s.n, s.L, s.n_occ, dtype="c128", kernel=s.kernel, omega=s.omega)
        phi64 = phi_d.to(torch.complex128)
        xi64 = plan64.empty(s.n_occ)
        fp64_ms = timed(lambda: plan64.build(phi64, want_w=False, want_m=False, xi=xi64), reps=2)
        out["fp64_ms_per_build"] = fp64_ms
        out["mixed_vs_fp64_build_speedup"] = fp64_ms / t["build_ms"]
        del plan64, phi64, xi64
    if not args.no_oversampled:
        # ACE with oversampling r = 1.5 (Sec. 3): the 128 orbitals plus 64 bands
        phi_all = torch.cat([phi_d, psi_d[:64]]).contiguous()
        ms = timed(lambda: plan.build_oversampled(phi_all, want_w=False, want_m=False), reps=3)
        code, piv = plan.status()
        out["oversampled"] = {"n_occ": s.n_occ, "n_phi": int(phi_all.shape[0]), "ms_per_build": ms,
                              "unique_pairs": pairs + s.n_occ * 64, "status": code}
        del phi_all
    if not args.no_entries:
        # the direct energy (Eq. EX: passes A and B of every unique pair with the
        # Parseval sum, no potentials) and the Poisson entry (bare kernel, as for
        # the Hartree potential) on the 192 bands
        e_ms = timed(lambda: plan.energy_grad(phi_d))
        pplan = ace.Plan(s.n, s.L, 1, dtype="c64", kernel="bare")
        v_d = pplan.empty(s.n_bands)
        p_ms = timed(lambda: pplan.poisson(psi_d, out=v_d))
        out["entries"] = {"energy_direct": {"ms": e_ms, "unique_pairs": pairs, "pair_solves_per_s": pairs / (e_ms / 1e3)},
                          "poisson": {"ms": p_ms, "vectors": s.n_bands, "solves_per_s": s.n_bands / (p_ms / 1e3),
                                      "kernel": "bare"}}
        del pplan, v_d
    if not args.no_cufft:
        w_ours = plan.build(phi_d)["W"]
        out["cufft_baseline"] = cufft_baseline(phi_d, s, w_ours)
        del w_ours
    del plan, phi_d, psi_d, xi_d, y_d
    return out


def batched_systems_inputs(ace, args, engine=None):
    import torch
    systems = synth.batched_systems()[:args.systems]
    engine = args.engine if engine is None else engine
    plans, phis_h, phis = [], [], []
    for i, s in enumerate(systems):
        plans.append(ace.Plan(s.n, s.L, s.n_occ, dtype="c64", kernel="bare", max_pairs=args.max_pairs,
                              tile=args.tile, overlap=not args.no_overlap, engine=engine))
        d = synth.orbitals_device(s, synth.seed_for(3, i))
        phis.append(d)
        phis_h.append(d.cpu().pin_memory())
    return systems, plans, phis_h, phis


def batched_model_bytes(systems):
    return sum(pair_model_bytes(s) for s in systems)


def time_batch(ace, args, K, engine):
    """ms per ace_build_batched step of the uneven systems (plans with or
    without the persistent pair engine)."""
    import torch
    systems, plans, _, phis = batched_systems_inputs(ace, args, engine=engine)
    batch = ace.Batch(plans, chains=args.chains)
    xis = [p.empty(p.n_occ) for p in plans]
    for _ in range(3):
        batch.build(phis, xis)
    for i, p in enumerate(plans):
        code, piv = p.status()
        if code != 0:
            raise RuntimeError(f"batched system {i}: status {code} (pivot {piv})")
    stream = torch.cuda.current_stream()
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for _ in range(K):
        batch.build(phis, xis)
    b.record(stream)
    torch.cuda.synchronize()
    del batch, plans, phis, xis
    return systems, a.elapsed_time(b) / K


def batched_extra(ace, args, K=3):
    """One batched step of the 64 uneven systems: ms per batch and its
    roofline against the summed pair model; the same batch with every system's
    pair solves as one persistent engine launch, for comparison."""
    systems, ms = time_batch(ace, args, K, engine=args.engine)
    _, ms_engine = time_batch(ace, args, K, engine=not args.engine)
    pairs = sum(unique_pairs(s.n_occ) for s in systems)
    hbm, peak_kind = peaks()
    alg = batched_model_bytes(systems)
    achieved = alg / (ms / 1e3) / 1e9
    out = {"value": pairs / (ms / 1e3), "unit": UNIT, "steps": K, "ms_per_build_batch": ms,
           "systems": len(systems), "unique_pairs": pairs,
           "roofline": {"kernel": "whole batched build (pairs, GEMMs, Cholesky) vs the pair model",
                        "bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s",
                        "frac": achieved / hbm, "peak_kind": peak_kind, "alg_bytes_per_launch": alg,
                        "traffic": None},
           ("four_kernel_ms_per_build_batch" if args.engine else "engine_ms_per_build_batch"): ms_engine}
    return out


# ----------------------------------------------------------------------------- batched workload
def run_batched(args):
    """The uneven batch: 64 systems, edges in {32,36,40,48,64}, N in [16,128],
    bare kernel, c64, one ace_build_batched graph per step. Every rank runs its
    own replica of the whole batch."""
    import torch
    rank, world, local, dist = init_dist()
    from paper_1601_07159_gb300 import ace

    systems, plans, phis_h, phis = batched_systems_inputs(ace, args)
    batch = ace.Batch(plans, chains=args.chains)
    xis = [p.empty(p.n_occ) for p in plans]
    for _ in range(max(args.warmup, 3)):
        batch.build(phis, xis)
    for i, p in enumerate(plans):
        code, piv = p.status()
        if code != 0:
            raise RuntimeError(f"system {i}: status {code} (pivot {piv})")
    torch.cuda.synchronize()
    K = args.steps
    stream = torch.cuda.current_stream()
    for p in plans:
        p.profile_begin(max_events=16)
    clocks = ClockSampler(physical_gpu_index(local))
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    for _ in range(K):
        batch.build(phis, xis)
    t1.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    launches = sum(p.profile_end()["launches"] for p in plans)
    elapsed_ms = t0.elapsed_time(t1)
    elapsed_ms = max_over_ranks(elapsed_ms, dist, "cuda")
    pairs = sum(unique_pairs(s.n_occ) for s in systems)
    value = whole_job_rate(pairs, K, world, elapsed_ms)
    # end to end: every step uploads all Phi from pinned host memory and reads
    # all E_x back. Two device buffer sets (one captured batch graph each): the
    # inputs of step i+1 are uploaded on a copy stream while step i computes.
    Ke = max(3, K // 5)
    ex_h = torch.empty(len(systems), dtype=torch.float64).pin_memory()
    h2d_s = torch.cuda.Stream()
    phis_b = [phis, [torch.empty_like(d) for d in phis]]
    ev_in = [torch.cuda.Event(), torch.cuda.Event()]
    ev_done = [torch.cuda.Event(), torch.cuda.Event()]
    batch.build(phis_b[1], xis)                       # second graph, outside the timed region
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)

    def upload(b, after):
        h2d_s.wait_event(after)
        with torch.cuda.stream(h2d_s):
            for h, d in zip(phis_h, phis_b[b]):
                d.copy_(h, non_blocking=True)
        ev_in[b].record(h2d_s)

    upload(0, e0)
    for i in range(Ke):
        b = i & 1
        stream.wait_event(ev_in[b])
        _, ex = batch.build(phis_b[b], xis)
        ev_done[b].record(stream)
        ex_h.copy_(ex, non_blocking=True)
        if i + 1 < Ke:                                # buffer 1-b was last read by step i-1
            upload(1 - b, ev_done[1 - b] if i >= 1 else e0)
    e1.record(stream)
    torch.cuda.synchronize()
    e2e_ms = max_over_ranks(e0.elapsed_time(e1), dist, "cuda")
    hbm, peak_kind = peaks()
    alg_bytes = batched_model_bytes(systems)
    achieved = alg_bytes / (elapsed_ms / K / 1e3) / 1e9
    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": K,
                "warmup": args.warmup, "ms_per_step": elapsed_ms / K, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": {"workload": BATCHED, "systems": len(systems),
                           "edges": sorted({s.n for s in systems}),
                           "n_occ_range": [min(s.n_occ for s in systems), max(s.n_occ for s in systems)],
                           "unique_pairs": pairs, "kernel": "bare",
                           "precision": "fp32 pair/FFT path, TF32 3-term-split M, fp64 Cholesky and L^-1, "
                                        "Xi = W L^-* to fp64 accuracy (fp16 tensor-core slices)",
                           "pair_solves": "persistent engine per system" if args.engine else
                                          "four kernels per batch, captured graph",
                           "chains": args.chains or 3, "l2": "working set > L2 every step (no flush needed)"},
                "ms_per_build_batch": elapsed_ms / K,
                "roofline": {"kernel": "whole batched build (pairs, GEMMs, Cholesky) vs the pair model",
                             "bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s",
                             "frac": achieved / hbm, "peak_kind": peak_kind,
                             "alg_bytes_per_launch": alg_bytes,
                             "alg_model": "sum over systems of 32 B/point/unique pair + Phi read + W write",
                             "ms_per_launch": elapsed_ms / K, "traffic": None},
                "cpu_baseline": None,
                "e2e": {"value": whole_job_rate(pairs, Ke, world, e2e_ms), "unit": UNIT,
                        "h2d_bytes_per_step": sum(h.numel() * h.element_size() for h in phis_h),
                        "d2h_bytes_per_step": 8 * len(systems), "steps": Ke},
                "gpu_launches": launches, "clocks": clk}
        print(json.dumps(line), flush=True)
    if dist:
        dist.barrier()
        dist.destroy_process_group()
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == BATCHED:
        return run_batched(args)
    return run_single(args)


if __name__ == "__main__":
    sys.exit(main())
