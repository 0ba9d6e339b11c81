#!/usr/bin/env python3
"""Benchmark of the ACE hot path on one GB300 (or N independent replicas).

A step is one pass of the whole path on the Si64-like 48^3 workload (L = 20.5
bohr, N = 128 orbitals, 192 bands, complex, screened kernel omega = 0.106):
ace_build (W over the 8256 unique pair FFT-Poisson solves, M = dV Phi^* W,
FP64 Cholesky and L^{-1}, Xi = W L^{-*}, E_x) followed by ace_apply on the 192
bands. The metric is unique pair FFT-Poisson solves per second of whole steps.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun each rank runs an independent replica (its own system): the
work is partitioned into independent problems, no data-path collective;
value = pairs over all ranks / max-over-ranks time ("scaling": "weak").
--impl reference times the FP64 CPU oracle on this host (rank 0 only).
--workload batched64_uneven times one ace_build_batched of 64 uneven systems
per step instead.

Besides the contract keys, the default line carries: ms per build and per
apply, the pair pipeline's roofline with its per-pass split (eager runs), the
end-to-end rate through pinned host buffers, the plain-FP64 build time, a
cuFFT/torch W build (`cufft_baseline`), the direct-energy and Poisson entry
points (`entries`), and an oversampled build (`oversampled`); the --no-*
flags skip those extras.
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

WORKLOAD = "si64_48cube_n128"
BATCHED = "batched64_uneven"
METRIC = "pair FFT-Poisson solves/s"
UNIT = "pair-solves/s"


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=50)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", choices=["ours", "reference"], default="ours")
    p.add_argument("--no-cpu-baseline", action="store_true")
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
    p.add_argument("--workload", choices=[WORKLOAD, BATCHED], default=WORKLOAD,
                   help=f"{BATCHED}: the 64-system uneven batch in one ace_build_batched graph")
    p.add_argument("--chains", type=int, default=0, help="concurrent stream chains of a batch (0 = default)")
    p.add_argument("--systems", type=int, default=64, help="systems of the batched workload")
    return p.parse_args()


def workload_config(s):
    return {"workload": WORKLOAD, "grid": f"{s.n}^3", "L_bohr": s.L, "n_occ": s.n_occ,
            "n_bands": s.n_bands, "kernel": f"erfc omega={s.omega}" if s.kernel == "erfc" else "bare",
            "orbitals": "seeded Gaussian-decaying plane waves |G|^2/2<=10 Ha, QR-orthonormal",
            "precision": "fp32 pair/FFT path and GEMMs, fp64 Cholesky and L^-1",
            "l2": "working set > L2 every step (no flush needed)"}


def unique_pairs(n):
    return n * (n + 1) // 2


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
def oracle_step(phi, psi, kern, dv, cols):
    """Time the FP64 oracle on a bounded sample of one step: `cols` columns of W
    (each N ordered pair solves, Eq. applyVX2), scaled to all N columns, plus the
    dense part (M, Cholesky, Xi, apply) at full size. The dense part is timed on
    the stand-in W = -Phi (same shapes, -M = I positive definite), since its cost
    does not depend on the values. Returns (estimated seconds per step, detail)."""
    import oracle
    n_occ = phi.shape[0]
    t0 = time.perf_counter()
    oracle.exchange_apply(phi, phi[cols], kern)
    t_cols = time.perf_counter() - t0
    t0 = time.perf_counter()
    w_stand = -phi
    M = oracle.overlap_M(phi, w_stand, dv)
    Lc = oracle.cholesky_neg(M)
    xi = oracle.xi_from(w_stand, Lc)
    t_dense = time.perf_counter() - t0
    t0 = time.perf_counter()
    oracle.ace_apply(xi, psi, dv)
    t_apply = time.perf_counter() - t0
    t_w = t_cols * n_occ / len(cols)
    return t_w + t_dense + t_apply, {"t_cols_s": t_cols, "t_w_est_s": t_w, "t_dense_s": t_dense,
                                     "t_apply_s": t_apply}


def input_seed(rank):
    """Seed of rank `rank`'s replica: every rank solves its own system."""
    return synth.seed_for(2, rank)


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


def make_inputs(s, rank=0):
    seed = input_seed(rank)
    phi = synth.orbitals(s, seed)
    psi = synth.targets(s, seed)
    return phi, psi


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    import oracle
    s = synth.SI64_48
    phi, psi = make_inputs(s)
    kern = oracle.coulomb_kernel((s.n,) * 3, (s.L,) * 3, s.kernel, s.omega)
    cols = [0]
    for _ in range(args.warmup):
        oracle_step(phi, psi, kern, s.dv, cols)
    total_t, total_pairs = 0.0, 0
    for k in range(args.steps):
        t, _ = oracle_step(phi, psi, kern, s.dv, [(37 * k) % s.n_occ])
        total_t += t
        total_pairs += unique_pairs(s.n_occ)
    value = total_pairs / total_t
    cores = os.cpu_count()
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total_t / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": workload_config(s),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": "per step: 1 of 128 W columns (128 ordered FFT-Poisson solves) "
                                       "scaled x128, plus full-size M/Cholesky/Xi/apply"},
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
def run_ours(args):
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
    from paper_1601_07159_gb300 import ace

    s = synth.SI64_48
    phi, psi = make_inputs(s, rank)
    plan = ace.Plan(s.n, s.L, s.n_occ, dtype="c64", kernel=s.kernel, omega=s.omega,
                    max_pairs=args.max_pairs, tile=args.tile, lanes=args.lanes,
                    graphs=not args.eager, engine=args.engine and not args.eager,
                    pdl=not args.no_pdl, overlap=not args.no_overlap)
    td = torch.complex64
    phi_h = torch.from_numpy(phi).to(td).pin_memory()
    psi_h = torch.from_numpy(psi).to(td).pin_memory()
    phi_d = phi_h.cuda()
    psi_d = psi_h.cuda()
    xi_d = plan.empty(s.n_occ)
    y_d = plan.empty(s.n_bands)
    y_h = torch.empty(y_d.shape, dtype=td).pin_memory()
    ex_h = torch.empty((), dtype=torch.float64).pin_memory()

    def step():
        out = plan.build(phi_d, want_w=False, want_m=False, xi=xi_d)
        plan.apply(xi_d, psi_d, out=y_d)
        return out["Ex"]

    for _ in range(max(args.warmup, 3)):
        step()
    code, piv = plan.status()
    if code != 0:
        raise RuntimeError(f"ace_build status {code} (pivot {piv})")
    torch.cuda.synchronize()

    K = args.steps
    stream = torch.cuda.current_stream()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True),
           torch.cuda.Event(enable_timing=True)) for _ in range(K)]
    batches_per_build = None
    plan.profile_begin(max_events=5 * (K + 1) * 64)
    clocks = ClockSampler(physical_gpu_index(local))
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
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
    clk = clocks.stop()
    prof = plan.profile_end()
    elapsed_ms = t_start.elapsed_time(t_end)
    build_ms = statistics.mean(e[0].elapsed_time(e[1]) for e in ev)
    apply_ms = statistics.mean(e[1].elapsed_time(e[2]) for e in ev)
    elapsed_ms = max_over_ranks(elapsed_ms, dist, "cuda")
    pairs = unique_pairs(s.n_occ)
    value = whole_job_rate(pairs, K, world, elapsed_ms)

    # end to end through the public API: every step copies its inputs (Phi, Psi)
    # from pinned host memory and its results (Y, E_x) back. Streamed the way a
    # caller feeding a sequence of systems would: two device buffers per array,
    # inputs of step i+1 uploaded and results of step i downloaded on copy
    # streams while step i+1 computes.
    Ke = max(4, K // 4)
    h2d_s, d2h_s = torch.cuda.Stream(), torch.cuda.Stream()
    phi_b = [phi_d, torch.empty_like(phi_d)]
    psi_b = [psi_d, torch.empty_like(psi_d)]
    y_b = [y_d, torch.empty_like(y_d)]
    y_hb = [y_h, torch.empty(y_d.shape, dtype=td).pin_memory()]
    ex_hb = [ex_h, torch.empty((), dtype=torch.float64).pin_memory()]
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
            y_hb[b].copy_(y_b[b], non_blocking=True)
            ex_hb[b].copy_(out["Ex"], non_blocking=True)
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
    e2e_ms = e0.elapsed_time(e1)
    e2e_ms = max_over_ranks(e2e_ms, dist, "cuda")
    e2e_value = whole_job_rate(pairs, Ke, world, e2e_ms)
    h2d = phi_h.numel() * phi_h.element_size() + psi_h.numel() * psi_h.element_size()
    d2h = y_h.numel() * y_h.element_size() + 8

    # roofline of the pair FFT-Poisson pipeline (passes A-D), per build
    hbm, peak_kind = peaks()
    ng = s.ng
    alg_bytes = 32.0 * ng * pairs + 2.0 * s.n_occ * ng * 8
    # DRAM bytes (read + write) of passes A-D per build from the warm ncu capture
    # summarised in profiles/pair_passes_si64_48cube_n128.md: 209.7 MB per 64-pair
    # batch x (120 + 8 x 72/64) batch equivalents; valid for the default plan.
    traffic = 27.05e9 if (args.max_pairs, args.tile, args.eager, args.engine) == (0, 0, False, False) else None
    pair_ms = prof["pair_ms"] / K
    achieved = alg_bytes / (pair_ms / 1e3) / 1e9
    pass_alg = {"A": 8.0 * ng * pairs, "B": 16.0 * ng * pairs, "C": 16.0 * ng * pairs,
                "D": 8.0 * ng * pairs + 2.0 * s.n_occ * ng * 8 * 2}
    passes = {}
    for k, ms in prof["pass_ms"].items():
        if not math.isfinite(ms):     # graph replay: per-pass shares come from the ncu launch list
            passes = None
            break
        per = ms / K
        passes[k] = {"ms_per_build": per, "share": ms / max(prof["pair_ms"], 1e-12),
                     "alg_GBps": pass_alg[k] / (per / 1e3) / 1e9 if per > 0 else None}

    # plain-FP64 form of the same build (denominator of the mixed-vs-FP64 ratio)
    fp64 = None
    if not args.no_fp64:
        plan64 = ace.Plan(s.n, s.L, s.n_occ, dtype="c128", kernel=s.kernel, omega=s.omega)
        phi64 = torch.from_numpy(phi).cuda()
        xi64 = plan64.empty(s.n_occ)
        plan64.build(phi64, want_w=False, want_m=False, xi=xi64)
        torch.cuda.synchronize()
        f0 = torch.cuda.Event(enable_timing=True)
        f1 = torch.cuda.Event(enable_timing=True)
        f0.record(stream)
        for _ in range(2):
            plan64.build(phi64, want_w=False, want_m=False, xi=xi64)
        f1.record(stream)
        torch.cuda.synchronize()
        fp64_ms = f0.elapsed_time(f1) / 2
        fp64 = {"fp64_ms_per_build": fp64_ms, "mixed_vs_fp64_build_speedup": fp64_ms / build_ms}
        del plan64, phi64, xi64

    # ACE with oversampling r = 1.5 (Sec. 3): the 128 orbitals plus 64 bands
    over = None
    if not args.no_oversampled:
        phi_all = torch.cat([phi_d, psi_d[:64]]).contiguous()
        plan.build_oversampled(phi_all, want_w=False, want_m=False)
        torch.cuda.synchronize()
        o0 = torch.cuda.Event(enable_timing=True)
        o1 = torch.cuda.Event(enable_timing=True)
        o0.record(stream)
        for _ in range(3):
            plan.build_oversampled(phi_all, want_w=False, want_m=False)
        o1.record(stream)
        torch.cuda.synchronize()
        code, piv = plan.status()
        over = {"n_occ": s.n_occ, "n_phi": int(phi_all.shape[0]), "ms_per_build": o0.elapsed_time(o1) / 3,
                "unique_pairs": unique_pairs(s.n_occ) + s.n_occ * 64, "status": code}
        del phi_all

    # the direct energy (Eq. EX: passes A and B of every unique pair with the
    # Parseval sum, no potentials) and the Poisson entry (V = sum_G K rho_hat
    # e^{iG.r}, bare kernel, as for the Hartree potential) on the 192 bands
    entries = None
    if not args.no_entries:
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
        e_ms = timed(lambda: plan.energy_grad(phi_d))
        pplan = ace.Plan(s.n, s.L, 1, dtype="c64", kernel="bare")
        v_d = pplan.empty(s.n_bands)
        p_ms = timed(lambda: pplan.poisson(psi_d, out=v_d))
        entries = {"energy_direct": {"ms": e_ms, "unique_pairs": pairs, "pair_solves_per_s": pairs / (e_ms / 1e3)},
                   "poisson": {"ms": p_ms, "vectors": s.n_bands, "solves_per_s": s.n_bands / (p_ms / 1e3),
                               "kernel": "bare"}}
        del pplan, v_d

    cufft = None
    if not args.no_cufft:
        w_ours = plan.build(phi_d)["W"]
        cufft = cufft_baseline(phi_d, s, w_ours)
        del w_ours

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        import oracle
        kern = oracle.coulomb_kernel((s.n,) * 3, (s.L,) * 3, s.kernel, s.omega)
        t1, _ = oracle_step(phi, psi, kern, s.dv, [0])
        ncols = int(max(1, min(s.n_occ, 15.0 / max(t1, 1e-3))))
        cols = list(range(0, s.n_occ, max(1, s.n_occ // ncols)))[:ncols]
        t, det = oracle_step(phi, psi, kern, s.dv, cols)
        cpu = {"value": pairs / t, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
               "sample": f"{len(cols)} of {s.n_occ} W columns ({len(cols) * s.n_occ} ordered FFT-Poisson "
                         f"solves) scaled to a full build, plus full-size M/Cholesky/Xi/apply",
               "detail": det}

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": K,
                "warmup": args.warmup, "ms_per_step": elapsed_ms / K, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": workload_config(s),
                "ms_per_build": build_ms, "ms_per_apply": apply_ms,
                "roofline": {"kernel": "pair FFT-Poisson pipeline (passes A-D, per ace_build)",
                             "bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s",
                             "frac": achieved / hbm, "peak_kind": peak_kind,
                             "alg_bytes_per_launch": alg_bytes,
                             "alg_model": "32 B/point/unique pair + Phi read + W write",
                             "ms_per_launch": pair_ms, "traffic": traffic, "passes": passes},
                "cpu_baseline": cpu,
                "cufft_baseline": cufft,
                "entries": entries,
                "oversampled": over,
                "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d,
                        "d2h_bytes_per_step": d2h, "steps": Ke},
                "gpu_launches": prof["launches"] + 0,
                "clocks": clk}
        if fp64:
            line.update(fp64)
        print(json.dumps(line), flush=True)
    if dist:
        dist.barrier()
        dist.destroy_process_group()
    return 0


# ----------------------------------------------------------------------------- batched workload
def run_batched(args):
    """The uneven batch: 64 systems, edges in {32,36,40,48,64}, N in [16,128],
    bare kernel, c64, one ace_build_batched graph per step. Every rank runs its
    own replica of the whole batch."""
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
    from paper_1601_07159_gb300 import ace

    systems = synth.batched_systems()[:args.systems]
    plans, phis_h, phis = [], [], []
    for i, s in enumerate(systems):
        phi = synth.orbitals(s, synth.seed_for(3, i))
        plans.append(ace.Plan(s.n, s.L, s.n_occ, dtype="c64", kernel="bare", max_pairs=args.max_pairs,
                              tile=args.tile, overlap=not args.no_overlap))
        h = torch.from_numpy(phi).to(torch.complex64).pin_memory()
        phis_h.append(h)
        phis.append(h.cuda())
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
    alg_bytes = sum(32.0 * s.ng * unique_pairs(s.n_occ) + 2.0 * s.n_occ * s.ng * 8 for s in systems)
    achieved = alg_bytes / (elapsed_ms / K / 1e3) / 1e9
    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": K,
                "warmup": args.warmup, "ms_per_step": elapsed_ms / K, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": {"workload": BATCHED, "systems": len(systems),
                           "edges": sorted({s.n for s in systems}),
                           "n_occ_range": [min(s.n_occ for s in systems), max(s.n_occ for s in systems)],
                           "unique_pairs": pairs, "kernel": "bare",
                           "precision": "fp32 pair/FFT path and GEMMs, fp64 Cholesky and L^-1",
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
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
