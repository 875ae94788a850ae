"""Benchmark: Haydock steps/s of the interpolated-BSE hot path on GB300.

Workload (one process per GPU): the single-system configuration -- coarse
8^3, 4 valence x 4 conduction bands, dense subdivision 4^3 (32768 dense k,
N = 524288 transitions), 3 polarisations, 300 Lanczos steps, Method 3 with
width 1 (near-diagonal divergence treatment), continued fraction on 1000
frequencies.  One bench step = one whole Haydock run (300 Lanczos steps of
all 3 chains: restrict, K_c apply, M3 near field, prolong + diagonal,
Lanczos update) plus the continued fraction.

Headline `value`: mixed path (K_c in BF16 on the tensor cores, FP32 vectors,
FP64 reductions), chain-steps/s summed over ranks.  The FP64 plain path is
timed on the same workload and reported beside it, with the Im eps error of
the mixed path against it.

Under torchrun each rank runs its own independent system (weak scaling): the
path has no exchange step between independent Haydock problems.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

N_OMEGA = 1000
# DRAM bytes (read + write) of one near-field launch on this workload from the
# committed ncu capture, or None when the kernel changed since the capture.
NEAR_TRAFFIC = None


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=3)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", choices=["ours", "reference"], default="ours")
    p.add_argument("--lanczos", type=int, default=300, help="Lanczos steps per Haydock run")
    p.add_argument("--skip-fp64", action="store_true")
    p.add_argument("--skip-cpu", action="store_true")
    p.add_argument("--skip-batched", action="store_true")
    return p.parse_args()


def dist_info():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def rank_seed(rank: int) -> int:
    """Each rank runs its own independent system of the single-system shape (weak scaling)."""
    return 2 + rank


def slowest_rank_time(t_step: float, ws: int, device=None) -> float:
    """Max over ranks of the per-rank step time (the job is as slow as its slowest rank)."""
    if ws == 1:
        return t_step
    import torch
    import torch.distributed as dist
    tt = torch.tensor([t_step], dtype=torch.float64, device=device)
    dist.all_reduce(tt, op=dist.ReduceOp.MAX)
    return float(tt.item())


def job_value(ws: int, chain_steps_per_rank: int, t_max: float) -> float:
    """Whole-job chain-steps/s: the chain-steps of all ranks over the slowest rank's time."""
    return ws * chain_steps_per_rank / t_max


class Clocks:
    """nvidia-smi sampler for the timed region (SM clock and throttle reasons)."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device: int):
        self.device = device
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.device), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        out, _ = self.proc.communicate(timeout=10)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def algorithmic(sysd, nchains, kc_bytes_per_entry, vec_bytes):
    """Algorithmic bytes / flops per launch of each kernel class (one Lanczos step)."""
    nv, nc = sysd["nv"], sysd["nc"]
    t = nv * nc
    Nc, N, Nk, nd = sysd["Nc"], sysd["N"], sysd["Nk"], sysd["n_div"]
    nbar = ((nd + (nd - 1)) / nd) ** 3                      # non-zero-weight corners per dense k
    dbytes = Nk * nbar * (nv * nv + nc * nc) * vec_bytes     # one pass over the d tables
    return {
        "kc_apply": {"bytes": Nc * Nc * kc_bytes_per_entry, "flops": 8.0 * nchains * Nc * Nc},
        "restrict": {"bytes": dbytes + nchains * N * vec_bytes + nchains * Nk * nbar * t * vec_bytes},
        "prolong": {"bytes": dbytes + nchains * (3 * N * vec_bytes + Nk * nbar * t * vec_bytes) + N * vec_bytes / 2},
    }


def near_field_work(nd, width, t, nchains, nkc, nb1=False):
    """Operation counts of the M3 near field per launch (one Lanczos step, all
    chains), from the near-pair geometry (integer enumeration, no arithmetic of
    the method):
      useful   real flops of the factored form -- stage 1: y1 and z over every
               (target, source pair) near pair, 2 t real entries per chain;
               stage 2: for every (target, active target corner, reached slot)
               the t x t head block applied to y1 and to z, complex, 8 flops per
               complex multiply-add;
      issued   real flops of the tensor-core MMAs the kernel issues (stage 1:
               128 x 32 chains x 32 per K-block; stage 2: 256 x 64 chains x 64
               per slot, one 128-row half when 16 t <= 128)."""
    import math
    R2 = math.floor(width * width * nd * nd + 1e-9)
    rad = int(math.floor(math.sqrt(R2) + 1e-12))
    offs = [(a, b, c) for a in range(-rad, rad + 1) for b in range(-rad, rad + 1) for c in range(-rad, rad + 1)
            if a * a + b * b + c * c <= R2]

    def fdiv(a, n):
        return (a - a % n) // n

    def wnum(j, l):
        if nb1:
            return int(all((2 * j[ax] > nd) == bool((l >> (2 - ax)) & 1) for ax in range(3)))
        r = 1
        for ax in range(3):
            r *= j[ax] if (l >> (2 - ax)) & 1 else nd - j[ax]
        return r

    subs = [(a, b, c) for a in range(nd) for b in range(nd) for c in range(nd)]
    rows, pairs, reach = {}, 0, set()
    for tj, j in enumerate(subs):
        for o in offs:
            g = [j[ax] + o[ax] for ax in range(3)]
            co = [fdiv(x, nd) for x in g]
            jp = tuple(g[ax] - co[ax] * nd for ax in range(3))
            for l in range(8):
                if wnum(jp, l) == 0:
                    continue
                slot = tuple(co[ax] + ((l >> (2 - ax)) & 1) for ax in range(3))
                rows.setdefault(slot, set()).add((tuple(co), jp, l))
                reach.add((tj, slot))
                pairs += 1
    act = [sum(1 for l in range(8) if wnum(j, l)) for j in subs]
    s2 = sum(act[tj] for tj, _ in reach)
    useful = nkc * nchains * (pairs * 2 * (2 * t) * 2 + s2 * 2 * t * t * 8)
    nkg = sum((len(v) + 31) // 32 for v in rows.values())
    nmh = 2 if 16 * t > 128 else 1
    issued = nkc * 2 * (nkg * 128 * 32 * nchains * 32 + len(rows) * nmh * 128 * 64 * nchains * 64)
    return {"useful_flops": float(useful), "issued_flops": float(issued), "near_pairs_per_cell": pairs,
            "head_blocks_per_cell": s2, "k_blocks_per_cell": nkg, "slots_per_cell": len(rows)}


def time_runs(ctx, bse, it, dirs, m, flags, steps, warmup, omega, pref, eta, barrier):
    import torch
    st = torch.cuda.current_stream()
    res = None
    for _ in range(warmup):
        res = ctx.bse_haydock_run([it], [dirs.shape[0]], dirs, m, flags)
    barrier()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(st)
    for _ in range(steps):
        res = ctx.bse_haydock_run([it], [dirs.shape[0]], dirs, m, flags)
        a, b, pn2, sd, _ = res
        eps = ctx.bse_spectrum(a, b, pn2, sd, pref, eta, omega)
    e1.record(st)
    torch.cuda.synchronize()
    barrier()
    return e0.elapsed_time(e1), res, eps


def run_ours(args):
    import torch
    import torch.distributed as dist
    from paper_1602_01863_gb300 import bse, synth

    ws, rank, local = dist_info()
    if ws > 1:
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream()

    def barrier():
        if ws > 1:
            dist.barrier()

    sysm = synth.single_system(seed=rank_seed(rank))
    m = args.lanczos
    dirs = sysm.pol_dirs
    p = dirs.shape[0]
    omega = synth.frequency_grid(N_OMEGA)
    ctx = bse.Context(local, stream.cuda_stream)
    info = {"nv": sysm.model.nv, "nc": sysm.model.nc, "Nc": sysm.n_coarse_dim, "N": sysm.n_dense_dim,
            "Nk": sysm.nk_dense, "n_div": sysm.n_div}
    pref = synth.S_EPS / sysm.nk_dense
    eta = synth.ETA

    # ---------------- mixed path: BF16 K_c on tensor cores, FP32 vectors, FP64 reductions
    co = ctx.bse_build_coarse(sysm.model, sysm.n_coarse, bse.PREC_BF16)
    it = ctx.bse_interp_setup(co, sysm.n_div, bse.SCHEME_M3, 1.0, bse.PREC_F32)
    clocks = Clocks(local)
    clocks.start()
    ms, res, eps_mixed = time_runs(ctx, bse, it, dirs, m, bse.USE_GRAPH, args.steps, args.warmup, omega, pref, eta, barrier)
    clk = clocks.stop()
    t_step = ms / 1e3 / args.steps
    t_max = slowest_rank_time(t_step, ws, dev)
    chain_steps = p * m
    value = job_value(ws, chain_steps, t_max)

    # ---------------- per-kernel device times (CUDA events on the launching stream)
    ctx.bse_haydock_run([it], [p], dirs, m, bse.PROFILE)
    kt = ctx.bse_last_kernel_times()
    alg = algorithmic(info, p, 4, 8)
    dom = max(("kc_apply", "restrict", "prolong", "near_field"), key=lambda k: kt[k][0])
    peaks_path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    peaks = json.load(open(peaks_path)) if os.path.exists(peaks_path) else {}
    hbm_peak = float(peaks.get("hbm_gbs", 6800.0))
    peak_src = "measured" if "hbm_gbs" in peaks else "fallback"
    # FP32 CUDA-core peak: 152 SMs x 128 lanes x 2 flop x max SM clock
    # TF32 dense tensor peak: the measured BF16 burst figure x the nominal TF32 / BF16 ratio (1.1 / 2.25)
    tf32_peak = float(peaks.get("bf16_tflops", 1900.0)) * 1.1 / 2.25
    nfw = near_field_work(sysm.n_div, 1.0, info["nv"] * info["nc"], p, sysm.nk_coarse)
    if dom == "near_field":
        achieved = nfw["useful_flops"] / (kt[dom][0] * 1e-3) / 1e12
        roof = {"bound": "tensor", "kernel": "k_near_tc (M3 near field, tcgen05 TF32)", "achieved": achieved,
                "peak": tf32_peak, "unit": "TFLOP/s", "frac": achieved / tf32_peak, "traffic": NEAR_TRAFFIC,
                "peak_source": f"{peak_src} bf16 burst x nominal TF32/BF16 ratio 1.1/2.25",
                "flops": "useful flops of the factored near field (stage 1 y1, z; stage 2 head blocks)",
                "issued_tflops": nfw["issued_flops"] / (kt[dom][0] * 1e-3) / 1e12}
    else:
        achieved = alg[dom]["bytes"] / (kt[dom][0] * 1e-3) / 1e9
        roof = {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": hbm_peak, "unit": "GB/s",
                "frac": achieved / hbm_peak, "traffic": None, "peak_source": peak_src}
    kc = alg["kc_apply"]
    kc_gbs = kc["bytes"] / (kt["kc_apply"][0] * 1e-3) / 1e9
    kernels = {k: {"ms": round(v[0], 5), "launches": v[1]} for k, v in kt.items()}

    # ---------------- FP64 plain path on the same workload
    fp64 = None
    if not args.skip_fp64:
        co64 = ctx.bse_build_coarse(sysm.model, sysm.n_coarse, bse.PREC_F64)
        it64 = ctx.bse_interp_setup(co64, sysm.n_div, bse.SCHEME_M3, 1.0, bse.PREC_F64)
        ms64, res64, eps64 = time_runs(ctx, bse, it64, dirs, m, bse.USE_GRAPH, 1, 1, omega, pref, eta, barrier)
        err = max(float(np.max(np.abs(eps_mixed[c].imag - eps64[c].imag)) / np.max(np.abs(eps64[c].imag)))
                  for c in range(p))
        fp64 = {"chain_steps_per_s": chain_steps / (ms64 / 1e3), "ms_per_run": ms64,
                "max_im_eps_err_mixed_vs_fp64": err}
        it64.free()
        co64.free()

    # ---------------- end to end through the public API with host buffers
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    co_e = ctx.bse_build_coarse(sysm.model, sysm.n_coarse, bse.PREC_BF16)
    it_e = ctx.bse_interp_setup(co_e, sysm.n_div, bse.SCHEME_M3, 1.0, bse.PREC_F32)
    a, b, pn2, sd, _ = ctx.bse_haydock_run([it_e], [p], dirs, m, bse.USE_GRAPH)
    eps_e = ctx.bse_spectrum(a, b, pn2, sd, pref, eta, omega)
    torch.cuda.synchronize()
    t_e2e = time.perf_counter() - t0
    mm = sysm.model
    h2d = 8 * (mm.offsets.size + 2 * (mm.gen_v.size + mm.gen_c.size + mm.mu.size + mm.dip.size)) + 8 * dirs.size
    h2d += 8 * (a.size + b.size + pn2.size + omega.size) + 4 * sd.size
    d2h = 8 * (a.size + b.size + pn2.size) + 4 * sd.size + 16 * eps_e.size
    it_e.free()
    co_e.free()

    # ---------------- uneven batch: 24 systems, 72 chains, 200 steps, one graph launch
    batched = None
    if not args.skip_batched:
        batched = run_batched(ctx, bse, synth, barrier)

    # ---------------- CPU oracle baseline (rank 0 only)
    cpu = None
    if rank == 0 and ws == 1 and not args.skip_cpu:
        cpu = cpu_baseline(sysm, rows=24)

    launches_per_step = 1 + 2 + 1 + 1 + 4          # restrict, tc apply + reduce, near field, prolong, 4 Lanczos
    launches = args.steps * (m * launches_per_step + 3 + 1)
    if rank == 0:
        line = {
            "metric": "Haydock steps/s at N transitions, mixed vs FP64 plain; max Im eps error",
            "value": value, "unit": "chain-steps/s", "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": t_max * 1e3, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "bf16 K_c / f32 vectors / f64 reductions", "data": "synthetic model crystal (seeded)",
            "config": {"workload": "single system: coarse 8^3, 4v x 4c, n_div 4, N = 524288, 3 polarisations, "
                                   "300 Lanczos steps, M3 w = 1, 1000 frequencies",
                       "N": info["N"], "N_c": info["Nc"], "chains": p, "lanczos_steps": m,
                       "l2": "working set above L2 (BF16 K_c alone 268 MB)", "parallelism": f"replicas x{ws}"},
            "fp64_plain": fp64,
            "kernels_ms_per_launch": kernels,
            "kc_apply": {"achieved_GBs": kc_gbs, "frac_of_hbm": kc_gbs / hbm_peak, "bytes_per_launch": kc["bytes"]},
            "roofline": roof,
            "clocks": clk,
            "e2e": {"value": chain_steps / t_e2e, "unit": "chain-steps/s", "h2d_bytes_per_step": int(h2d),
                    "d2h_bytes_per_step": int(d2h), "includes": "build_coarse + interp_setup + haydock + spectrum"},
            "gpu_launches": launches,
            "batched_24_systems": batched,
            "cpu_baseline": cpu,
        }
        print(json.dumps(line))
    it.free()
    co.free()
    ctx.close()
    if ws > 1:
        dist.destroy_process_group()


def run_batched(ctx, bse, synth, barrier, m=200):
    """The uneven batch (24 seeded systems: coarse 4^3-8^3, n_div 2-4, bands
    2x2-6x6, eps_inf ~ U(5, 15), kappa ~ U(0.2, 0.5), 3 polarisations each,
    M3 w = 1, BF16 K_c) as one CUDA-graph launch per Haydock run."""
    import torch
    systems = synth.batched_systems()
    t0 = time.perf_counter()
    hs = []
    for s in systems:
        co = ctx.bse_build_coarse(s.model, s.n_coarse, bse.PREC_BF16)
        hs.append((co, ctx.bse_interp_setup(co, s.n_div, bse.SCHEME_M3, 1.0, bse.PREC_F32)))
    torch.cuda.synchronize()
    t_setup = time.perf_counter() - t0
    dirs = np.concatenate([s.pol_dirs for s in systems])
    its = [h[1] for h in hs]
    ctx.bse_haydock_run(its, [3] * len(its), dirs, m, bse.USE_GRAPH)           # warm-up
    barrier()
    st = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(st)
    ctx.bse_haydock_run(its, [3] * len(its), dirs, m, bse.USE_GRAPH)
    e1.record(st)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    for co, it in hs:
        it.free()
        co.free()
    return {"value": 3 * len(systems) * m / (ms / 1e3), "unit": "chain-steps/s", "systems": len(systems),
            "chains": 3 * len(systems), "lanczos_steps": m, "ms_per_run": ms, "setup_s": t_setup,
            "sum_N": int(sum(s.n_dense_dim for s in systems)), "launch": "one CUDA graph per run"}


def cpu_baseline(sysm, rows=24, reps=1):
    """The FP64 oracle, as it stands, on the host cores: one M1 matrix-free H
    application (Eqs. matmul1-3) on the full vector and the M3 near field on a
    sample of dense rows, extrapolated to one full Lanczos chain step."""
    from oracle import interp as oi
    from paper_1602_01863_gb300 import synth
    I = oi.Interp(sysm.model, sysm.n_coarse, sysm.n_div, width=1.0)
    v = synth.random_vectors(1, I.N)
    t0 = time.perf_counter()
    for _ in range(reps):
        I.apply_m1(v)
    t_m1 = (time.perf_counter() - t0) / reps
    sample = np.linspace(0, I.Nk - 1, rows).astype(np.int64)
    t0 = time.perf_counter()
    I.near_field_rows(v, sample)
    t_nf = (time.perf_counter() - t0) / rows * I.Nk
    t_step = t_m1 + t_nf
    return {"value": 1.0 / t_step, "unit": "chain-steps/s", "cores": os.cpu_count(), "kind": "oracle",
            "sample": f"one full M1 apply ({t_m1:.2f} s) + M3 near field on {rows} of {I.Nk} dense rows, "
                      f"extrapolated to a full chain step ({t_step:.0f} s)"}


def run_reference(args):
    ws, rank, local = dist_info()
    if rank != 0:
        return
    from oracle import interp as oi
    from paper_1602_01863_gb300 import synth
    sysm = synth.single_system(seed=2)
    I = oi.Interp(sysm.model, sysm.n_coarse, sysm.n_div, width=1.0)
    v = synth.random_vectors(1, I.N)
    rows = 8
    times = []
    for k in range(args.warmup + args.steps):
        sample = (np.arange(rows) * 4099 + 17 * k) % I.Nk
        t0 = time.perf_counter()
        I.apply_m1(v)
        t1 = time.perf_counter()
        I.near_field_rows(v, sample)
        t2 = time.perf_counter()
        if k >= args.warmup:
            times.append((t1 - t0) + (t2 - t1) / rows * I.Nk)
    t_step = float(np.mean(times))
    value = 1.0 / t_step
    line = {"metric": "Haydock steps/s at N transitions, mixed vs FP64 plain; max Im eps error", "impl": "reference",
            "value": value, "unit": "chain-steps/s", "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": t_step * 1e3, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64", "data": "synthetic model crystal (seeded)",
            "config": {"workload": "single system: coarse 8^3, 4v x 4c, n_div 4, N = 524288, 3 polarisations, "
                                   "300 Lanczos steps, M3 w = 1, 1000 frequencies"},
            "cpu_baseline": {"value": value, "unit": "chain-steps/s", "cores": os.cpu_count(), "kind": "oracle",
                             "sample": f"per step: one full M1 apply + M3 near field on {rows} dense rows, "
                                       "extrapolated to a full chain step"},
            "e2e": {"value": value, "unit": "chain-steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


if __name__ == "__main__":
    a = parse()
    if a.impl == "reference":
        run_reference(a)
    else:
        run_ours(a)
