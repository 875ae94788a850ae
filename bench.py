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
# committed ncu capture (profiles/k_near_tc_single_system.md: 428.7 + 56.5 MB),
# or None when the kernel changed since the capture.
NEAR_TRAFFIC = 485.2e6


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
    p.add_argument("--skip-largest", action="store_true")
    p.add_argument("--sweep", action="store_true",
                   help="instead of the benchmark: the Method-3 width sweep and the Matmul scaling grid")
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
    the method).  The factored form of the Method-3 correction (Sec. 4, Eq. diverg):
      y1(k, k~') = sum_{k' near k} h_head(q_d) x(k', k~'),  z(k, k~') = sum x(k', k~')
      u(k, k~)  += A_c(k~, k~') [y1(k, k~') - h_head(q_c) z(k, k~')]
      useful   real flops of that form -- per (target, source piece) near pair,
               y1 and z each gain t complex entries times a real scalar
               (4 t real multiply-adds = 8 t flops); per (target, active target
               corner, reached source corner) the head block is applied once to
               y1 - h_head(q_c) z: t complex scalings and subtractions (4 t flops)
               and a t x t complex matrix-vector product (8 t^2 flops);
      issued   real flops of the tensor-core MMAs the kernel issues (stage 1:
               128 x 32 chains x 32 per 32-row K-block; stage 2: two 128-row
               halves x 64 chains x 64 per reached slot)."""
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
    useful = nkc * nchains * (pairs * 8 * t + s2 * (8 * t * t + 4 * t))
    nkg = sum((len(v) + 31) // 32 for v in rows.values())
    issued = nkc * 2 * (nkg * 128 * 32 * nchains * 32 + len(rows) * 2 * 128 * 64 * nchains * 64)
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
    # FP16 dense tensor peak (the near field's operands): the measured BF16 figure
    # (FP16 and BF16 run at the same dense rate); sustained, since the kernel is
    # timed inside a long Haydock run
    f16_peak = float(peaks.get("bf16_tflops_sustained", 1700.0))
    nfw = near_field_work(sysm.n_div, 1.0, info["nv"] * info["nc"], p, sysm.nk_coarse)
    if dom == "near_field":
        achieved = nfw["useful_flops"] / (kt[dom][0] * 1e-3) / 1e12
        roof = {"bound": "tensor", "kernel": "k_near_tc (M3 near field, tcgen05 FP16 operands, FP32 accumulation)",
                "achieved": achieved, "peak": f16_peak, "unit": "TFLOP/s", "frac": achieved / f16_peak,
                "traffic": NEAR_TRAFFIC,
                "peak_source": f"{peak_src} bf16 sustained (FP16 dense rate = BF16)",
                "flops": "useful flops of the factored near field per launch "
                         f"({nfw['useful_flops'] / 1e9:.1f} GFLOP: stage 1 y1, z; head block once on y1 - h_c z)",
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
        errs = [float(np.max(np.abs(eps_mixed[c].imag - eps64[c].imag)) / np.max(np.abs(eps64[c].imag)))
                for c in range(p)]
        a_m, a_p = res[0], res64[0]
        fp64 = {"chain_steps_per_s": chain_steps / (ms64 / 1e3), "ms_per_run": ms64,
                "max_im_eps_err_mixed_vs_fp64": max(errs), "im_eps_err_per_chain": errs,
                "a_1_10_max_rel_diff_mixed_vs_fp64": float(np.max(np.abs(a_m[:, :10] - a_p[:, :10]) / np.abs(a_p[:, :10])))}
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
    largest = None
    if not args.skip_largest:
        largest = run_largest(ctx, bse, synth, barrier)

    # ---------------- CPU oracle baseline (rank 0 only)
    cpu = None
    if rank == 0 and ws == 1 and not args.skip_cpu:
        cpu = cpu_baseline(rows=24)


    launches_per_step = 1 + 1 + 1 + 1 + 2          # restrict, tc apply, near field, prolong, 2 Lanczos
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
            "largest_system": largest,
            "cpu_baseline": cpu,
        }
        print(json.dumps(line))
    it.free()
    co.free()
    ctx.close()
    if ws > 1:
        dist.destroy_process_group()


def train_network(ctx, bse, synth, nv, nc, n=4, nd=4, radius=8, seeds=range(200, 208), blocks=512, steps=2500):
    """A residual network for nv x nc bands trained on the method's own pairs
    (bse_pairs_generate: N_k (K_explicit - K_M1) on dense pairs closer than
    `radius` dense steps) of seeded coarse n^3 systems refined by nd, with the
    library's forward / backward / Adam kernels.  Returns (mlp, first, last loss)."""
    import torch
    t = nv * nc
    d_in = 6 + 2 * t
    rng = np.random.default_rng(123)
    L = n * nd
    g = np.stack(np.meshgrid(*(np.arange(n),) * 3, indexing="ij"), -1).reshape(-1, 3)
    sj = np.stack(np.meshgrid(*(np.arange(nd),) * 3, indexing="ij"), -1).reshape(-1, 3)
    gint = (np.repeat(g, nd ** 3, axis=0) * nd + np.tile(sj, (n ** 3, 1)))        # coarse-major dense coordinates
    lin = {tuple(v): i for i, v in enumerate(gint)}
    r2 = radius * radius
    offs = np.array([(a, b, c) for a in range(-radius, radius + 1) for b in range(-radius, radius + 1)
                     for c in range(-radius, radius + 1) if a * a + b * b + c * c < r2])
    Xs, Ys = [], []
    for seed in seeds:
        m = synth.draw_model(seed, nv, nc)
        co = ctx.bse_build_coarse(m, n, bse.PREC_F32)
        it = ctx.bse_interp_setup(co, nd, bse.SCHEME_M1, 1.0, bse.PREC_F32)
        kd = rng.integers(0, it.Nk, blocks)
        pick = offs[rng.integers(0, len(offs), blocks)]
        kd2 = np.array([lin[tuple(np.mod(gint[k] - d, L))] for k, d in zip(kd, pick)])
        X = torch.zeros((blocks * t * t, d_in), dtype=torch.float32, device="cuda")
        Y = torch.zeros((blocks * t * t, 2), dtype=torch.float32, device="cuda")
        ctx.bse_pairs_generate(it, kd, kd2, X.data_ptr(), Y.data_ptr())
        Xs.append(X)
        Ys.append(Y)
        it.free()
        co.free()
    X = torch.cat(Xs)
    Y = torch.cat(Ys)
    init = np.random.default_rng(11)
    dims = [d_in, 128, 128, 128, 2]
    params = []
    for i in range(4):
        params.append(init.standard_normal((dims[i + 1], dims[i])).reshape(-1) * np.sqrt(2.0 / dims[i]))
        params.append(np.zeros(dims[i + 1]))
    mlp = ctx.bse_mlp_create(d_in, 4096, np.concatenate(params).astype(np.float32))
    prng = np.random.default_rng(5)
    first = last = None
    for step in range(steps):
        idx = torch.from_numpy(prng.integers(0, X.shape[0], 4096)).cuda()
        xb, yb = X[idx].contiguous(), Y[idx].contiguous()
        loss = ctx.bse_mlp_train_step(mlp, 4096, xb.data_ptr(), yb.data_ptr(), 2e-3 if step < 0.6 * steps else 5e-4)
        first = loss if first is None else first
        last = loss
    del X, Y, Xs, Ys
    torch.cuda.empty_cache()
    return mlp, first, last


def run_largest(ctx, bse, synth, barrier, m=500, nw=2000):
    """The largest single system: coarse 12^3, 4v x 6c, n_div 4 (N = 2654208),
    BF16 K_c 41472^2 (6.9 GB), 3 polarisations, 500 steps, 2000 frequencies,
    Method 1 with the learned near-diagonal correction (network trained here on
    coarse 4^3 4v x 6c systems, seeds 200-207) and the FP64 continued fraction."""
    import torch
    s = synth.largest_system()
    t0 = time.perf_counter()
    mlp, first, last = train_network(ctx, bse, synth, s.model.nv, s.model.nc)
    t_train = time.perf_counter() - t0
    t0 = time.perf_counter()
    co = ctx.bse_build_coarse(s.model, s.n_coarse, bse.PREC_BF16)
    it = ctx.bse_interp_setup(co, s.n_div, bse.SCHEME_M1, 1.0, bse.PREC_F32)
    ctx.bse_interp_set_learned(it, mlp, 8)
    torch.cuda.synchronize()
    t_setup = time.perf_counter() - t0
    w = synth.frequency_grid(nw)
    pref = synth.S_EPS / s.nk_dense
    ctx.bse_haydock_run([it], [3], s.pol_dirs, m, bse.USE_GRAPH)                     # warm-up (graph capture)
    barrier()
    st = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(st)
    a, b, pn2, sd, rc = ctx.bse_haydock_run([it], [3], s.pol_dirs, m, bse.USE_GRAPH)
    eps = ctx.bse_spectrum(a, b, pn2, sd, pref, synth.ETA, w)
    e1.record(st)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    ctx.bse_haydock_run([it], [3], s.pol_dirs, 10, bse.PROFILE)
    kt = ctx.bse_last_kernel_times()
    ok = bool(np.all(np.isfinite(a)) and np.all(b[:, 1:] > 0) and np.all(eps.imag > -1e-9 * np.abs(eps.imag).max()))
    it.free()
    co.free()
    mlp.free()
    return {"value": 3 * m / (ms / 1e3), "unit": "chain-steps/s", "ms_per_run": ms, "chains": 3, "lanczos_steps": m,
            "N": s.n_dense_dim, "N_c": s.n_coarse_dim, "frequencies": nw, "kc_bytes": 4 * s.n_coarse_dim ** 2,
            "kernels_ms_per_launch": {k: round(v[0], 5) for k, v in kt.items()},
            "learned": {"radius_dense_steps": 8, "train_loss_first": first, "train_loss_last": last,
                        "train_s": t_train}, "setup_s": t_setup, "finite_positive": ok,
            "workload": "coarse 12^3, 4v x 6c, n_div 4, N = 2654208, BF16 K_c 41472^2, M1 + learned correction, "
                        "3 polarisations, 500 steps, 2000 frequencies"}


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


def cpu_model() -> str:
    """The host CPU's model name (first model-name line of /proc/cpuinfo, or the
    Arm part number when the kernel lists none)."""
    try:
        txt = open("/proc/cpuinfo").read()
    except OSError:
        return "unknown"
    arm_parts = {"0xd4f": "Arm Neoverse V2", "0xd40": "Arm Neoverse V1", "0xd0c": "Arm Neoverse N1",
                 "0xd49": "Arm Neoverse N2", "0xd83": "Arm Neoverse V3"}
    for key in ("model name", "Model Name", "CPU part"):
        for line in txt.splitlines():
            if line.split(":")[0].strip() == key:
                val = line.split(":", 1)[1].strip()
                return arm_parts.get(val, f"{key}: {val}") if key == "CPU part" else val
    return "unknown"


CPU_SAMPLE_CODE = """
import json, sys, time
import numpy as np
sys.path.insert(0, {root!r})
from oracle import interp as oi
from paper_1602_01863_gb300 import synth
sysm = synth.single_system(seed=2)
I = oi.Interp(sysm.model, sysm.n_coarse, sysm.n_div, width=1.0)
v = synth.random_vectors(1, I.N)
t0 = time.perf_counter()
I.apply_m1(v)
t_m1 = time.perf_counter() - t0
sample = np.linspace(0, I.Nk - 1, {rows}).astype(np.int64)
t0 = time.perf_counter()
I.near_field_rows(v, sample)
t_nf = (time.perf_counter() - t0) / {rows} * I.Nk
print(json.dumps({{"t_m1": t_m1, "t_nf": t_nf, "nk": I.Nk}}))
"""


def cpu_baseline(rows=24):
    """The FP64 oracle, as it stands, on the host cores: one M1 matrix-free H
    application (Eqs. matmul1-3) on the full vector and the M3 near field on a
    sample of dense rows, extrapolated to one full Lanczos chain step; run with
    every core and with one (OMP / BLAS threads 1), each in a fresh process."""
    out = {}
    for label, threads in (("all", None), ("one", 1)):
        env = dict(os.environ)
        if threads:
            for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
                env[k] = str(threads)
        r = subprocess.run([sys.executable, "-c", CPU_SAMPLE_CODE.format(root=ROOT, rows=rows)], env=env,
                           capture_output=True, text=True, timeout=900)
        res = json.loads(r.stdout.strip().splitlines()[-1])
        out[label] = res
    t_all = out["all"]["t_m1"] + out["all"]["t_nf"]
    t_one = out["one"]["t_m1"] + out["one"]["t_nf"]
    return {"value": 1.0 / t_all, "unit": "chain-steps/s", "cores": os.cpu_count(), "kind": "oracle",
            "value_one_core": 1.0 / t_one, "cpu": cpu_model(),
            "sample": f"one full M1 apply ({out['all']['t_m1']:.2f} s all cores, {out['one']['t_m1']:.2f} s one core) "
                      f"+ M3 near field on {rows} of {out['all']['nk']} dense rows, extrapolated to a full chain "
                      f"step ({t_all:.0f} s all cores, {t_one:.0f} s one core)"}


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


def run_sweep(args):
    """Two studies of Sec. 5.2-5.3 on the synthetic model, through the library only.

    Width sweep (the LiF width figure of Sec. 5.2): held-out seed 299, coarse
    6^3, 3v x 3c, n_div 2, x polarisation, 300 steps (FP64 plain path, CGS2):
    peak-normalised Im eps error of M1 and of M3 at w = 0.5, 1, 1.5, 2 against
    the explicit dense-mesh BSE (the model's kernel built on the 12^3 dense mesh
    itself, interpolated with n_div = 1, i.e. not interpolated), and the near-field
    time per launch of the mixed path at each w.

    Scaling grid (Tab. scalings of Sec. 5.3): 2v x 2c, coarse n^3 for
    n = 4, 5, 6, 8, 10, 12, n_div = 2, 3, 4, mixed path, per-launch device time
    of the Matmul parts (restrict + K_c apply + prolong: M1) and of the M3 near
    field (w = 1, the paper's "Hinterp"), with least-squares fits of
    t_M1 = a N~_k^2 + b N~_k N_div and t_M3near = c N~_k N_div^2."""
    import torch
    from paper_1602_01863_gb300 import bse, synth
    torch.cuda.set_device(0)
    ctx = bse.Context(0, torch.cuda.current_stream().cuda_stream)
    w = synth.frequency_grid(N_OMEGA)
    m = synth.draw_model(299, 3, 3)
    n, nd, steps = 6, 2, 300
    e = np.array([[1.0, 0.0, 0.0]])
    pref = synth.S_EPS / (n * nd) ** 3

    def spectrum(co_n, ndiv, scheme, width, kc, vec, flags=bse.REORTH_CGS2):
        co = ctx.bse_build_coarse(m, co_n, kc)
        it = ctx.bse_interp_setup(co, ndiv, scheme, width, vec)
        a, b, pn2, sd, _ = ctx.bse_haydock_run([it], [1], e, steps, flags)
        eps = ctx.bse_spectrum(a, b, pn2, sd, pref, synth.ETA, w)[0]
        it.free()
        co.free()
        return eps

    def im_err(x, ref):
        return float(np.max(np.abs(x.imag - ref.imag)) / np.max(np.abs(ref.imag)))

    explicit = spectrum(n * nd, 1, bse.SCHEME_M1, 1.0, bse.PREC_F64, bse.PREC_F64)
    width_rows = [{"method": "M1", "im_eps_err": im_err(spectrum(n, nd, bse.SCHEME_M1, 1.0, bse.PREC_F64, bse.PREC_F64),
                                                        explicit)}]
    for wd in (0.5, 1.0, 1.5, 2.0):
        err = im_err(spectrum(n, nd, bse.SCHEME_M3, wd, bse.PREC_F64, bse.PREC_F64), explicit)
        co = ctx.bse_build_coarse(m, n, bse.PREC_BF16)
        it = ctx.bse_interp_setup(co, nd, bse.SCHEME_M3, wd, bse.PREC_F32)
        ctx.bse_haydock_run([it], [1], e, 20, bse.PROFILE)
        kt = ctx.bse_last_kernel_times()
        width_rows.append({"method": "M3", "w": wd, "n_near": it.n_near, "im_eps_err": err,
                           "near_field_ms": kt["near_field"][0]})
        it.free()
        co.free()

    grid = []
    mg = synth.draw_model(7, 2, 2)
    for ncg in (4, 5, 6, 8, 10, 12):
        for ndv in (2, 3, 4):
            co = ctx.bse_build_coarse(mg, ncg, bse.PREC_BF16)
            row = {"n": ncg, "n_div": ndv, "Nk_coarse": ncg ** 3, "N_div": ndv ** 3}
            for scheme, key in ((bse.SCHEME_M1, "m1"), (bse.SCHEME_M3, "m3")):
                it = ctx.bse_interp_setup(co, ndv, scheme, 1.0, bse.PREC_F32)
                ctx.bse_haydock_run([it], [3], synth.POL3, 10, bse.PROFILE)
                kt = ctx.bse_last_kernel_times()
                row[f"{key}_matmul_ms"] = kt["restrict"][0] + kt["kc_apply"][0] + kt["prolong"][0]
                if scheme == bse.SCHEME_M3:
                    row["m3_near_ms"] = kt["near_field"][0]
                it.free()
            co.free()
            grid.append(row)
    nkc = np.array([r["Nk_coarse"] for r in grid], dtype=float)
    ndiv = np.array([r["N_div"] for r in grid], dtype=float)
    t1 = np.array([r["m1_matmul_ms"] for r in grid])
    tn = np.array([r["m3_near_ms"] for r in grid])
    A = np.stack([nkc ** 2, nkc * ndiv], axis=1)
    c1, *_ = np.linalg.lstsq(A, t1, rcond=None)
    c3, *_ = np.linalg.lstsq((nkc * ndiv ** 2)[:, None], tn, rcond=None)
    # power-law exponents of the near field in N~_k (fixed N_div) and N_div (fixed N~_k)
    big = [r for r in grid if r["n_div"] == 4]
    ex_nk = float(np.polyfit(np.log([r["Nk_coarse"] for r in big]), np.log([r["m3_near_ms"] for r in big]), 1)[0])
    at8 = [r for r in grid if r["n"] == 8]
    ex_nd = float(np.polyfit(np.log([r["N_div"] for r in at8]), np.log([r["m3_near_ms"] for r in at8]), 1)[0])
    out = {"width_sweep": {"config": "held-out seed 299, coarse 6^3, 3v x 3c, n_div 2, 300 steps, CGS2; reference: "
                                     "the model's kernel on the 12^3 dense mesh (no interpolation)",
                           "rows": width_rows},
           "scaling": {"config": "2v x 2c, 3 chains, mixed path (BF16 K_c, FP32 vectors), per-launch device times",
                       "rows": grid,
                       "fit_m1_matmul_ms": {"a_Nk2": float(c1[0]), "b_Nk_Ndiv": float(c1[1])},
                       "fit_m3_near_ms": {"c_Nk_Ndiv2": float(c3[0])},
                       "near_field_exponent_in_Nk_at_ndiv4": ex_nk, "near_field_exponent_in_Ndiv_at_n8": ex_nd}}
    print(json.dumps(out))
    ctx.close()


if __name__ == "__main__":
    a = parse()
    if a.sweep:
        run_sweep(a)
    elif a.impl == "reference":
        run_reference(a)
    else:
        run_ours(a)
