#!/usr/bin/env python3
"""Benchmark: hybrid key switches per second for HRotate at N = 2^16, L = 24.

Workload (one "step"): a batch of B independent HRotates at N = 2^16, level
24, K = 8 special primes, dnum = 3, each on its own ciphertext with its own
rotation key (uniform residues, rotation index uniform in [1, 2^15)).  The B
distinct ciphertext + key pairs (~503 MB at B = 8) are larger than the 129 MB
L2, so every step streams its keys from HBM.  The headline `value` replays the
batch as one captured CUDA graph (fused pipeline); the plain per-kernel
pipeline and the fused pipeline without a graph are timed on the same inputs
and reported beside it.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
N > 1 runs one process per GPU under torchrun (each rank its own batch: the
key switches are independent, so ranks share nothing; weak scaling).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = "hrotate_N65536_L24_plain"
METRIC = "key-switches/s at N=2^16,L=24 (HRotate, batched+TC-BConv)"
UNIT = "key-switches/s"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=400)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--batch", type=int, default=8)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extra", action="store_true", help="skip the 64-item batch and linear-transform lines")
    ap.add_argument("--lanes", type=int, default=0, help="concurrent lanes of the batched plans (0: library default)")
    ap.add_argument("--ntt", choices=["auto", "0", "1", "2", "3"], default="auto",
                    help="NTT kernel variant (fhe_ctx_set_ntt flags: 1 on-the-fly twiddles, 2 single pass); "
                         "auto: measured by the autotuner")
    ap.add_argument("--l2-budget-mb", type=int, default=0,
                    help="L2 budget that sizes a plan's item groups, in MB (0: library default)")
    ap.add_argument("--sweep", action="store_true",
                    help="kernel-utilisation sweep (NTT over 10..250 limbs, BConv over output counts, key-switch "
                         "batch sizes) as one JSON line instead of the benchmark line")
    ap.add_argument("--shape", default="",
                    help="kernel shape for --profile-run, comma-separated key=value (fhe_ctx_set_kernel_shape fields, "
                         "e.g. fuse_ip_moddown=1)")
    ap.add_argument("--profile-run", choices=["scalar", "tc", "cts", "lt"], default=None,
                    help="only launch the batched stage programs (one lane, no graph) warmup + steps times, "
                         "in a fixed launch order for profilers ('cts': the CoeffToSlot chain at N = 2^16, "
                         "L = 48 instead; 'lt': the level-24 BSGS transform); prints no JSON line")
    return ap.parse_args()


def rank_seed(base_seed: int, rank: int) -> int:
    """Seed of a rank's batch: every rank key-switches its own inputs (the key
    switches are independent; weak scaling, no data-path collective)."""
    return base_seed + 1000 * rank


def max_over_ranks(ms: float, ws: int, device=None) -> float:
    """The slowest rank's time: the job ends when its last rank does."""
    if ws <= 1:
        return ms
    import torch
    import torch.distributed as dist
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(units_per_rank: int, ws: int, ms: float) -> float:
    """Whole-job rate: the units all ranks processed over the slowest rank's time."""
    return units_per_rank * ws / (ms / 1e3)


def dist_setup(args):
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if ws > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device(f"cuda:{local}"))
    return ws, rank, local


# ---------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi sampling of SM clock and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device: int):
        self.device, self.proc, self.lines = device, None, []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.device), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (FileNotFoundError, OSError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.t.join(timeout=2)
        sm, mx, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            v = [x.strip() for x in ln.split(",")]
            if len(v) < 9:
                continue
            try:
                sm.append(float(v[1]))
                mx = max(mx, float(v[2]))
            except ValueError:
                continue
            for n, flag in zip(names, v[5:9]):
                if flag.lower() == "active":
                    reasons.add(n)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


def arm_config(P, level: int, B: int) -> dict:
    """The workload both arms report (the headline configuration)."""
    return {"workload": f"HRotate x{B} per step, N=2^16 L=24 K=8 dnum=3", "N": P.N, "L": level,
            "K": P.K, "dnum": P.dnum, "batch_per_gpu": B,
            "l2": f"inputs larger than L2: {B} distinct ciphertext+key pairs, "
                  f"{B * (2 * level + 2 * P.dnum * (P.L + P.K)) * P.N * 4 / 1e6:.0f} MB per step"}


# ---------------------------------------------------------------- reference arm: the CPU oracle
def run_reference(args, ws, rank):
    if rank != 0:
        return
    import numpy as np
    import oracle
    from paper_2512_18345_gb300 import inputs
    P = inputs.workload_params(WORKLOAD)
    OP = oracle.OracleParams.from_params(P)
    cores = os.cpu_count() or 1
    oracle.set_num_threads(cores)
    g = inputs.rng(inputs.WORKLOADS[WORKLOAD]["seed"])
    level = P.L
    ct = np.stack([inputs.uniform_residues(g, P.q, P.N) for _ in range(2)])
    key = np.stack([np.stack([inputs.uniform_residues(g, P.primes, P.N) for _ in range(2)]) for _ in range(P.dnum)])
    rot = inputs.rotation_index(g)
    for _ in range(min(args.warmup, 1)):
        oracle.rotate(OP, ct, level, rot, key)
    budget, done, t0 = 120.0, 0, time.perf_counter()
    while done < args.steps:
        oracle.rotate(OP, ct, level, rot, key)
        done += 1
        if time.perf_counter() - t0 > budget:
            break
    dt = time.perf_counter() - t0
    value = done / dt
    sample = (f"{done} HRotates of the workload (one per step instead of {args.batch}; N=2^16, L=24, K=8, "
              f"dnum=3), {args.steps} steps requested, 120 s budget, {cores} threads")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus, "steps": done,
        "warmup": min(args.warmup, 1), "ms_per_step": dt / done * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u32", "data": "synthetic",
        "config": dict(arm_config(P, level, args.batch), path="CPU oracle, one rotation per step"),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": oracle.num_threads(), "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def cpu_baseline(P, ct_np, key_np, rot, budget_s=12.0):
    """The oracle as it stands, one HRotate at a time on all host cores, ~budget_s of work."""
    import oracle
    OP = oracle.OracleParams.from_params(P)
    cores = os.cpu_count() or 1
    oracle.set_num_threads(cores)
    done, t0 = 0, time.perf_counter()
    while True:
        oracle.rotate(OP, ct_np, P.L, rot, key_np)
        done += 1
        if time.perf_counter() - t0 > budget_s or done >= 50:
            break
    dt = time.perf_counter() - t0
    return {"value": done / dt, "unit": UNIT, "cores": oracle.num_threads(), "kind": "oracle",
            "sample": f"{done} HRotates at N=2^16, L=24 (one workload item each), {dt:.1f} s"}


def rand_key_np(inputs, P, g):
    import numpy as np
    return np.stack([np.stack([inputs.uniform_residues(g, P.primes, P.N) for _ in range(2)]) for _ in range(P.dnum)])


def bench_batch64(binding, inputs, roofline, dev, timed, steps, bconv_mode):
    """Fourth workload: 64 ciphertexts, levels uniform in 4..24, relin / rotate mix, one graph."""
    import numpy as np
    name = "batch64_N65536_L4to24"
    w = inputs.WORKLOADS[name]
    P = inputs.workload_params(name)
    g = inputs.rng(w["seed"])
    spec = inputs.batch_items(g, w["items"], w["level_lo"], w["level_hi"])
    ctx = binding.Context.from_params(P, device=dev)
    ctx.set_bconv(bconv_mode)
    ctx.set_relin_key(binding.to_device(rand_key_np(inputs, P, g), dev))
    seen, items, nbytes = set(), [], 0
    for it in spec:
        lv = it["level"]
        a = binding.to_device(np.stack([inputs.uniform_residues(g, P.q[:lv], P.N) for _ in range(2)]), dev)
        out = binding.empty((2, lv, P.N), dev)
        if it["op"] == "rotate":
            if it["rot"] not in seen:
                seen.add(it["rot"])
                ctx.set_rot_key(it["rot"], binding.to_device(rand_key_np(inputs, P, g), dev))
            items.append(dict(op=binding.FHE_OP_ROTATE, level=lv, rot=it["rot"], **{"in": a}, out=out))
        else:
            b = binding.to_device(np.stack([inputs.uniform_residues(g, P.q[:lv], P.N) for _ in range(2)]), dev)
            items.append(dict(op=binding.FHE_OP_RELIN, level=lv, **{"in": a}, in2=b, out=out))
        nbytes += roofline.ks_bytes(P.N, lv, P.K, P.alpha)
    # schedule: measured by the library's autotuner at the mean level of the mix
    tune = ctx.autotune(sum(it["level"] for it in items) // len(items), 16, binding.FHE_TUNE_SHAPE)
    plan = ctx.batch_plan(items, binding.FHE_PLAN_GRAPH)
    for _ in range(3):
        plan.launch()
    k = max(3, min(steps, 30))
    ms = timed(plan.launch, k)
    ctx.sync()
    res = {"value": 64 * k / (ms / 1e3), "unit": "key-switches/s", "ms_per_batch": ms / k, "items": 64,
           "autotune": tune, "groups": plan.groups, "graph_kernels": plan.kernel_count, "bytes_per_batch_model": nbytes,
           "distinct_rotation_keys": len(seen)}
    plan.close()
    ctx.close()
    return res


def bench_lt(binding, inputs, dev, timed, bconv_mode, runs=0):
    """Fifth workload: BSGS linear transform at N = 2^16, level 24, 16 baby x 8 giant steps.
    With `runs`, the transform runs that many times untimed (a profiler's target) and nothing
    is returned."""
    import numpy as np
    name = "bsgs_lt_N65536_L24"
    w = inputs.WORKLOADS[name]
    P = inputs.workload_params(name)
    g = inputs.rng(w["seed"])
    baby, giant, level = w["baby"], w["giant"], P.L
    ctx = binding.Context.from_params(P, device=dev)
    ctx.set_bconv(bconv_mode)
    for r in list(range(1, baby)) + [baby * gg for gg in range(1, giant)]:
        ctx.set_rot_key(r, binding.to_device(rand_key_np(inputs, P, g), dev))
    ct = binding.to_device(np.stack([inputs.uniform_residues(g, P.q, P.N) for _ in range(2)]), dev)
    diags = binding.empty((baby * giant, level, P.N), dev)
    for d in range(baby * giant):
        diags[d].copy_(binding.to_device(inputs.uniform_residues(g, P.q, P.N), dev))
    out = binding.empty((2, level, P.N), dev)
    if runs:
        for _ in range(runs):
            ctx.linear_transform(ct, level, diags, baby, giant, out=out)
        ctx.sync()
        ctx.close()
        print(f"profile run: {runs} BSGS transforms at N={P.N}, level {level}, {baby} x {giant} steps")
        return None
    for _ in range(2):
        ctx.linear_transform(ct, level, diags, baby, giant, out=out)
    k = 5
    ms = timed(lambda: ctx.linear_transform(ct, level, diags, baby, giant, out=out), k)
    ctx.sync()
    # per-kernel breakdown of one call (trace; the auxiliary branch serialised)
    ctx.trace(True)
    ctx.linear_transform(ct, level, diags, baby, giant, out=out)
    stats = ctx.trace_read()
    ctx.trace(False)
    diag_bytes = baby * giant * level * P.N * 4
    ctx.close()
    return {"ms": ms / k, "key_switches": (baby - 1) + (giant - 1), "nominal_steps": [baby, giant],
            "diagonals": baby * giant, "diagonal_bytes": diag_bytes,
            "kernels_ms": {k2: round(v[1], 4) for k2, v in sorted(stats.items(), key=lambda kv: -kv[1][1])}}


def bench_bootstrap_lt(binding, inputs, dev, timed, hbm_peak, only=None, runs=0):
    """Bootstrapping linear transforms at the paper's bootstrapping parameters (N = 2^16,
    L = 48, alpha = K = 12, dnum = 4): CoeffToSlot from l = 48 and SlotToCoeff from l = 33,
    each three radix-32 levels of the special FFT, every level one double-hoisted
    baby-step / giant-step transform plus a rescale.  Keys, ciphertext and diagonals are
    uniform residues (timing does not depend on their values; the diagonals and keys are
    distinct device buffers, so they stream from HBM as real ones would).  With `runs`, the
    chain `only` names runs that many times untimed (a profiler's target) and nothing is
    returned."""
    import numpy as np
    import torch
    name = "cts_stc_N65536_L48_a12"
    w = inputs.WORKLOADS[name]
    P = inputs.workload_params(name)
    g = inputs.rng(w["seed"])
    ctx = binding.Context.from_params(P, device=dev)
    ctx.set_bconv(binding.FHE_BCONV_TC)  # the K = 64 shape for the 12-limb digits
    key = binding.to_device(rand_key_np(inputs, P, g), dev)
    tg = torch.Generator(device=f"cuda:{dev}")
    tg.manual_seed(w["seed"])
    res = {}
    for kind, start in (("cts", w["cts_level"]), ("stc", w["stc_level"])):
        if only and kind != only:
            continue
        plans = inputs.transform_plans(P.N, w["levels"], kind)
        for pl in plans:
            for r in pl.rotations():
                ctx.set_rot_key(r, key)  # the context keeps its own copy per rotation
        levels, pts = [], []
        for i, pl in enumerate(plans):
            level = start - i
            primes = tuple(P.q[:level]) + tuple(P.p)
            d = torch.empty((pl.n_diag, len(primes), P.N), dtype=torch.int64, device=f"cuda:{dev}")
            for j, q in enumerate(primes):
                d[:, j].random_(0, q, generator=tg)
            pts.append(d.to(torch.int32).contiguous())
            del d
            levels.append(level)
        ct = binding.to_device(np.stack([inputs.uniform_residues(g, P.q[:start], P.N) for _ in range(2)]), dev)
        outs = [binding.empty((2, lv, P.N), dev) for lv in levels]
        resc = [binding.empty((2, lv - 1, P.N), dev) for lv in levels]

        def chain():
            x = ct
            for pl, lv, pt, o, r in zip(plans, levels, pts, outs, resc):
                ctx.linear_transform_dh(x, lv, pl.baby, pl.giant, pt, pl.idx, out=o)
                ctx.rescale(o, lv, out=r)
                x = r

        if runs:
            for _ in range(runs):
                chain()
            ctx.sync()
            print(f"profile run: {runs} {kind} chains at N={P.N}, levels {levels}", file=sys.stderr)
            continue
        for _ in range(2):
            chain()
        k = 5
        ms = timed(chain, k) / k
        ctx.sync()
        ctx.trace(True)
        chain()
        stats = ctx.trace_read()
        ctx.trace(False)
        n_ks = sum(sum(1 for r in pl.baby if r % (P.N // 2)) + sum(1 for r in pl.giant if r % (P.N // 2))
                   for pl in plans)
        diag_bytes = sum(pl.n_diag * (lv + P.K) * P.N * 4 for pl, lv in zip(plans, levels))
        # the diagonal kernel's algorithmic bytes: each diagonal once, each baby rotation once per
        # group of 4 giant steps, each inner sum written once (extended basis, both halves)
        mac_bytes = sum((pl.n_diag + 2 * len(pl.baby) * -(-len(pl.giant) // 4) + 2 * len(pl.giant)) *
                        (lv + P.K) * P.N * 4 for pl, lv in zip(plans, levels))
        mac_ms = stats.get("diag_mac", (0, 0.0))[1]
        # the hoisted inner products' algorithmic bytes: per rotating baby step its key and its u
        # over the extended basis, the shared digit set and pass-through once per level; per
        # rotating giant step its key, its own digit set and its u
        ip_words = 0
        for pl, lv in zip(plans, levels):
            beta, ext = P.beta(lv), lv + P.K
            nb = sum(1 for r in pl.baby if r % (P.N // 2))
            ng = sum(1 for r in pl.giant if r % (P.N // 2))
            if nb:
                ip_words += nb * (2 * beta + 2) * ext + beta * ext + lv
            ip_words += ng * (3 * beta + 2) * ext
        ip_bytes = ip_words * P.N * 4
        ip_ms = stats.get("inner_product", (0, 0.0))[1]
        res[kind] = {
            "ms": ms, "levels": levels, "key_switches": n_ks, "ks_per_s": n_ks / (ms / 1e3),
            "diagonals": [pl.n_diag for pl in plans], "baby_giant": [[len(pl.baby), len(pl.giant)] for pl in plans],
            "diagonal_bytes": diag_bytes, "hbm_floor_ms": diag_bytes / (hbm_peak * 1e9) * 1e3,
            "diag_mac": {"bytes": mac_bytes, "ms_traced": mac_ms,
                         "gbs": mac_bytes / (mac_ms / 1e3) / 1e9 if mac_ms else None,
                         "frac_of_measured_hbm": (mac_bytes / (mac_ms / 1e3) / 1e9) / hbm_peak if mac_ms else None},
            "inner_product": {"bytes": ip_bytes, "ms_traced": ip_ms,
                              "gbs": ip_bytes / (ip_ms / 1e3) / 1e9 if ip_ms else None,
                              "frac_of_measured_hbm": (ip_bytes / (ip_ms / 1e3) / 1e9) / hbm_peak if ip_ms else None},
            "kernels_ms": {k2: round(v[1], 4) for k2, v in sorted(stats.items(), key=lambda kv: -kv[1][1])}}
        del pts, outs, resc
    ctx.close()
    return None if runs else res


def bench_paper_shapes(binding, inputs, roofline, dev, timed, steps, l2_gbs, B=8):
    """The paper's key-switching shapes (alpha = K = 12; (l, beta) = (24, 2), (48, 4)):
    B rotations with distinct keys per step, autotuned schedule and conversion kernel
    (CUDA cores or the tensor-core K = 64 shape), one CUDA graph."""
    import numpy as np
    res = {}
    for name in ("paper_ks_N65536_L24_a12", "paper_ks_N65536_L48_a12"):
        P = inputs.workload_params(name)
        g = inputs.rng(inputs.WORKLOADS[name]["seed"] + 500)
        ctx = binding.Context.from_params(P, device=dev)
        items, used = [], set()
        while len(items) < B:
            r = inputs.rotation_index(g)
            k = pow(5, r % (P.N // 2), 2 * P.N)
            if k in used:
                continue
            used.add(k)
            ctx.set_rot_key(r, binding.to_device(rand_key_np(inputs, P, g), dev))
            ct = binding.to_device(np.stack([inputs.uniform_residues(g, P.q, P.N) for _ in range(2)]), dev)
            items.append(dict(op=binding.FHE_OP_ROTATE, level=P.L, rot=r, **{"in": ct},
                              out=binding.empty((2, P.L, P.N), dev)))
        tune = ctx.autotune(P.L, B, binding.FHE_TUNE_BCONV | binding.FHE_TUNE_SHAPE)
        plan = ctx.batch_plan(items, binding.FHE_PLAN_GRAPH)
        for _ in range(3):
            plan.launch()
        k = max(3, min(steps, 30))
        ms = timed(plan.launch, k)
        ctx.sync()
        t_ks = ms / 1e3 / (k * B)
        pipe = comp_pipe_on_off(binding, ctx, items, timed, k, B)
        ctx.set_pipelining(bool(tune["comp_pipe"]))
        bks = roofline.ks_bytes(P.N, P.L, P.K, P.alpha)
        res[f"l{P.L}_alpha{P.alpha}_beta{P.beta(P.L)}"] = {
            "value": 1.0 / t_ks, "unit": "key-switches/s", "us_per_ks": t_ks * 1e6, "items": B,
            "bytes_per_ks_model": bks, "l2_roofline_frac": (bks / (l2_gbs * 1e9)) / t_ks,
            "groups": plan.groups, "autotune": tune, "comp_pipe_ks_per_s": pipe,
            "bconv": "tensor cores (K = 64)" if tune["bconv_mode"] == binding.FHE_BCONV_TC else "cuda cores"}
        plan.close()
        ctx.close()
    return res


def run_sweep(args, dev):
    """Throughput of the stage kernels against the amount of work per launch (the
    paper's kernel-utilisation and batching study, Section III-B): NTT passes over
    10..250 limbs, BConv with 12 (CUDA cores) or 8 (both kernels) inputs over the
    output count, and batched key switches at l = 24 over the batch size.  Kernel
    times come from the library's trace (CUDA events around each launch)."""
    import numpy as np
    import torch
    from paper_2512_18345_gb300 import binding, inputs
    out = {"ntt": [], "bconv": [], "batch": [], "int_peaks": measure_alu_peaks(binding, dev)}
    alu = ALU_PEAK["bfly"]

    def traced(ctx, fn, reps):
        fn()
        torch.cuda.synchronize()
        ctx.trace(True)
        for _ in range(reps):
            fn()
        stats = ctx.trace_read()
        ctx.trace(False)
        return stats

    P = inputs.workload_params("paper_ks_N65536_L48_a12")  # 60 primes
    ctx = binding.Context.from_params(P, device=dev)
    g = inputs.rng(4242)
    nprime = len(P.primes)
    for L in (10, 24, 48, 96, 160, 250):
        a = binding.to_device(g.integers(0, 1 << 20, size=(L, P.N), dtype=np.uint32), dev)
        idx = [i % nprime for i in range(L)]
        stats = traced(ctx, lambda: ctx.ntt(a, idx), 10)
        row = {"limbs": L}
        for name, (n, ms) in stats.items():
            us = 1e3 * ms / n
            bfly = L * (P.N // 2) * 8
            row[name] = {"us": us, "tbutterflies_per_s": bfly / (us * 1e-6) / 1e12, "frac_alu": bfly / (us * 1e-6) / alu}
        out["ntt"].append(row)
    for n_in, n_outs, modes in ((12, (12, 24, 36, 48), ("scalar",)),):
        for n_out in n_outs:
            x = binding.to_device(g.integers(0, 1 << 20, size=(n_in, P.N), dtype=np.uint32), dev)
            in_idx = list(range(nprime - n_in, nprime))
            out_idx = list(range(n_out))
            stats = traced(ctx, lambda: ctx.bconv(x, in_idx, out_idx), 5)
            n, ms = stats["bconv"]
            us = 1e3 * ms / n
            out["bconv"].append({"n_in": n_in, "n_out": n_out, "kernel": "cuda cores", "us": us,
                                 "tmac_per_s": n_in * n_out * P.N / (us * 1e-6) / 1e12})
    ctx.close()
    P8 = inputs.workload_params("hrotate_N65536_L24_tc")  # alpha = K = 8: both kernels
    ctx = binding.Context.from_params(P8, device=dev)
    for mode, name in ((binding.FHE_BCONV_SCALAR, "bconv"), (binding.FHE_BCONV_TC, "bconv_tc")):
        ctx.set_bconv(mode)
        for n_out in (8, 16, 24):
            x = binding.to_device(g.integers(0, 1 << 20, size=(8, P8.N), dtype=np.uint32), dev)
            in_idx = list(range(24, 32))
            out_idx = list(range(n_out))
            stats = traced(ctx, lambda: ctx.bconv(x, in_idx, out_idx), 5)
            n, ms = stats[name]
            us = 1e3 * ms / n
            out["bconv"].append({"n_in": 8, "n_out": n_out, "kernel": "tensor cores" if name == "bconv_tc" else
                                 "cuda cores", "us": us, "tmac_per_s": 8 * n_out * P8.N / (us * 1e-6) / 1e12})
    # batched key switches at l = 24 over the batch size (default schedule, graph)
    ctx.set_bconv(binding.FHE_BCONV_TC)
    keys, cts = [], []
    for b in range(16):
        r = 1 + 37 * b
        ctx.set_rot_key(r, binding.to_device(rand_key_np(inputs, P8, g), dev))
        cts.append((r, binding.to_device(np.stack([inputs.uniform_residues(g, P8.q, P8.N) for _ in range(2)]), dev)))
    for B in (1, 2, 4, 8, 16):
        items = [dict(op=binding.FHE_OP_ROTATE, level=P8.L, rot=r, **{"in": c}, out=binding.empty((2, P8.L, P8.N), dev))
                 for r, c in cts[:B]]
        plan = ctx.batch_plan(items, binding.FHE_PLAN_GRAPH)
        for _ in range(3):
            plan.launch()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        reps = 20
        e0.record()
        for _ in range(reps):
            plan.launch()
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / reps
        out["batch"].append({"batch": B, "groups": plan.groups, "us_per_ks": 1e3 * ms / B, "ks_per_s": B / (ms / 1e3)})
        plan.close()
    ctx.close()
    print(json.dumps({"sweep": out}), flush=True)


def kernel_model(name, P, level, G, fused_ip_md=False):
    """Algorithmic bytes and operations of the stage kernel `name` summed over its
    launches in one batched group of G HRotates at `level` (fused pipeline): each
    NTT pass reads and writes its limbs once, the base conversions read their input
    and write their output limbs once, the inner product reads the decomposed limbs
    and both key halves and writes two extended polynomials.  With fused_ip_md the
    special limbs' inner product and ModDown's first inverse pass are one kernel
    ("ip+intt_blk": the K special limbs' digits and keys read once, the pass's two
    outputs written), and the inner product covers the ciphertext limbs only."""
    W = 4 * P.N
    K, A, beta = P.K, P.alpha, P.beta(level)
    widths = [min(A, level - j * A) for j in range(beta)]
    conv = sum(level + K - w for w in widths)  # limbs ModUp produces by conversion
    logn = P.N.bit_length() - 1
    bf_col, bf_blk = P.N // 2 * (logn - 8), P.N // 2 * 8  # butterflies of one pass over one limb
    macs = (sum(w * (level + K - w) for w in widths) + 2 * K * level) * P.N
    m = {
        "intt_blk+gather": (2 * level * W, level * bf_blk, "bfly"),
        "intt_col+scale": (2 * (level + 2 * K) * W, (level + 2 * K) * bf_col, "bfly"),
        "ntt_col": (2 * (conv + 2 * level) * W, (conv + 2 * level) * bf_col, "bfly"),
        "ntt_blk": (2 * conv * W, conv * bf_blk, "bfly"),
        "intt_blk": (2 * 2 * K * W, 2 * K * bf_blk, "bfly"),
        "ntt_blk+combine": (7 * level * W, 2 * level * bf_blk, "bfly"),
        "bconv": ((level + conv + 2 * K + 2 * level) * W, macs, "mac"),
        "bconv_tc": ((level + conv + 2 * K + 2 * level) * W, macs, "mac"),
        # per extended limb: beta decomposed limbs, 2 beta key limbs, two u limbs; plus the
        # pass-through limb (sigma(c0)) each q-limb reads for the u += P sigma(c0) fold
        "inner_product": (((level + K) * (3 * beta + 2) + level) * W, 2 * beta * (level + K) * P.N, "mac"),
    }
    if fused_ip_md:
        m["inner_product"] = ((level * (3 * beta + 2) + level) * W, 2 * beta * level * P.N, "mac")
        m["ip+intt_blk"] = (K * (3 * beta + 2) * W, 2 * beta * K * P.N + 2 * K * bf_blk, "mac")
    b, o, unit = m.get(name, (0, 0, "bfly"))
    return b * G, o * G, unit


# ALU peaks: measured on the device by the library's integer-pipe probe (fhe_probe_int) --
# register-only chains of the NTT's forward Shoup butterfly and of the 64-bit
# multiply-accumulate, at four CTAs per SM -- and filled in by main(); the fallback below is
# the earlier derivation (16 butterflies and 23 multiply-accumulates per clock per SM,
# 152 SMs, 2.07 GHz), used only when the probe fails.
ALU_PEAK = {"bfly": 16 * 152 * 2.07e9, "mac": 23 * 152 * 2.07e9}
ALU_PEAK_SOURCE = ["derived from probe unit counts x 152 SMs x 2.07 GHz"]
NTT_KERNELS = ("intt_blk+gather", "intt_col+scale", "ntt_col", "ntt_blk", "intt_blk", "ntt_blk+combine")


def measured_traffic_per_item(name, fused_ip_md=False):
    """DRAM bytes per item of kernel `name` (summed over its launches in one group) from
    its committed ncu summary, or None when there is none or the kernel's sources
    changed since the capture.  With the fused special-limb kernel the inner product
    covers the q-limbs only (its own figure in the summary)."""
    import hashlib
    import re
    files = {"inner_product": "inner_product_N65536_L24.md"}
    if name not in files:
        return None
    try:
        text = open(os.path.join(ROOT, "profiles", files[name])).read()
        key = "traffic_bytes_per_item_qlimbs" if fused_ip_md else "traffic_bytes_per_item"
        per_item = int(re.search(r"^" + key + r": (\d+)$", text, re.M).group(1))
        want = re.search(r"^kernel_sources_sha256: ([0-9a-f]+)$", text, re.M).group(1)
        srcs = re.search(r"^kernel_sources: (.+)$", text, re.M).group(1).split()
        h = hashlib.sha256()
        for f in srcs:
            h.update(open(os.path.join(ROOT, f), "rb").read())
    except (OSError, AttributeError, ValueError):
        return None
    return per_item if h.hexdigest() == want else None


def kernel_roofline(name, launches_per_group, launch_ms, P, level, G, hbm_peak, fused_ip_md=False):
    """Roofline entry of one kernel: the bound (HBM bytes or ALU operations) with the
    larger achieved fraction of its peak."""
    nbytes, ops, unit = kernel_model(name, P, level, G, fused_ip_md)
    lpg = max(launches_per_group, 1e-9)
    per_launch_bytes, per_launch_ops = nbytes / lpg, ops / lpg
    gbs = per_launch_bytes / (launch_ms / 1e3) / 1e9
    ach_ops = per_launch_ops / (launch_ms / 1e3)
    f_hbm, f_alu = gbs / hbm_peak, ach_ops / ALU_PEAK[unit]
    per_item = measured_traffic_per_item(name, fused_ip_md)
    common = {"traffic": per_item * G / lpg if per_item else None, "kernel": name, "launch_ms": launch_ms,
              "algorithmic_bytes_per_launch": per_launch_bytes, "algorithmic_ops_per_launch": per_launch_ops,
              "frac_hbm": f_hbm, "frac_alu": f_alu}
    if f_alu >= f_hbm:
        return {"bound": "alu", "achieved": ach_ops / 1e12, "peak": ALU_PEAK[unit] / 1e12, "unit": f"T{unit}/s",
                "frac": f_alu, "peak_source": ALU_PEAK_SOURCE[0], **common}
    return {"bound": "hbm", "achieved": gbs, "peak": hbm_peak, "unit": "GB/s", "frac": f_hbm,
            "peak_source": "measured (hbm_gbs)", **common}


def measure_alu_peaks(binding, dev):
    """Set ALU_PEAK from the library's integer-pipe probe on this device; on failure keep
    the derived fallback and report why."""
    try:
        ipk = binding.probe_int(dev)
        ALU_PEAK["bfly"], ALU_PEAK["mac"] = ipk["butterflies_per_s"], ipk["mac64_per_s"]
        ALU_PEAK_SOURCE[0] = (f"measured (fhe_probe_int register-only chains at {ipk['clock_mhz']:.0f} MHz: "
                              f"{ipk['butterflies_per_s'] / 1e12:.2f} T butterflies/s, "
                              f"{ipk['mac64_per_s'] / 1e12:.2f} T 64-bit MAC/s)")
        return ipk
    except Exception as ex:
        return {"failed": str(ex)}


def kernel_rates(stats, P, level, G, groups_traced, hbm_peak, fused_ip_md=False):
    """Per traced kernel: its algorithmic rate over its summed event time and the fraction of
    the peak that bounds it; and the NTT family's aggregate butterfly rate (all forward and
    inverse passes of the key switch: their butterflies over their summed time)."""
    rows, ntt_ops, ntt_ms = {}, 0.0, 0.0
    for name, (n, t_ms) in stats.items():
        nbytes, ops, unit = kernel_model(name, P, level, G, fused_ip_md)
        if not t_ms or not (nbytes or ops):
            continue
        secs = t_ms / 1e3
        ach = ops * groups_traced / secs
        rows[name] = {"alu_rate": ach, "alu_unit": f"{unit}/s", "frac_alu": ach / ALU_PEAK[unit],
                      "gbs": nbytes * groups_traced / secs / 1e9,
                      "frac_hbm": nbytes * groups_traced / secs / 1e9 / hbm_peak}
        if name in NTT_KERNELS:
            ntt_ops += ops * groups_traced
            ntt_ms += t_ms
    fam = None
    if ntt_ms:
        rate = ntt_ops / (ntt_ms / 1e3)
        fam = {"butterflies_per_s": rate, "frac_alu": rate / ALU_PEAK["bfly"], "share_ms": ntt_ms,
               "peak": ALU_PEAK["bfly"], "peak_source": ALU_PEAK_SOURCE[0]}
    return rows, fam


def comp_pipe_on_off(binding, ctx, items, timed, steps, B):
    """Complementary pipelining (Section IV-B) on and off under the context's current
    schedule: key switches per second of the graph-captured plan each way."""
    res = {}
    for on in (True, False):
        ctx.set_pipelining(on)
        pl = ctx.batch_plan(items, binding.FHE_PLAN_GRAPH)
        for _ in range(3):
            pl.launch()
        ms = timed(pl.launch, steps)
        res["on" if on else "off"] = B * steps / (ms / 1e3)
        pl.close()
    return res


def main():
    args = parse()
    ws, rank, local = dist_setup(args)
    if args.impl == "reference":
        run_reference(args, ws, rank)
        if ws > 1:
            import torch.distributed as dist
            dist.destroy_process_group()
        return

    import numpy as np
    import torch
    from paper_2512_18345_gb300 import binding, build, inputs, roofline

    build.build_library()
    dev = local
    torch.cuda.set_device(dev)
    if args.profile_run == "cts":  # the CoeffToSlot chain alone, for a profiler
        bench_bootstrap_lt(binding, inputs, dev, None, 0.0, only="cts", runs=max(3, args.warmup) + args.steps)
        return
    if args.profile_run == "lt":  # the level-24 BSGS transform alone, for a profiler
        bench_lt(binding, inputs, dev, None, binding.FHE_BCONV_TC, runs=max(3, args.warmup) + args.steps)
        return
    P = inputs.workload_params(WORKLOAD)
    level, B = P.L, args.batch
    g = inputs.rng(rank_seed(inputs.WORKLOADS[WORKLOAD]["seed"], rank))
    ctx = binding.Context.from_params(P, device=dev)
    cts_np, keys_np, rots = [], [], []
    used = set()
    for b in range(B):
        r = inputs.rotation_index(g)
        while pow(5, r % (P.N // 2), 2 * P.N) in used:
            r = inputs.rotation_index(g)
        used.add(pow(5, r % (P.N // 2), 2 * P.N))
        rots.append(r)
        cts_np.append(np.stack([inputs.uniform_residues(g, P.q, P.N) for _ in range(2)]))
        keys_np.append(np.stack([np.stack([inputs.uniform_residues(g, P.primes, P.N) for _ in range(2)])
                                 for _ in range(P.dnum)]))
    cts = [binding.to_device(c, dev) for c in cts_np]
    for r, k in zip(rots, keys_np):
        ctx.set_rot_key(r, binding.to_device(k, dev))
    outs = [binding.empty((2, level, P.N), dev) for _ in range(B)]
    items = [dict(op=binding.FHE_OP_ROTATE, level=level, rot=r, **{"in": c}, out=o) for r, c, o in zip(rots, cts, outs)]
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()

    if args.sweep:
        run_sweep(args, dev)
        ctx.close()
        return

    if args.profile_run:
        ctx.set_fused(True)
        ctx.set_bconv(binding.FHE_BCONV_TC if args.profile_run == "tc" else binding.FHE_BCONV_SCALAR)
        ctx.set_batch(0, 0, 1)
        if args.ntt != "auto":
            ctx.set_ntt(int(args.ntt))
        if args.shape:
            ctx.set_kernel_shape(**{k: int(v) for k, v in (kv.split("=") for kv in args.shape.split(","))})
        plan_p = ctx.batch_plan(items, 0)
        for _ in range(args.warmup + args.steps):
            plan_p.launch()
        ctx.sync()
        print(f"profile run: {B} HRotates at N={P.N}, L={level}, groups {plan_p.groups}, "
              f"{args.warmup + args.steps} launches of {plan_p.kernel_count} kernels", file=sys.stderr)
        plan_p.close()
        ctx.close()
        return

    def timed(fn, steps):
        if ws > 1:
            import torch.distributed as dist
            dist.barrier()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        if ws > 1:
            import torch.distributed as dist
            dist.barrier()
        return max_over_ranks(e0.elapsed_time(e1), ws, f"cuda:{dev}")

    # --- schedule of the batched plans: the library's autotuner (measured on this GPU
    # for this batch, tensor-core BConv kept), unless fixed on the command line
    ctx.set_fused(True)
    tune = None
    if args.lanes or args.l2_budget_mb:
        ctx.set_batch(args.l2_budget_mb << 20, 0, args.lanes)
    else:
        ctx.set_bconv(binding.FHE_BCONV_TC)
        tune = ctx.autotune(level, B, binding.FHE_TUNE_SHAPE | (binding.FHE_TUNE_NTT if args.ntt == "auto" else 0))
    if args.ntt != "auto":
        ctx.set_ntt(int(args.ntt))
    budget = tune["l2_budget_bytes"] if tune else args.l2_budget_mb << 20
    # --- batched fused pipeline in one CUDA graph, CUDA-core base conversion (comparison)
    ctx.set_bconv(binding.FHE_BCONV_SCALAR)
    plan_sc = ctx.batch_plan(items, binding.FHE_PLAN_GRAPH)
    for _ in range(max(3, args.warmup)):
        plan_sc.launch()
    ms_sc = timed(plan_sc.launch, max(3, min(args.steps, 100)))
    graph_scalar_ks = B * max(3, min(args.steps, 100)) * ws / (ms_sc / 1e3)
    plan_sc.close()
    # --- headline: batched fused pipeline, tensor-core base conversion, one CUDA graph
    ctx.set_bconv(binding.FHE_BCONV_TC)
    plan = ctx.batch_plan(items, binding.FHE_PLAN_GRAPH)
    head_groups = plan.groups
    for _ in range(max(3, args.warmup)):
        plan.launch()
    ctx.sync()
    clocks = ClockSampler(dev)
    clocks.start()
    time.sleep(0.15)
    ms = timed(plan.launch, args.steps)
    clk = clocks.stop()
    ctx.sync()
    value = job_throughput(B * args.steps, ws, ms)
    graph_kernels = plan.kernel_count

    # --- per-step distribution (after the timed region): CUDA events on the launching
    # stream around each of a run of back-to-back graph launches
    dist_steps = max(10, min(args.steps, 100))
    evs = [torch.cuda.Event(enable_timing=True) for _ in range(dist_steps + 1)]
    evs[0].record(stream)
    for i in range(dist_steps):
        plan.launch()
        evs[i + 1].record(stream)
    torch.cuda.synchronize()
    step_ms = np.array([evs[i].elapsed_time(evs[i + 1]) for i in range(dist_steps)])
    per_step = {"steps": dist_steps, "median_ms": float(np.median(step_ms)),
                "p10_ms": float(np.percentile(step_ms, 10)), "p90_ms": float(np.percentile(step_ms, 90)),
                "median_ks_per_s": B * ws / (float(np.median(step_ms)) / 1e3)}

    # --- comparison paths on the same inputs (fewer steps)
    cmp_steps = max(3, min(args.steps, 50))

    def direct():
        for it in items:
            ctx.rotate(it["in"], level, it["rot"], out=it["out"])

    ctx.set_bconv(binding.FHE_BCONV_SCALAR)
    for _ in range(3):
        direct()
    ms_fused = timed(direct, cmp_steps)
    ctx.set_fused(False)
    for _ in range(3):
        direct()
    ms_plain = timed(direct, cmp_steps)
    ctx.set_fused(True)
    ctx.set_bconv(binding.FHE_BCONV_TC)
    plain_ks = B * cmp_steps * ws / (ms_plain / 1e3)
    fused_ks = B * cmp_steps * ws / (ms_fused / 1e3)

    # --- warm L2 (labelled; not the headline): the 8 rotations of a step share one
    # ciphertext and one rotation key, so after the first item the key (50 MB) and the input
    # are read from L2; outputs and the ModUp working set are as in the headline
    items_w = [dict(op=binding.FHE_OP_ROTATE, level=level, rot=rots[0], **{"in": cts[0]}, out=o) for o in outs]
    plan_w = ctx.batch_plan(items_w, binding.FHE_PLAN_GRAPH)
    for _ in range(3):
        plan_w.launch()
    ms_warm = timed(plan_w.launch, cmp_steps)
    warm_l2 = {"value": B * cmp_steps * ws / (ms_warm / 1e3), "unit": UNIT, "steps": cmp_steps,
               "inputs": "one ciphertext and one rotation key shared by the step's 8 rotations"}
    plan_w.close()

    # --- complementary pipelining (Section IV-B) on and off under the tuned schedule
    pipe_head = comp_pipe_on_off(binding, ctx, items, timed, cmp_steps, B)
    ctx.set_pipelining(bool(tune["comp_pipe"]) if tune else True)

    # --- per-kernel times (CUDA events around each launch on its stream): the same batched
    # stage programs as the headline, launched directly on one lane (no concurrent lane
    # inflates a kernel's event interval)
    ctx.set_batch(budget, 0, 1)
    plan_direct = ctx.batch_plan(items, 0)
    ctx.set_batch(budget, 0, tune["lanes"] if tune else args.lanes)
    for _ in range(3):
        plan_direct.launch()
    ctx.trace(True)
    for _ in range(cmp_steps):
        plan_direct.launch()
    stats = ctx.trace_read()
    ctx.trace(False)
    ms_batched_direct = timed(plan_direct.launch, cmp_steps)
    batched_direct_ks = B * cmp_steps * ws / (ms_batched_direct / 1e3)
    groups = plan_direct.groups
    plan_direct.close()
    total_ms = sum(v[1] for v in stats.values())
    top_name, (top_n, top_ms) = max(stats.items(), key=lambda kv: kv[1][1])
    per_launch_ms = top_ms / top_n

    # --- peaks: HBM from the measured file; L2 measured here with the library's probe
    # (read + write of a 64 MB block, smaller than the L2, as in the paper's method)
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        pass
    hbm_peak = float(peaks.get("hbm_gbs", 6800.0))
    l2 = binding.probe_bandwidth(dev, 64 << 20, 50)
    l2_gbs = l2["copy"]
    ipk = measure_alu_peaks(binding, dev)

    # algorithmic bytes of the headline step and its L2-roofline fraction (paper's definition)
    bks = roofline.ks_bytes(P.N, level, P.K, P.alpha)
    l2_frac = (bks / (l2_gbs * 1e9)) / ((ms / 1e3) / (B * args.steps))

    # dominant kernel of the batched step: algorithmic bytes and operations per launch
    ngroups = max(1, len(groups))
    fused_md = bool(ctx.kernel_shape()["fuse_ip_moddown"])
    roof = kernel_roofline(top_name, top_n / (cmp_steps * ngroups), per_launch_ms, P, level, B / ngroups,
                           hbm_peak, fused_md)
    roof["share"] = top_ms / total_ms if total_ms else None
    krates, ntt_family = kernel_rates(stats, P, level, B / ngroups, cmp_steps * ngroups, hbm_peak, fused_md)

    # --- e2e: every step copies its inputs from pinned host memory and its results back,
    # inside the timed region, through the same public API.  Steps alternate between two
    # device buffer sets (each with its own plan), so the copies of neighbouring steps run
    # on their own streams beside the current step's key switches.  A step's ciphertexts sit
    # in one contiguous buffer on each side (the items point into it), so each direction is
    # one copy: the host link runs at about 170 GB/s each way for one large copy per
    # direction, 158 GB/s for one copy per ciphertext.
    h_in = torch.from_numpy(np.stack(cts_np).view(np.int32)).pin_memory()  # [B][2][level][N]
    h_out = torch.empty((B, 2, level, P.N), dtype=torch.int32).pin_memory()
    sets = []
    for _ in range(2):
        d_in = torch.empty((B, 2, level, P.N), dtype=torch.int32, device=f"cuda:{dev}")
        d_out = torch.empty_like(d_in)
        items_e = [dict(op=binding.FHE_OP_ROTATE, level=level, rot=r, **{"in": d_in[i]}, out=d_out[i])
                   for i, r in enumerate(rots)]
        sets.append((d_in, d_out, ctx.batch_plan(items_e, binding.FHE_PLAN_GRAPH)))
    s_in, s_out = torch.cuda.Stream(device=dev), torch.cuda.Stream(device=dev)
    ev_in = [torch.cuda.Event() for _ in range(2)]
    ev_done = [torch.cuda.Event() for _ in range(2)]
    ev_back = [torch.cuda.Event() for _ in range(2)]
    for k in range(2):  # nothing pending at the start
        ev_done[k].record(stream)
        ev_back[k].record(stream)
    step_no = [0]

    def e2e_step():
        k = step_no[0] % 2
        step_no[0] += 1
        d_in, d_out, pl = sets[k]
        with torch.cuda.stream(s_in):
            s_in.wait_event(ev_done[k])  # the set's previous step has read its inputs
            d_in.copy_(h_in, non_blocking=True)
            ev_in[k].record(s_in)
        stream.wait_event(ev_in[k])
        stream.wait_event(ev_back[k])  # the set's previous results have been read back
        pl.launch(stream)
        ev_done[k].record(stream)
        with torch.cuda.stream(s_out):
            s_out.wait_event(ev_done[k])
            h_out.copy_(d_out, non_blocking=True)
            ev_back[k].record(s_out)
        if step_no[0] in join_at:  # close the warm-up and the timed region on the main stream
            stream.wait_event(ev_back[0])
            stream.wait_event(ev_back[1])

    # the host link's own rate for these copies (100 MB each way per step): the e2e ceiling
    def link_gbs(copy_fn, reps=5):
        copy_fn()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(reps):
            copy_fn()
        torch.cuda.synchronize()
        return reps * bytes_io / (time.perf_counter() - t0) / 1e9

    bytes_io = B * 2 * level * P.N * 4

    def h2d():
        sets[1][0].copy_(h_in, non_blocking=True)

    def d2h():
        h_out.copy_(sets[1][1], non_blocking=True)

    link = {"h2d_gbs": link_gbs(h2d), "d2h_gbs": link_gbs(d2h)}

    def both():
        with torch.cuda.stream(s_in):
            h2d()
        with torch.cuda.stream(s_out):
            d2h()

    link["concurrent_gbs_each_way"] = link_gbs(both)
    link["copy_bound_ks_per_s"] = B / (bytes_io / (link["concurrent_gbs_each_way"] * 1e9))

    e2e_steps, e2e_warm = max(4, min(args.steps, 50)), 4
    join_at = {e2e_warm, e2e_warm + e2e_steps}
    for _ in range(e2e_warm):
        e2e_step()
    ms_e2e = timed(e2e_step, e2e_steps)
    torch.cuda.synchronize()
    # the results read back equal the headline plan's device results (same inputs and keys)
    # and both buffer sets'
    e2e_ok = all(torch.equal(h_out[i], outs[i].cpu()) for i in range(B)) and \
        all(torch.equal(h_out, s[1].cpu()) for s in sets)
    for s in sets:
        s[2].close()
    e2e_val = job_throughput(B * e2e_steps, ws, ms_e2e)

    # --- the fourth and fifth workloads (reported beside the headline)
    extra = {}
    if not args.no_extra:
        extra["batch64_mixed_levels"] = bench_batch64(binding, inputs, roofline, dev, timed, args.steps,
                                                      binding.FHE_BCONV_TC)
        lt = bench_lt(binding, inputs, dev, timed, binding.FHE_BCONV_TC)
        lt["hbm_floor_ms"] = lt["diagonal_bytes"] / (hbm_peak * 1e9) * 1e3
        extra["bsgs_linear_transform_L24"] = lt
        extra["paper_shapes"] = bench_paper_shapes(binding, inputs, roofline, dev, timed, args.steps, l2_gbs)
        extra["bootstrap_linear_transforms_L48"] = bench_bootstrap_lt(binding, inputs, dev, timed, hbm_peak)

    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        try:
            cpu = cpu_baseline(P, cts_np[0], keys_np[0], rots[0])
        except Exception as ex:  # the oracle is optional on a box without a C compiler
            cpu = {"value": None, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle", "sample": f"failed: {ex}"}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": max(3, args.warmup), "ms_per_step": ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic",
            "config": dict(arm_config(P, level, B),
                           path="fused pipeline, tensor-core BConv, batch captured in one CUDA graph"),
            "gpu_launches": graph_kernels * args.steps,
            "clocks": clk,
            "e2e": {"value": e2e_val, "unit": UNIT, "h2d_bytes_per_step": bytes_io, "d2h_bytes_per_step": bytes_io,
                    "pipelined": "two device buffer sets; a step's copies overlap its neighbours' key switches",
                    "outputs_match": e2e_ok, "host_link": link},
            "roofline": roof,
            "cpu_baseline": cpu,
            # the metric's comparison: plain per-kernel path against batched + tensor-core BConv
            "plain_per_kernel_single_scalar": plain_ks, "graph_batched_scalar_bconv": graph_scalar_ks,
            "graph_batched_tc_bconv": value, "batched_tc_over_plain": value / plain_ks,
            "tc_over_scalar_bconv": value / graph_scalar_ks, "l2_roofline_frac": l2_frac,
            "ntt_family": ntt_family, "int_peaks": ipk,
            "l2_roofline": {"bytes_per_ks": bks, "l2_gbs_measured": l2_gbs, "frac": l2_frac, "l2_probe": l2,
                            "definition": "B_KS(l) / measured L2 read+write bandwidth / time per key switch"},
            "paths": {"graph_batched_tc_bconv": value, "graph_batched_scalar_bconv": graph_scalar_ks,
                      "direct_batched_tc_bconv": batched_direct_ks, "direct_fused_single_scalar": fused_ks,
                      "plain_per_kernel_single_scalar": plain_ks},
            "per_step": per_step, "warm_l2": warm_l2,
            "batch_groups": head_groups, "lanes": tune["lanes"] if tune else (args.lanes or 2),
            "autotune": tune, "traced_groups_one_lane": groups,
            "other_workloads": extra,
            "kernels": {k: dict({"launches": v[0], "ms": v[1], "share": v[1] / total_ms}, **krates.get(k, {}))
                        for k, v in sorted(stats.items(), key=lambda kv: -kv[1][1])},
        }
        # last (the end of the line survives truncated logs): the headline comparisons
        line["summary"] = {
            "ks_per_s": {"graph_batched_tc_bconv": value, "graph_batched_scalar_bconv": graph_scalar_ks,
                         "plain_per_kernel_single_scalar": plain_ks, "e2e": e2e_val},
            "batched_tc_over_plain": value / plain_ks, "tc_over_scalar_bconv": value / graph_scalar_ks,
            "l2_roofline_frac": l2_frac, "inner_product_hbm_frac": roof.get("frac_hbm"),
            "ntt_family_alu_frac": ntt_family["frac_alu"] if ntt_family else None,
            "comp_pipe_ks_per_s": {"headline": pipe_head,
                                   "l48_alpha12_beta4": extra.get("paper_shapes", {}).get(
                                       "l48_alpha12_beta4", {}).get("comp_pipe_ks_per_s")},
        }
        print(json.dumps(line), flush=True)
    plan.close()
    ctx.close()
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
