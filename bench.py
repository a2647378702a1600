"""Benchmark: block-sparse tensordot useful TFLOP/s on one GB300 (or N, one process each).

Workload (default): the large U(1)xU(1) Hubbard-like iPEPS environment contraction
X2 . a over two legs -- bond dimension D = 20 split over 13 charge sectors, chi = D^2 =
400 over 61 sectors, 103,725 + 103,725 blocks, 225 charge sectors up to 4648^3, 1.86e12
useful FLOPs per contraction. Synthetic N(0,1) data (seeded), every allowed block
stored. A step is one full contraction through the C ABI (gather the blocks into sector
matrices, grouped GEMM over all sectors, scatter into the output blocks), plan cached.
Inputs (2.7 GB each) are larger than L2, so no flush is needed between steps.

python bench.py [--gpus N] [--steps K] [--warmup W] [--precision split|fp64]

The headline precision (default: split, at rtol 1e-10) is timed over K steps after W
warm-up steps; the FP64 tensor-core path is timed beside it (--fp64-steps) and the
relative Frobenius difference of the two results is reported.
python bench.py --impl reference ...   (the CPU oracle, timed on host cores)

Multi-GPU (torchrun, one rank per GPU): every rank contracts its own independent
problem (its own seed); there is no data-path collective. value = all ranks' useful
FLOPs / max-over-ranks time ("scaling": "weak").
"""
import os

# The oracle's CPU timing runs numpy with one BLAS thread; set before numpy loads.
for _v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
    os.environ.setdefault(_v, "1")

import argparse  # noqa: E402
import json  # noqa: E402
import subprocess  # noqa: E402
import sys  # noqa: E402
import time  # noqa: E402

import numpy as np  # noqa: E402

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import workloads as W  # noqa: E402

METRIC = "block-sparse tensordot useful TFLOP/s, FP64 vs split-precision at ≤1e-10; p50/p99"


def load_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            return json.load(f), "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


# Nominal GB300 dense rates (TFLOP/s) used to scale the measured BF16 peak to other
# operand types.
NOMINAL = {"bf16": 2250.0, "fp64": 1.25}


def read_traffic(kernel, workload):
    """DRAM bytes per launch of a kernel, from the committed ncu summary (or None)."""
    path = os.path.join(ROOT, "profiles", "traffic.txt")
    if not os.path.exists(path):
        return None
    with open(path) as f:
        for line in f:
            parts = line.split()
            if len(parts) >= 3 and parts[0] == kernel and parts[1] == workload:
                try:
                    return float(parts[2])
                except ValueError:
                    return None
    return None


class ClockSampler:
    """nvidia-smi clocks and throttle reasons, sampled every 200 ms while running."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            out, _ = self.proc.communicate()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            p = [x.strip() for x in line.split(",")]
            if len(p) < 9:
                continue
            try:
                sm.append(float(p[1]))
                smax.append(float(p[2]))
            except ValueError:
                continue
            for n, v in zip(names, p[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": float(max(smax)) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def make_workload(name, rank):
    seed_shift = 100 * rank
    if name == "cfg5":
        return W.config5(seed=5001 + seed_shift)
    if name == "cfg5b":
        return W.config5b(seed=5101 + seed_shift)
    if name == "d14":
        return W.config5(seed=5201 + seed_shift, D=14)
    if name == "cfg3":
        c = W.config3(seed=3001 + seed_shift)
        dl = c["dleg"]
        a = W.random_tensor((0, 0), [W.Leg(-1, dl.t, dl.D), W.Leg(1, dl.t, dl.D), W.Leg(1, dl.t, dl.D),
                                     W.Leg(-1, dl.t, dl.D)], (0, 0), 3999 + seed_shift)
        return {"A": c["X2"], "B": a, "axa": (1, 2), "axb": (0, 1), "dleg": dl, "name": c["name"]}
    raise ValueError(name)


WORKLOAD_DESC = {
    "cfg5": "U(1)xU(1) iPEPS environment contraction X2.a, D=20 (13 sectors), chi=400 (61 sectors)",
    "cfg5b": "U(1)xU(1) iPEPS environment contraction X2.a, D=20 (9 sectors, 25-sector D^2 legs), chi=400",
    "cfg3": "U(1)xU(1) CTMRG X2.a, D=12, chi=144",
    "d14": "U(1)xU(1) iPEPS environment contraction X2.a, D=14, chi=D^2 (profiling size)",
}


# ------------------------------------------------------------------ CPU oracle baseline

def oracle_sample(cfg, budget_s, seed=0):
    """Time the CPU oracle on a bounded sample of the workload: the contraction restricted
    to a random subset of the contracted charge tuples x (every block pair of those x).
    Returns (useful FLOPs, seconds, description)."""
    import oracle as O
    A, B, axa, axb = cfg["A"], cfg["B"], cfg["axa"], cfg["axb"]
    ta, tb = A["t"], B["t"]
    xa = [tuple(map(tuple, ta[b, list(axa)])) for b in range(ta.shape[0])]
    xb = [tuple(map(tuple, tb[b, list(axb)])) for b in range(tb.shape[0])]
    xs = sorted(set(xa) & set(xb))
    rng = np.random.default_rng(seed)
    order = rng.permutation(len(xs))
    offa = W.block_offsets(A["D"])
    offb = W.block_offsets(B["D"])
    sza = np.prod(A["D"], axis=1)
    szb = np.prod(B["D"], axis=1)
    byxa, byxb = {}, {}
    for b, x in enumerate(xa):
        byxa.setdefault(x, []).append(b)
    for b, x in enumerate(xb):
        byxb.setdefault(x, []).append(b)

    def sub(rec, idx, off, sz):
        idx = sorted(idx)
        return {"mods": rec["mods"], "sig": rec["sig"], "n": rec["n"], "t": rec["t"][idx], "D": rec["D"][idx],
                "data": np.concatenate([rec["data"][off[i]:off[i] + sz[i]] for i in idx]) if idx else np.zeros(0)}

    flops, secs, nx, npairs = 0, 0.0, 0, 0
    chunk = 8
    i = 0
    while secs < budget_s and i < len(order):
        pick = [xs[j] for j in order[i:i + chunk]]
        i += chunk
        ia = [b for x in pick for b in byxa[x]]
        ib = [b for x in pick for b in byxb[x]]
        sa, sb = sub(A, ia, offa, sza), sub(B, ib, offb, szb)
        oA, oB = O.from_record(sa), O.from_record(sb)
        t0 = time.perf_counter()
        O.tensordot(oA, oB, axa, axb)
        secs += time.perf_counter() - t0
        flops += O.useful_flops(oA, oB, axa, axb)
        nx += len(pick)
        npairs += sum(len(byxa[x]) * len(byxb[x]) for x in pick)
    desc = (f"oracle tensordot over {nx} of {len(xs)} contracted charge tuples "
            f"({npairs} block pairs, {flops:.3e} useful FLOPs), numpy with 1 BLAS thread")
    return flops, secs, desc


# ------------------------------------------------------------------ reference arm

def run_reference(args):
    _, rank, _ = rank_env()
    if rank != 0:
        return 0
    cfg = make_workload(args.workload, 0)
    times, flops_all, desc = [], [], ""
    for step in range(args.warmup + args.steps):
        f, s, desc = oracle_sample(cfg, args.ref_budget, seed=step)
        if step >= args.warmup:
            times.append(s)
            flops_all.append(f)
    tflops = sum(flops_all) / sum(times) / 1e12
    line = {
        "metric": METRIC, "value": tflops, "unit": "TFLOP/s", "impl": "reference", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * float(np.mean(times)),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": {"workload": WORKLOAD_DESC[args.workload]},
        "cpu_baseline": {"value": tflops, "unit": "TFLOP/s", "cores": 1, "kind": "oracle", "sample": desc},
        "e2e": {"value": tflops, "unit": "TFLOP/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------------ ranks

def rank_env():
    """(world size, rank, local rank) from the torchrun environment (1, 0, 0 alone)."""
    return (int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0")),
            int(os.environ.get("LOCAL_RANK", "0")))


def max_over_ranks(value, device):
    """The largest value over all ranks (a timing reduction, not a data-path one)."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    if dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def weak_value(flops_per_rank, steps, world, seconds):
    """Whole-job useful TFLOP/s: every rank contracts its own problem of the same
    size, the slowest rank's time counts."""
    return world * flops_per_rank * steps / seconds / 1e12


# ------------------------------------------------------------------ our arm

def run_ours(args):
    import torch
    import torch.distributed as dist

    from paper_2405_12196_gb300 import ytn

    world, rank, local = rank_env()
    if world > 1:
        dist.init_process_group("nccl", init_method="env://")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    PREC = {"fp64": ytn.YTN_FP64, "split": ytn.YTN_SPLIT_BF16}
    prec = PREC[args.precision]

    t_gen = time.perf_counter()
    cfg = make_workload(args.workload, rank)
    A, B, axa, axb = cfg["A"], cfg["B"], cfg["axa"], cfg["axb"]
    t_gen = time.perf_counter() - t_gen
    ctx = ytn.ytn_ctx_create(local)
    t_plan = time.perf_counter()
    plan = ytn.ytn_plan(ctx, ytn.YTN_OP_TENSORDOT, A, B, axa, axb)
    t_plan = time.perf_counter() - t_plan
    t_plan_cached = time.perf_counter()
    plan2 = ytn.ytn_plan(ctx, ytn.YTN_OP_TENSORDOT, A, B, axa, axb)
    t_plan_cached = time.perf_counter() - t_plan_cached
    assert plan2.handle == plan.handle
    flops = plan.info["useful_flops"]
    stream = torch.cuda.Stream(device=dev)
    with torch.cuda.stream(stream):
        da = torch.from_numpy(A["data"]).to(dev)
        db = torch.from_numpy(B["data"]).to(dev)
        dc = torch.empty(plan.out["size"], dtype=torch.float64, device=dev)
        ws_bytes = max(ytn.ytn_workspace_size(plan, p, args.rtol) for p in PREC.values())
        ws = torch.empty(ws_bytes, dtype=torch.uint8, device=dev)
    stream.synchronize()

    def step(p):
        return ytn.ytn_tensordot(plan, da, db, dc, prec=p, rtol=args.rtol, workspace=ws, stream=stream)

    def measure(p, steps, warmup, clocks=False):
        res = None
        for _ in range(warmup):
            res = step(p)
        stream.synchronize()
        sampler = ClockSampler(local) if clocks else None
        if sampler:
            sampler.start()
            time.sleep(0.3)
        ytn.ytn_profile_enable(ctx, True)
        ytn.ytn_profile_read(ctx)
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize(dev)
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(steps + 1)]
        ev[0].record(stream)
        for k in range(steps):
            res = step(p)
            ev[k + 1].record(stream)
        torch.cuda.synchronize(dev)
        if world > 1:
            dist.barrier()
        clk = sampler.stop() if sampler else None
        prof = ytn.ytn_profile_read(ctx)
        ytn.ytn_profile_enable(ctx, False)
        step_ms = [ev[k].elapsed_time(ev[k + 1]) for k in range(steps)]
        total_ms = max_over_ranks(ev[0].elapsed_time(ev[-1]), dev)
        return {"total_ms": total_ms, "step_ms": step_ms, "prof": prof, "res": res, "clocks": clk,
                "value": weak_value(flops, steps, world, total_ms * 1e-3)}

    peaks, peak_src = load_peaks()

    def roofline(p, m):
        gemm_calls, gemm_ms = m["prof"].get("gemm", (0, 0.0))
        kernel_ms = gemm_ms / max(1, gemm_calls)
        if p == ytn.YTN_FP64:
            kernel, kflops = "gemm_fp64_kernel", flops
            peak = peaks["bf16_tflops"] * NOMINAL["fp64"] / NOMINAL["bf16"]
            note = (f"{peak_src} dense BF16 burst ({peaks['bf16_tflops']} TFLOP/s) x nominal FP64/BF16 ratio "
                    f"{NOMINAL['fp64']}/{NOMINAL['bf16']}")
        else:
            s = m["res"]["slices"]
            kernel, kflops = "gemm_split_kernel", flops * s * (s + 1) / 2
            peak = peaks["bf16_tflops"]
            note = (f"{peak_src} dense BF16 burst; achieved counts the BF16 slice-product FLOPs "
                    f"(s(s+1)/2 = {s * (s + 1) // 2} per useful FLOP, s = {s} slices)")
        achieved = kflops / (kernel_ms * 1e-3) / 1e12 if kernel_ms > 0 else None
        return {"bound": "tensor", "kernel": kernel, "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "frac": (achieved / peak) if achieved else None, "traffic": read_traffic(kernel, args.workload),
                "kernel_ms": kernel_ms, "effective_fp64_tflops": flops / (kernel_ms * 1e-3) / 1e12 if kernel_ms else None,
                "peak_source": note}

    def phases(m):
        return {k: {"calls": v[0], "ms_per_call": v[1] / max(1, v[0])} for k, v in m["prof"].items() if k != "dropped"}

    # ---- headline precision: device-resident steps
    head = measure(prec, args.steps, args.warmup, clocks=True)
    value = head["value"]
    ph = phases(head)
    # the split GEMM writes device-resident C's blocks itself: then only A and B move
    moved_elems = plan.info["moved_elems"] - (0 if "scatter" in ph else plan.info["out_size"])
    moved_bytes = 16.0 * moved_elems
    mover_ms = sum(ph[k]["ms_per_call"] for k in ("gather_a", "gather_b", "scatter") if k in ph)
    out_head = dc.clone() if prec != ytn.YTN_FP64 else None

    # ---- the other precision, for the FP64 vs split comparison
    other = None
    if prec != ytn.YTN_FP64 and args.fp64_steps > 0:
        m64 = measure(ytn.YTN_FP64, args.fp64_steps, 1)
        diff = float(torch.linalg.vector_norm(out_head - dc) / torch.linalg.vector_norm(dc))
        other = {"precision": "fp64", "value": m64["value"], "unit": "TFLOP/s", "steps": args.fp64_steps,
                 "ms_per_step": m64["total_ms"] / args.fp64_steps, "roofline": roofline(ytn.YTN_FP64, m64),
                 "split_speedup": value / m64["value"], "split_vs_fp64_rel_frobenius": diff}
        del out_head

    # ---- end to end through the C ABI with HOST buffers: A and B are read from page-locked
    # host memory and C is written back to it by the library's data movers, every step
    ha = torch.from_numpy(A["data"]).pin_memory()
    hb = torch.from_numpy(B["data"]).pin_memory()
    hc = torch.empty(plan.out["size"], dtype=torch.float64).pin_memory()
    e2e_steps = max(1, min(args.steps, args.e2e_steps))

    def timed_e2e(body):
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize(dev)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(e2e_steps):
            body()
        e1.record(stream)
        torch.cuda.synchronize(dev)
        return weak_value(flops, e2e_steps, world, max_over_ranks(e0.elapsed_time(e1), dev) * 1e-3)

    def host_call():
        ytn.ytn_tensordot(plan, ha, hb, hc, prec=prec, rtol=args.rtol, workspace=ws, stream=stream)

    def staged_call():
        with torch.cuda.stream(stream):
            da.copy_(ha, non_blocking=True)
            db.copy_(hb, non_blocking=True)
            step(prec)
            hc.copy_(dc, non_blocking=True)

    host_call()
    e2e_serial = timed_e2e(host_call)
    e2e_staged = timed_e2e(staged_call)
    # two calls in flight on two streams (own workspace and host result buffer each):
    # a step's result travels back over the link while the next step's inputs travel in
    stream2 = torch.cuda.Stream(device=dev)
    ws2 = torch.empty_like(ws)
    hc2 = torch.empty_like(hc).pin_memory()
    k_e2e = [0]

    def pipelined_call():
        k = k_e2e[0]
        k_e2e[0] += 1
        st, w, c = (stream, ws, hc) if k % 2 == 0 else (stream2, ws2, hc2)
        ytn.ytn_tensordot(plan, ha, hb, c, prec=prec, rtol=args.rtol, workspace=w, stream=st)

    # the GEMM leaves a few SMs free, so that one call's host-link data movers run
    # beside the other call's GEMM
    reserve = 8

    def timed_pipelined():
        ytn.ytn_ctx_set_gemm_sms(ctx, torch.cuda.get_device_properties(dev).multi_processor_count - reserve)
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        for _ in range(e2e_steps):
            pipelined_call()
        torch.cuda.synchronize(dev)
        elapsed = time.perf_counter() - t0
        ytn.ytn_ctx_set_gemm_sms(ctx, 0)
        return weak_value(flops, e2e_steps, world, max_over_ranks(elapsed, dev))

    pipelined_call()
    pipelined_call()
    torch.cuda.synchronize(dev)
    e2e_direct_pipelined = timed_pipelined()
    del ws2

    # three calls in flight, each staging its host operands through its own workspace
    # with the copy engines (ytn_workspace_size_staged): one call's inputs travel in
    # and another's result travels out while a third computes on every SM
    nfly = 3
    sbytes = ytn.ytn_workspace_size_staged(plan, prec, args.rtol)
    step(prec)
    torch.cuda.synchronize(dev)
    ref_c = dc.cpu()
    del ws
    torch.cuda.empty_cache()
    s_streams = [stream] + [torch.cuda.Stream(device=dev) for _ in range(nfly - 1)]
    s_ws = [torch.empty(sbytes, dtype=torch.uint8, device=dev) for _ in range(nfly)]
    s_hc = [hc] + [torch.empty_like(hc).pin_memory() for _ in range(nfly - 1)]
    k_s = [0]

    def staged_pipelined_call():
        k = k_s[0] % nfly
        k_s[0] += 1
        ytn.ytn_tensordot(plan, ha, hb, s_hc[k], prec=prec, rtol=args.rtol, workspace=s_ws[k], stream=s_streams[k])

    for _ in range(nfly):
        staged_pipelined_call()
    torch.cuda.synchronize(dev)
    if world > 1:
        dist.barrier()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        staged_pipelined_call()
    torch.cuda.synchronize(dev)
    e2e_value = weak_value(flops, e2e_steps, world, max_over_ranks(time.perf_counter() - t0, dev))
    staged_ok = bool(torch.equal(s_hc[(k_s[0] - 1) % nfly], ref_c))
    del s_ws

    res = head["res"]
    line = {
        "metric": METRIC, "value": value, "unit": "TFLOP/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": head["total_ms"] / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": "f64" if prec == ytn.YTN_FP64 else "bf16 slices, f32 accumulate, f64 recombine",
        "data": "synthetic", "precision": args.precision,
        "config": {"workload": WORKLOAD_DESC[args.workload], "useful_flops_per_step": flops,
                   "blocks": [int(A["t"].shape[0]), int(B["t"].shape[0]), int(plan.out["t"].shape[0])],
                   "sectors": plan.info["nsectors"],
                   "max_mnk": [plan.info["max_m"], plan.info["max_n"], plan.info["max_k"]],
                   "l2": "inputs larger than L2 (no flush)",
                   "rtol": args.rtol if prec != ytn.YTN_FP64 else None},
        "latency_ms": {"p50": float(np.percentile(head["step_ms"], 50)),
                       "p99": float(np.percentile(head["step_ms"], 99))},
        "clocks": head["clocks"],
        "e2e": {"value": e2e_value, "unit": "TFLOP/s", "steps": e2e_steps,
                "h2d_bytes_per_step": int(8 * (A["data"].size + B["data"].size)),
                "d2h_bytes_per_step": int(8 * plan.out["size"]),
                "path": "ytn_tensordot on page-locked host A, B, C with a staging workspace "
                        "(ytn_workspace_size_staged): each call copies its inputs in and its result out with "
                        "the copy engines; three calls in flight on three streams",
                "staged_result_equals_device_result": staged_ok,
                "direct_pipelined_value": e2e_direct_pipelined,
                "serial_value": e2e_serial, "staged_copies_value": e2e_staged},
        # kernels of the library per timed region (the split phase launches two)
        "gpu_launches": int(sum(v["calls"] for v in ph.values()) + ph.get("split", {}).get("calls", 0)),
        "roofline": roofline(prec, head),
        "phases_ms": ph,
        "data_movers": {"bytes_per_step": moved_bytes, "ms_per_step": mover_ms,
                        "GB_per_s": moved_bytes / (mover_ms * 1e-3) / 1e9 if mover_ms else None,
                        "peak_GB_per_s": peaks["hbm_gbs"]},
        "host": {"generate_s": t_gen, "plan_s": t_plan, "plan_cached_s": t_plan_cached},
    }
    if prec != ytn.YTN_FP64:
        line["split"] = {"slices": res["slices"], "err_est": res["err_est"]}
    if other is not None:
        line["fp64"] = other
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        f, s, desc = oracle_sample(cfg, args.cpu_budget)
        line["cpu_baseline"] = {"value": f / s / 1e12, "unit": "TFLOP/s", "cores": 1, "kind": "oracle",
                                "sample": desc}
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()
    if rank == 0:
        print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------------ serving (continuous batching)

def run_serving(args):
    """Poisson stream of tensordot requests from independent U(1) iPEPS runs (D uniform
    in {4,6,8,10,12}, chi in [4D, 8D], random sector splits per run), tensors resident on
    the device, admission by an HBM budget, served by the library's continuous-batching
    server. First the saturation rate is measured (all requests at once), then the
    requests arrive as a Poisson stream at 0.8x that rate; latency = completion time -
    arrival time."""
    import torch

    from paper_2405_12196_gb300 import ytn
    dev = torch.device("cuda:0")
    prec = {"fp64": ytn.YTN_FP64, "split": ytn.YTN_SPLIT_BF16}[args.precision]
    ctx = ytn.ytn_ctx_create(0)
    runs = W.serving_runs(nruns=args.serve_runs)
    res = []
    resident = 0
    for r in runs:
        X2, a = W.serving_request(r)
        plan = ytn.ytn_plan(ctx, ytn.YTN_OP_TENSORDOT, X2, a, (1, 2), (0, 1))
        da = torch.from_numpy(X2["data"]).to(dev)
        db = torch.from_numpy(a["data"]).to(dev)
        dc = torch.empty(max(plan.out["size"], 1), dtype=torch.float64, device=dev)
        resident += 8 * (da.numel() + db.numel() + dc.numel())
        res.append({"plan": plan, "a": da, "b": db, "c": dc, "flops": plan.info["useful_flops"],
                    "D": r["D"], "chi": r["chi"]})
    budget = int(args.serve_budget_gb * 1e9)
    arena_bytes = (budget - resident) // 256 * 256
    arena = torch.empty(arena_bytes, dtype=torch.uint8, device=dev)
    rng = np.random.default_rng(4242)
    pick = rng.integers(0, len(res), size=args.serve_requests)
    total_flops = float(sum(res[i]["flops"] for i in pick))

    def serve(arrivals):
        srv = ytn.Server(ctx, args.serve_slots, arena)
        t0 = srv.now_ms()
        for k, i in enumerate(pick):
            ta = t0 + arrivals[k]
            while True:
                now = srv.now_ms()
                if now >= ta:
                    break
                if ta - now > 0.2:
                    time.sleep((ta - now - 0.1) * 1e-3)
            r = res[i]
            srv.submit(k, r["plan"], r["a"], r["b"], r["c"], prec=prec, rtol=args.rtol, t_arrive=ta)
        srv.drain(timeout_ms=600000)
        infos = srv.poll(len(pick) + 16)
        srv.close()
        assert len(infos) == len(pick) and all(x["status"] == 0 for x in infos), "request failed"
        lat = np.array([x["t_done"] - x["t_arrive"] for x in infos])
        span = max(x["t_done"] for x in infos) - min(x["t_arrive"] for x in infos)
        return lat, span

    for i in range(len(res)):   # warm every plan once
        r = res[i]
        ws = torch.empty(ytn.ytn_workspace_size(r["plan"], prec, args.rtol), dtype=torch.uint8, device=dev)
        ytn.ytn_tensordot(r["plan"], r["a"], r["b"], r["c"], prec=prec, rtol=args.rtol, workspace=ws)
        del ws
    torch.cuda.synchronize()
    lat_sat, span_sat = serve(np.zeros(len(pick)))
    rate = len(pick) / span_sat            # requests per ms at saturation
    lam = 0.8 * rate
    arrivals = np.cumsum(rng.exponential(1.0 / lam, size=len(pick)))
    lat, span = serve(arrivals)
    line = {
        "metric": "serving: block-sparse tensordot requests, p50/p99 latency and useful TFLOP/s",
        "value": total_flops / (span * 1e-3) / 1e12, "unit": "TFLOP/s", "impl": "ours", "n_gpus": 1,
        "higher_is_better": True, "precision": args.precision, "data": "synthetic",
        "config": {"workload": f"{len(pick)} requests from {len(res)} independent U(1) iPEPS runs, D in "
                               f"{{4,6,8,10,12}}, chi in [4D,8D]; X2 . a over two legs",
                   "slots": args.serve_slots, "hbm_budget_gb": args.serve_budget_gb,
                   "resident_gb": resident / 1e9, "arena_gb": arena_bytes / 1e9,
                   "requests_flops": total_flops},
        "saturation": {"requests_per_s": rate * 1e3, "tflops": total_flops / (span_sat * 1e-3) / 1e12,
                       "p50_ms": float(np.percentile(lat_sat, 50)), "p99_ms": float(np.percentile(lat_sat, 99))},
        "poisson": {"rate_per_s": lam * 1e3, "p50_ms": float(np.percentile(lat, 50)),
                    "p99_ms": float(np.percentile(lat, 99)), "mean_ms": float(lat.mean()),
                    "span_ms": span},
    }
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------------ CTM chain as one graph

def ctm_chain(ytn, ctx, dev, prec, rtol, seed=3001):
    """The contractions of one CTMRG step of the U(1)xU(1) D=12, chi=144 workload
    as one chain of library calls: A.A* over the physical leg, fuse of the ket/bra
    pairs into the double layer a, C.T, CT.T, and X2.a over two legs (X2 carries
    the conjugate fusion records of a's legs). Returns (run(stream), plans, output
    buffer of X2.a, its size, useful FLOPs per chain)."""
    import torch
    cfg = W.config3(seed=seed)
    A, C, T, X2 = cfg["A"], cfg["C"], cfg["T"], dict(cfg["X2"])
    Ac = dict(A)
    Ac["sig"] = tuple(-s for s in A["sig"])
    p_aa = ytn.ytn_plan(ctx, ytn.YTN_OP_TENSORDOT, A, Ac, (4,), (4,))
    groups = ((0, 4), (1, 5), (2, 6), (3, 7))
    p_fuse = ytn.ytn_plan(ctx, ytn.YTN_OP_FUSE, dict(p_aa.out), groups=groups)
    a = dict(p_fuse.out)
    conj = lambda f: dict(f, sig=tuple(-x for x in f["sig"]))   # noqa: E731
    X2["fus"] = [None, conj(a["fus"][0]), conj(a["fus"][1]), None]
    p_ct = ytn.ytn_plan(ctx, ytn.YTN_OP_TENSORDOT, C, T, (1,), (0,))
    p_ctt = ytn.ytn_plan(ctx, ytn.YTN_OP_TENSORDOT, dict(p_ct.out, data=None), T, (2,), (0,))
    p_x2a = ytn.ytn_plan(ctx, ytn.YTN_OP_TENSORDOT, X2, a, (1, 2), (0, 1))

    def dbuf(n):
        return torch.empty(max(int(n), 1), dtype=torch.float64, device=dev)

    buf = {k: torch.from_numpy(v["data"]).to(dev) for k, v in (("A", A), ("C", C), ("T", T), ("X2", X2))}
    buf["AA"], buf["a"] = dbuf(p_aa.out["size"]), dbuf(a["size"])
    buf["CT"], buf["CTT"], buf["X2a"] = dbuf(p_ct.out["size"]), dbuf(p_ctt.out["size"]), dbuf(p_x2a.out["size"])
    tds = [(p_aa, "A", "A", "AA"), (p_ct, "C", "T", "CT"), (p_ctt, "CT", "T", "CTT"), (p_x2a, "X2", "a", "X2a")]
    ws = {id(p): torch.empty(max(ytn.ytn_workspace_size(p, prec, rtol), 1), dtype=torch.uint8, device=dev)
          for p, *_ in tds}

    def run(stream):
        p, x, y, z = tds[0]
        ytn.ytn_tensordot(p, buf[x], buf[y], buf[z], prec=prec, rtol=rtol, workspace=ws[id(p)], stream=stream)
        ytn.ytn_fuse(p_fuse, buf["AA"], buf["a"], stream=stream)
        for p, x, y, z in tds[1:]:
            ytn.ytn_tensordot(p, buf[x], buf[y], buf[z], prec=prec, rtol=rtol, workspace=ws[id(p)],
                              stream=stream)

    flops = sum(p.info["useful_flops"] for p, *_ in tds)
    return run, [p_aa, p_fuse, p_ct, p_ctt, p_x2a], buf["X2a"], p_x2a.out["size"], flops


def run_chain(args):
    """Eager calls vs one CUDA-graph launch per chain (YTN_AUTO picks each
    contraction's path on the eager warm-up, before the capture)."""
    import torch

    from paper_2405_12196_gb300 import ytn
    dev = torch.device("cuda:0")
    ctx = ytn.ytn_ctx_create(0)
    stream = torch.cuda.Stream(device=dev)
    run, plans, out, n, flops = ctm_chain(ytn, ctx, dev, ytn.YTN_AUTO, args.rtol)
    for _ in range(args.warmup):
        run(stream)
    stream.synchronize()
    eager = out[:n].clone()

    def timed(body):
        torch.cuda.synchronize(dev)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.steps):
            body()
        e1.record(stream)
        torch.cuda.synchronize(dev)
        return e0.elapsed_time(e1) / args.steps

    ms_eager = timed(lambda: run(stream))
    ytn.ytn_graph_begin(ctx, stream)
    run(stream)
    graph = ytn.ytn_graph_end(ctx, stream)
    graph.launch(stream)
    stream.synchronize()
    same = bool(torch.equal(out[:n], eager))
    ms_graph = timed(lambda: graph.launch(stream))
    graph.close()
    line = {
        "metric": "CTMRG step chain (A.A*, fuse, C.T, CT.T, X2.a): useful TFLOP/s, eager vs one graph",
        "value": flops / (ms_graph * 1e-3) / 1e12, "unit": "TFLOP/s", "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "higher_is_better": True, "precision": "auto", "data": "synthetic",
        "config": {"workload": WORKLOAD_DESC["cfg3"] + ", chain of 4 contractions and 1 fuse",
                   "useful_flops_per_chain": flops, "rtol": args.rtol},
        "eager": {"ms_per_chain": ms_eager, "tflops": flops / (ms_eager * 1e-3) / 1e12},
        "graph": {"ms_per_chain": ms_graph, "tflops": flops / (ms_graph * 1e-3) / 1e12},
        "graph_equals_eager": same,
    }
    print(json.dumps(line), flush=True)
    return 0 if same else 1


def run_reduce(args):
    """Scalar product <X2, X2'> of two D=20 environment tensors on the same legs
    (3.36e8 common elements, 5.4 GB read per call): HBM-bound."""
    import torch

    from paper_2405_12196_gb300 import ytn
    dev = torch.device("cuda:0")
    ctx = ytn.ytn_ctx_create(0)
    A = W.config5(seed=5001)["A"]
    B = W.config5(seed=6001)["A"]
    plan = ytn.ytn_plan(ctx, ytn.YTN_OP_VDOT, A, B)
    da, db = torch.from_numpy(A["data"]).to(dev), torch.from_numpy(B["data"]).to(dev)
    out = torch.empty(1, dtype=torch.float64, device=dev)
    ws = torch.empty(max(ytn.ytn_workspace_size(plan), 1), dtype=torch.uint8, device=dev)
    stream = torch.cuda.Stream(device=dev)
    for _ in range(args.warmup):
        ytn.ytn_vdot(plan, da, db, out, workspace=ws, stream=stream)
    stream.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        ytn.ytn_vdot(plan, da, db, out, workspace=ws, stream=stream)
    e1.record(stream)
    torch.cuda.synchronize(dev)
    ms = e0.elapsed_time(e1) / args.steps
    nbytes = 16.0 * plan.info["moved_elems"]
    peaks, src = load_peaks()
    line = {
        "metric": "FP64 scalar product of two block-sparse tensors: GB/s", "value": nbytes / (ms * 1e-3) / 1e9,
        "unit": "GB/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
        "higher_is_better": True, "data": "synthetic", "dtype": "f64",
        "config": {"workload": WORKLOAD_DESC["cfg5"] + "; <X2, X2'> on the same legs",
                   "common_elements": plan.info["moved_elems"], "l2": "inputs larger than L2 (no flush)"},
        "roofline": {"bound": "hbm", "achieved": nbytes / (ms * 1e-3) / 1e9, "peak": peaks["hbm_gbs"],
                     "unit": "GB/s", "frac": nbytes / (ms * 1e-3) / 1e9 / peaks["hbm_gbs"], "traffic": None,
                     "peak_source": src},
        "result": float(out.cpu()[0]),
    }
    print(json.dumps(line), flush=True)
    return 0


def run_swap(args):
    """Fermionic swap gate on a D=20 environment tensor (3.36e8 elements, lines 0, 1
    against 2, 3), out of place: 16 bytes moved per element, HBM-bound."""
    import torch

    from paper_2405_12196_gb300 import ytn
    dev = torch.device("cuda:0")
    ctx = ytn.ytn_ctx_create(0)
    A = W.config5(seed=5001)["A"]
    plan = ytn.ytn_plan(ctx, ytn.YTN_OP_SWAP_GATE, A, groups=((0, 1), (2, 3)))
    da = torch.from_numpy(A["data"]).to(dev)
    out = torch.empty_like(da)
    stream = torch.cuda.Stream(device=dev)
    for _ in range(args.warmup):
        ytn.ytn_swap_gate(plan, da, out, stream=stream)
    stream.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        ytn.ytn_swap_gate(plan, da, out, stream=stream)
    e1.record(stream)
    torch.cuda.synchronize(dev)
    ms = e0.elapsed_time(e1) / args.steps
    nbytes = 16.0 * plan.info["moved_elems"]
    peaks, src = load_peaks()
    gbs = nbytes / (ms * 1e-3) / 1e9
    line = {
        "metric": "fermionic swap gate on a block-sparse tensor: GB/s", "value": gbs, "unit": "GB/s",
        "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
        "data": "synthetic", "dtype": "f64",
        "config": {"workload": WORKLOAD_DESC["cfg5"] + "; swap gate of legs (0, 1) against (2, 3) on X2",
                   "elements": plan.info["moved_elems"], "blocks": int(A["t"].shape[0]),
                   "l2": "inputs larger than L2 (no flush)"},
        "roofline": {"bound": "hbm", "achieved": gbs, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                     "frac": gbs / peaks["hbm_gbs"], "traffic": None, "peak_source": src},
    }
    print(json.dumps(line), flush=True)
    return 0


def run_ncon(args):
    """The enlarged corner of a U(1)xU(1) CTMRG step (C.T.T.a, D=12, chi=144) as one
    ncon network: four library calls planned once, timed per network."""
    import torch

    from paper_2405_12196_gb300 import ytn
    dev = torch.device("cuda:0")
    ctx = ytn.ytn_ctx_create(0)
    ts, labels = W.ctm_corner_network(W.config3())
    nc = ytn.ytn_ncon_plan(ctx, ts, labels)
    data = [torch.from_numpy(t["data"]).to(dev) for t in ts]
    out = torch.empty(max(nc.out["size"], 1), dtype=torch.float64, device=dev)
    stream = torch.cuda.Stream(device=dev)
    res = {}
    for name, prec, rtol in (("fp64", ytn.YTN_FP64, 0.0), ("split", ytn.YTN_SPLIT_BF16, args.rtol)):
        ws = torch.empty(max(ytn.ytn_ncon_workspace_size(nc, prec, rtol), 1), dtype=torch.uint8, device=dev)
        steps = args.steps if name == "split" else max(1, args.steps // 10)
        for _ in range(args.warmup):
            ytn.ytn_ncon(nc, data, out, prec=prec, rtol=rtol, workspace=ws, stream=stream)
        stream.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            ytn.ytn_ncon(nc, data, out, prec=prec, rtol=rtol, workspace=ws, stream=stream)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        ms = e0.elapsed_time(e1) / steps
        res[name] = {"ms_per_network": ms, "tflops": nc.info["useful_flops"] / (ms * 1e-3) / 1e12, "steps": steps}
    line = {
        "metric": "CTMRG enlarged corner as one ncon network: useful TFLOP/s", "value": res["split"]["tflops"],
        "unit": "TFLOP/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": res["split"]["ms_per_network"], "higher_is_better": True, "data": "synthetic",
        "dtype": "bf16 slices, f32 accumulate, f64 recombine",
        "config": {"workload": WORKLOAD_DESC["cfg3"] + "; ncon([C, T, T, a]) -> 4 library calls",
                   "useful_flops_per_network": nc.info["useful_flops"], "rtol": args.rtol},
        "fp64": res["fp64"], "split": res["split"],
    }
    print(json.dumps(line), flush=True)
    return 0


def run_svd(args):
    """Block-diagonal SVD of the U(1)xU(1) D=12 CTMRG enlarged corner (C.T.T.a as a
    (chi D^2) x (chi D^2) matrix: 81 sectors up to 1456 x 1456), through the
    library's gathers, the dense solver per sector and the U, S, V scatters."""
    import torch

    from paper_2405_12196_gb300 import ytn
    dev = torch.device("cuda:0")
    ctx = ytn.ytn_ctx_create(0)
    ts, labels = W.ctm_corner_network(W.config3())
    nc = ytn.ytn_ncon_plan(ctx, ts, labels)
    data = [torch.from_numpy(t["data"]).to(dev) for t in ts]
    corner = torch.empty(nc.out["size"], dtype=torch.float64, device=dev)
    ws = torch.empty(max(ytn.ytn_ncon_workspace_size(nc), 1), dtype=torch.uint8, device=dev)
    ytn.ytn_ncon(nc, data, corner, workspace=ws)
    plan = ytn.ytn_plan(ctx, ytn.YTN_OP_SVD, dict(nc.out), groups=((0, 2), (1, 3)))
    bufs = [torch.empty(max(o["size"], 1), dtype=torch.float64, device=dev) for o in plan.outs]
    sws = torch.empty(ytn.ytn_workspace_size(plan), dtype=torch.uint8, device=dev)
    stream = torch.cuda.Stream(device=dev)
    torch.cuda.synchronize(dev)
    for _ in range(args.warmup):
        ytn.ytn_svd(plan, corner, *bufs, workspace=sws, stream=stream)
    stream.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        ytn.ytn_svd(plan, corner, *bufs, workspace=sws, stream=stream)
    e1.record(stream)
    torch.cuda.synchronize(dev)
    ms = e0.elapsed_time(e1) / args.steps
    ks = plan.outs[1]["D"][:, 0]
    line = {
        "metric": "block-diagonal SVD of a CTMRG enlarged corner: ms per SVD", "value": ms, "unit": "ms",
        "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": False,
        "data": "synthetic", "dtype": "f64",
        "config": {"workload": WORKLOAD_DESC["cfg3"] + "; enlarged corner C.T.T.a, rows (chi, D^2), cols (chi, D^2)",
                   "sectors": int(len(ks)), "largest_sector": int(ks.max()), "elements": int(nc.out["size"])},
        "nominal_flops_per_svd": plan.info["useful_flops"],
        "nominal_tflops": plan.info["useful_flops"] / (ms * 1e-3) / 1e12,
    }
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="split", choices=["fp64", "split"])
    ap.add_argument("--fp64-steps", type=int, default=2)
    ap.add_argument("--rtol", type=float, default=1e-10)
    ap.add_argument("--workload", default="cfg5", choices=sorted(WORKLOAD_DESC))
    ap.add_argument("--e2e-steps", type=int, default=20)
    ap.add_argument("--cpu-budget", type=float, default=15.0)
    ap.add_argument("--ref-budget", type=float, default=8.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--serving", action="store_true", help="run the continuous-batching serving benchmark")
    ap.add_argument("--chain", action="store_true", help="time the CTMRG-step chain eager and as one CUDA graph")
    ap.add_argument("--reduce", action="store_true", help="time the FP64 scalar product of two D=20 tensors")
    ap.add_argument("--swap", action="store_true", help="time the fermionic swap gate on a D=20 tensor")
    ap.add_argument("--ncon", action="store_true", help="time the CTMRG enlarged corner as one ncon network")
    ap.add_argument("--svd", action="store_true", help="time the block-diagonal SVD of the CTMRG enlarged corner")
    ap.add_argument("--serve-runs", type=int, default=64)
    ap.add_argument("--serve-requests", type=int, default=2000)
    ap.add_argument("--serve-slots", type=int, default=8)
    ap.add_argument("--serve-budget-gb", type=float, default=120.0)
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be at least 3")
    if args.impl == "reference":
        return run_reference(args)
    if args.serving:
        return run_serving(args)
    if args.chain:
        return run_chain(args)
    if args.reduce:
        return run_reduce(args)
    if args.swap:
        return run_swap(args)
    if args.ncon:
        return run_ncon(args)
    if args.svd:
        return run_svd(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
