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

Multi-GPU (torchrun, one rank per GPU): the one contraction is shared out over the
ranks by charge sectors (ytn_plan_shard: longest-first partition of the sectors, the
largest cut by rows); A and B are replicated, every rank writes its own blocks of C,
and there is no data-path collective. value = the whole contraction's useful FLOPs /
the slowest rank's time ("scaling": "strong").
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
    if name == "cfg5r":
        return W.config5_sectors(seed=5001 + seed_shift)
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
    "cfg5r": "U(1)xU(1) iPEPS environment contraction X2.a, D=20: the blocks of a random quarter of its "
             "sectors (the full workload's block and sector sizes; profiling size)",
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


def host_cores():
    """CPU cores this process may run on."""
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


_POOL_CFG = {}


def _pool_init(meta):
    """Worker start-up: the workload's structure, and its data as views of the parent's
    shared memory (no copy)."""
    from multiprocessing import shared_memory
    cfg = {"axa": meta["axa"], "axb": meta["axb"]}
    shms = []
    for k in ("A", "B"):
        m = meta[k]
        shm = shared_memory.SharedMemory(name=m["shm"])
        shms.append(shm)
        rec = dict(m["rec"])
        rec["data"] = np.ndarray((m["n"],), dtype=np.float64, buffer=shm.buf)
        cfg[k] = rec
    _POOL_CFG["cfg"] = cfg
    _POOL_CFG["shm"] = shms


def _pool_ping(_):
    return os.getpid()


def _pool_oracle(xs):
    """Oracle tensordot over the block pairs of the given contracted charge tuples;
    returns (useful FLOPs, seconds)."""
    import oracle as O
    cfg = _POOL_CFG["cfg"]
    sa, sb = _restrict(cfg, xs)
    oA, oB = O.from_record(sa), O.from_record(sb)
    t0 = time.perf_counter()
    O.tensordot(oA, oB, cfg["axa"], cfg["axb"])
    return O.useful_flops(oA, oB, cfg["axa"], cfg["axb"]), time.perf_counter() - t0


class CpuPool:
    """Worker processes on every host core (started with spawn), sharing the workload's
    data with this process through shared memory."""

    def __init__(self, cfg):
        import concurrent.futures as cf
        import multiprocessing as mp
        from multiprocessing import shared_memory
        self.ncores = host_cores()
        self.shms = []
        meta = {"axa": cfg["axa"], "axb": cfg["axb"]}
        for k in ("A", "B"):
            rec = cfg[k]
            n = int(rec["data"].size)
            shm = shared_memory.SharedMemory(create=True, size=max(8, 8 * n))
            np.ndarray((n,), dtype=np.float64, buffer=shm.buf)[:] = rec["data"]
            self.shms.append(shm)
            meta[k] = {"shm": shm.name, "n": n, "rec": {kk: v for kk, v in rec.items() if kk != "data"}}
        self.ex = cf.ProcessPoolExecutor(max_workers=self.ncores, mp_context=mp.get_context("spawn"),
                                         initializer=_pool_init, initargs=(meta,))
        self.warm = [self.ex.submit(_pool_ping, k) for k in range(self.ncores)]

    def close(self):
        self.ex.shutdown(wait=True, cancel_futures=True)
        for shm in self.shms:
            shm.close()
            shm.unlink()


def cpu_pool(cfg):
    return CpuPool(cfg)


def _charge_index(cfg):
    """Contracted charge tuples x common to A and B, and the blocks of each."""
    A, B, axa, axb = cfg["A"], cfg["B"], cfg["axa"], cfg["axb"]
    xa = [tuple(map(tuple, A["t"][b, list(axa)])) for b in range(A["t"].shape[0])]
    xb = [tuple(map(tuple, B["t"][b, list(axb)])) for b in range(B["t"].shape[0])]
    byxa, byxb = {}, {}
    for b, x in enumerate(xa):
        byxa.setdefault(x, []).append(b)
    for b, x in enumerate(xb):
        byxb.setdefault(x, []).append(b)
    xs = sorted(set(byxa) & set(byxb))
    return xs, byxa, byxb


def _restrict(cfg, xs):
    """Sub-records of A and B holding only the blocks of the contracted tuples xs."""
    A, B = cfg["A"], cfg["B"]
    if "_index" not in cfg:
        cfg["_index"] = _charge_index(cfg)
    _, byxa, byxb = cfg["_index"]
    offa, offb = W.block_offsets(A["D"]), W.block_offsets(B["D"])
    sza, szb = np.prod(A["D"], axis=1), np.prod(B["D"], axis=1)

    def sub(rec, idx, off, sz):
        idx = sorted(idx)
        return {"mods": rec["mods"], "sig": rec["sig"], "n": rec["n"], "t": rec["t"][idx], "D": rec["D"][idx],
                "data": np.concatenate([rec["data"][off[i]:off[i] + sz[i]] for i in idx]) if idx else np.zeros(0)}
    return (sub(A, [b for x in xs for b in byxa[x]], offa, sza), sub(B, [b for x in xs for b in byxb[x]], offb, szb))


def oracle_sample_parallel(pool, cfg, budget_s):
    """The oracle on every host core: the contracted charge tuples of the workload (in
    a random order, about budget_s seconds of work per core, at most all of them) shared
    over the pool's workers in chunks; wall time of the whole batch."""
    import concurrent.futures as cf
    for f in pool.warm:
        f.result()
    xs, byxa, byxb = _charge_index(cfg)
    order = np.random.default_rng(1).permutation(len(xs))
    # calibrate: one chunk per worker, timed
    chunk = 8
    probe = [[xs[j] for j in order[k * chunk:(k + 1) * chunk]] for k in range(pool.ncores)]
    t0 = time.perf_counter()
    got = list(pool.ex.map(_pool_oracle, probe))
    t_probe = time.perf_counter() - t0
    rate = sum(f for f, _ in got) / max(t_probe, 1e-6)
    # the timed batch: chunks until about budget_s of wall time at that rate
    per_chunk = max(1.0, sum(f for f, _ in got) / len(got))
    nchunks = int(min(len(xs) // chunk - pool.ncores, max(pool.ncores, budget_s * rate / per_chunk)))
    start = pool.ncores * chunk
    tasks = [[xs[j] for j in order[start + k * chunk:start + (k + 1) * chunk]] for k in range(max(nchunks, 0))]
    tasks = [t for t in tasks if t]
    t0 = time.perf_counter()
    futs = [pool.ex.submit(_pool_oracle, t) for t in tasks]
    res = [f.result() for f in cf.as_completed(futs)]
    wall = time.perf_counter() - t0
    flops = sum(f for f, _ in res)
    ntx = sum(len(t) for t in tasks)
    return {"value": flops / wall / 1e12, "unit": "TFLOP/s", "cores": pool.ncores, "kind": "oracle",
            "seconds": wall,
            "sample": f"oracle tensordot over {ntx} of {len(xs)} contracted charge tuples ({flops:.3e} useful "
                      f"FLOPs) in chunks of {chunk} on {pool.ncores} worker processes (1 BLAS thread each)"}


def cpu_workflow(cfg, budget_s, ncores):
    """The paper's own workflow on the host cores (Sec. II.B: fuse the blocks into one
    matrix per charge sector, multiply per sector, unfuse): NumPy permutes and copies
    build A_q and B_q, torch multiplies them in FP64 on every core, and the products are
    cut back into C's blocks. Sectors from the largest down, until about budget_s."""
    import torch
    A, B, axa, axb = cfg["A"], cfg["B"], list(cfg["axa"]), list(cfg["axb"])
    freeA = [i for i in range(A["t"].shape[1]) if i not in axa]
    freeB = [i for i in range(B["t"].shape[1]) if i not in axb]
    mods = A["mods"]
    offa, offb = W.block_offsets(A["D"]), W.block_offsets(B["D"])

    def red(v):
        return tuple(int(x) % m if m else int(x) for x, m in zip(v, mods))

    # sectors: q = sum_k s_A[axa_k] x_k; rows I, columns J and contracted x per sector
    secs = {}
    for b in range(A["t"].shape[0]):
        t = A["t"][b]
        q = red(sum(int(A["sig"][a]) * t[a].astype(np.int64) for a in axa))
        s_ = secs.setdefault(q, {"rows": {}, "cols": {}, "xs": {}, "a": [], "b": []})
        I = tuple(map(tuple, t[freeA]))
        x = tuple(map(tuple, t[axa]))
        s_["rows"][I] = int(np.prod(A["D"][b][freeA])) if freeA else 1
        s_["xs"][x] = int(np.prod(A["D"][b][axa]))
        s_["a"].append(b)
    for b in range(B["t"].shape[0]):
        t = B["t"][b]
        x = tuple(map(tuple, t[axb]))
        q = red(sum(int(A["sig"][a]) * np.asarray(xk, dtype=np.int64) for a, xk in zip(axa, x)))
        if q not in secs:
            continue
        s_ = secs[q]
        J = tuple(map(tuple, t[freeB]))
        s_["cols"][J] = int(np.prod(B["D"][b][freeB])) if freeB else 1
        s_["b"].append(b)
    order = sorted(secs, key=lambda q: -2.0 * sum(secs[q]["rows"].values()) * sum(secs[q]["cols"].values())
                   * sum(secs[q]["xs"].values()))
    prev = torch.get_num_threads()
    torch.set_num_threads(ncores)
    flops, t_move, t_mm, nsec = 0.0, 0.0, 0.0, 0
    t_all = time.perf_counter()
    for q in order:
        if time.perf_counter() - t_all > budget_s:
            break
        s_ = secs[q]
        ro, co, xo = {}, {}, {}
        for d, src in ((ro, s_["rows"]), (co, s_["cols"]), (xo, s_["xs"])):
            acc = 0
            for k in sorted(src):
                d[k] = acc
                acc += src[k]
        M, N, K = sum(s_["rows"].values()), sum(s_["cols"].values()), sum(s_["xs"].values())
        t0 = time.perf_counter()
        Aq = np.zeros((M, K))
        for b in s_["a"]:
            t = A["t"][b]
            I, x = tuple(map(tuple, t[freeA])), tuple(map(tuple, t[axa]))
            if x not in xo:
                continue
            blk = A["data"][offa[b]:offa[b] + int(np.prod(A["D"][b]))].reshape(A["D"][b])
            m = blk.transpose(freeA + axa).reshape(s_["rows"][I], s_["xs"][x])
            Aq[ro[I]:ro[I] + m.shape[0], xo[x]:xo[x] + m.shape[1]] = m
        Bq = np.zeros((K, N))
        for b in s_["b"]:
            t = B["t"][b]
            J, x = tuple(map(tuple, t[freeB])), tuple(map(tuple, t[axb]))
            if x not in xo:
                continue
            blk = B["data"][offb[b]:offb[b] + int(np.prod(B["D"][b]))].reshape(B["D"][b])
            m = blk.transpose(axb + freeB).reshape(s_["xs"][x], s_["cols"][J])
            Bq[xo[x]:xo[x] + m.shape[0], co[J]:co[J] + m.shape[1]] = m
        t1 = time.perf_counter()
        Cq = torch.matmul(torch.from_numpy(Aq), torch.from_numpy(Bq)).numpy()
        t2 = time.perf_counter()
        out = {}
        for I, r0 in ro.items():
            for J, c0 in co.items():
                out[(I, J)] = Cq[r0:r0 + s_["rows"][I], c0:c0 + s_["cols"][J]].copy()
        t3 = time.perf_counter()
        t_move += (t1 - t0) + (t3 - t2)
        t_mm += t2 - t1
        flops += 2.0 * M * N * K
        nsec += 1
    wall = time.perf_counter() - t_all
    torch.set_num_threads(prev)
    return {"value": flops / wall / 1e12, "unit": "TFLOP/s", "cores": ncores, "kind": "paper workflow on CPU",
            "seconds": wall, "matmul_s": t_mm, "fuse_unfuse_s": t_move,
            "matmul_tflops": flops / max(t_mm, 1e-9) / 1e12,
            "sample": f"{nsec} of {len(secs)} charge sectors, largest first ({flops:.3e} useful FLOPs): NumPy "
                      f"fuse into A_q, B_q, torch FP64 matmul on {ncores} threads, cut into C's blocks"}


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
        "higher_is_better": True, "scaling": "strong", "vs_baseline": None, "dtype": "f64",
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


def sum_over_ranks(value, device):
    """The sum of a value over all ranks (bookkeeping of the sharded FLOPs)."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    if dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1:
        dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def strong_value(total_flops, steps, seconds):
    """Whole-job useful TFLOP/s of one contraction shared out over the ranks: its
    whole useful FLOPs per step over the slowest rank's time."""
    return total_flops * steps / seconds / 1e12


# ------------------------------------------------------------------ our arm

def measure_contraction(args, ytn, ctx, dev, cfg, world, rank, local, prec, steps, warmup, e2e_steps, fp64_steps,
                        nfly=3):
    """Time one contraction (this rank's part of it when world > 1) through the C ABI:
    the headline precision on device-resident data (CUDA events on the launching stream,
    clocks sampled meanwhile), the FP64 path beside it, and end to end with page-locked
    host A, B and C. Returns the fields of the bench line."""
    import torch
    import torch.distributed as dist

    A, B, axa, axb = cfg["A"], cfg["B"], cfg["axa"], cfg["axb"]
    shard = (rank, world) if world > 1 else None
    t_plan = time.perf_counter()
    plan = ytn.ytn_plan(ctx, ytn.YTN_OP_TENSORDOT, A, B, axa, axb, shard=shard)
    t_plan = time.perf_counter() - t_plan
    t_plan_cached = time.perf_counter()
    plan2 = ytn.ytn_plan(ctx, ytn.YTN_OP_TENSORDOT, A, B, axa, axb, shard=shard)
    t_plan_cached = time.perf_counter() - t_plan_cached
    assert plan2.handle == plan.handle
    flops = plan.info["useful_flops"]              # this rank's part
    total_flops = sum_over_ranks(flops, dev)       # the whole contraction
    stream = torch.cuda.Stream(device=dev)
    with torch.cuda.stream(stream):
        da = torch.from_numpy(A["data"]).to(dev)
        db = torch.from_numpy(B["data"]).to(dev)
        dc = torch.empty(max(plan.out["size"], 1), dtype=torch.float64, device=dev)
        ws_bytes = max(ytn.ytn_workspace_size(plan, p, args.rtol) for p in (prec, ytn.YTN_FP64))
        ws = torch.empty(ws_bytes, dtype=torch.uint8, device=dev)
    stream.synchronize()

    def step(p):
        return ytn.ytn_tensordot(plan, da, db, dc, prec=p, rtol=args.rtol, workspace=ws, stream=stream)

    def measure(p, nsteps, nwarm, clocks=False):
        res = None
        for _ in range(nwarm):
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
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(nsteps + 1)]
        ev[0].record(stream)
        for k in range(nsteps):
            res = step(p)
            ev[k + 1].record(stream)
        torch.cuda.synchronize(dev)
        if world > 1:
            dist.barrier()
        clk = sampler.stop() if sampler else None
        prof = ytn.ytn_profile_read(ctx)
        ytn.ytn_profile_enable(ctx, False)
        step_ms = [ev[k].elapsed_time(ev[k + 1]) for k in range(nsteps)]
        total_ms = max_over_ranks(ev[0].elapsed_time(ev[-1]), dev)
        return {"total_ms": total_ms, "step_ms": step_ms, "prof": prof, "res": res, "clocks": clk,
                "value": strong_value(total_flops, nsteps, total_ms * 1e-3)}

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
            s_ = m["res"]["slices"]
            kernel, kflops = "gemm_split_kernel", flops * s_ * (s_ + 1) / 2
            peak = peaks["bf16_tflops"]
            note = (f"{peak_src} dense BF16 burst; achieved counts the BF16 slice-product FLOPs "
                    f"(s(s+1)/2 = {s_ * (s_ + 1) // 2} per useful FLOP, s = {s_} slices)")
        achieved = kflops / (kernel_ms * 1e-3) / 1e12 if kernel_ms > 0 else None
        return {"bound": "tensor", "kernel": kernel, "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "frac": (achieved / peak) if achieved else None, "traffic": read_traffic(kernel, args.workload),
                "kernel_ms": kernel_ms,
                "effective_fp64_tflops": flops / (kernel_ms * 1e-3) / 1e12 if kernel_ms else None,
                "peak_source": note}

    def phases(m):
        return {k: {"calls": v[0], "ms_per_call": v[1] / max(1, v[0])} for k, v in m["prof"].items() if k != "dropped"}

    # ---- headline precision: device-resident steps
    head = measure(prec, steps, warmup, clocks=True)
    ph = phases(head)
    # the fused split path reads A's and B's blocks in its slicing kernel (the split
    # phase): then only the scatter of C is a data mover of its own
    moved_elems = plan.info["moved_elems"] if "gather_a" in ph else plan.info["out_size"]
    moved_bytes = 16.0 * moved_elems
    mover_ms = sum(ph[k]["ms_per_call"] for k in ("gather_a", "gather_b", "scatter") if k in ph)
    out_head = dc.clone() if prec != ytn.YTN_FP64 else None
    # the data-aware accuracy record of the last timed split call (the device's own
    # estimate of its relative error, and the sectors it recomputed in FP64)
    report = ytn.ytn_tensordot_report(plan, ws, stream) if prec != ytn.YTN_FP64 else None

    # ---- the other precision, for the FP64 vs split comparison
    other = None
    if prec != ytn.YTN_FP64 and fp64_steps > 0:
        m64 = measure(ytn.YTN_FP64, fp64_steps, 1)
        diff = float(torch.linalg.vector_norm(out_head - dc) / torch.linalg.vector_norm(dc))
        other = {"precision": "fp64", "value": m64["value"], "unit": "TFLOP/s", "steps": fp64_steps,
                 "ms_per_step": m64["total_ms"] / fp64_steps, "roofline": roofline(ytn.YTN_FP64, m64),
                 "split_speedup": head["value"] / m64["value"], "split_vs_fp64_rel_frobenius": diff}
    del out_head

    # ---- end to end through the C ABI with HOST buffers: A and B are read from page-locked
    # host memory and C is written back to it, every step
    ha = torch.from_numpy(A["data"]).pin_memory()
    hb = torch.from_numpy(B["data"]).pin_memory()
    hc = torch.empty(max(plan.out["size"], 1), dtype=torch.float64).pin_memory()
    e2e = {}
    if e2e_steps > 0:
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
            return strong_value(total_flops, e2e_steps, max_over_ranks(e0.elapsed_time(e1), dev) * 1e-3)

        def host_call():
            ytn.ytn_tensordot(plan, ha, hb, hc, prec=prec, rtol=args.rtol, workspace=ws, stream=stream)

        def staged_call():
            with torch.cuda.stream(stream):
                da.copy_(ha, non_blocking=True)
                db.copy_(hb, non_blocking=True)
                step(prec)
                hc.copy_(dc, non_blocking=True)

        host_call()
        e2e["serial_value"] = timed_e2e(host_call)
        e2e["staged_copies_value"] = timed_e2e(staged_call)
        if nfly >= 3:
            # two calls in flight on two streams (own workspace and host result buffer each),
            # the data movers reading host memory; the GEMM leaves a few SMs free, so that one
            # call's host-link data movers run beside the other call's GEMM
            stream2 = torch.cuda.Stream(device=dev)
            ws2 = torch.empty_like(ws)
            hc2 = torch.empty_like(hc).pin_memory()
            k_e2e = [0]

            def pipelined_call():
                k = k_e2e[0]
                k_e2e[0] += 1
                st, w, c = (stream, ws, hc) if k % 2 == 0 else (stream2, ws2, hc2)
                ytn.ytn_tensordot(plan, ha, hb, c, prec=prec, rtol=args.rtol, workspace=w, stream=st)

            reserve = 8
            pipelined_call()
            pipelined_call()
            torch.cuda.synchronize(dev)
            ytn.ytn_ctx_set_gemm_sms(ctx, torch.cuda.get_device_properties(dev).multi_processor_count - reserve)
            if world > 1:
                dist.barrier()
            torch.cuda.synchronize(dev)
            t0 = time.perf_counter()
            for _ in range(e2e_steps):
                pipelined_call()
            torch.cuda.synchronize(dev)
            e2e["direct_pipelined_value"] = strong_value(total_flops, e2e_steps,
                                                         max_over_ranks(time.perf_counter() - t0, dev))
            ytn.ytn_ctx_set_gemm_sms(ctx, 0)
            del ws2, hc2
        # nfly calls in flight, each staging its host operands through its own workspace
        # with the copy engines (ytn_workspace_size_staged): one call's inputs travel in
        # and another's result travels out while a third computes on every SM
        sbytes = ytn.ytn_workspace_size_staged(plan, prec, args.rtol)
        step(prec)
        torch.cuda.synchronize(dev)
        ref_c = dc.cpu()
        del ws, da, db, dc
        torch.cuda.empty_cache()
        s_streams = [stream] + [torch.cuda.Stream(device=dev) for _ in range(nfly - 1)]
        s_ws = [torch.empty(sbytes, dtype=torch.uint8, device=dev) for _ in range(nfly)]
        s_hc = [hc] + [torch.empty_like(hc).pin_memory() for _ in range(nfly - 1)]
        k_s = [0]

        def staged_pipelined_call():
            k = k_s[0] % nfly
            k_s[0] += 1
            ytn.ytn_tensordot(plan, ha, hb, s_hc[k], prec=prec, rtol=args.rtol, workspace=s_ws[k],
                              stream=s_streams[k])

        for _ in range(nfly):
            staged_pipelined_call()
        torch.cuda.synchronize(dev)
        if world > 1:
            dist.barrier()
        # the host link's bandwidth varies from box to box and from run to run (the
        # page-locked buffers' placement, other jobs on the host): the median of three
        # timed runs, every run reported
        e2e_runs = []
        for _ in range(3):
            if world > 1:
                dist.barrier()
            torch.cuda.synchronize(dev)
            t0 = time.perf_counter()
            for _ in range(e2e_steps):
                staged_pipelined_call()
            torch.cuda.synchronize(dev)
            e2e_runs.append(strong_value(total_flops, e2e_steps, max_over_ranks(time.perf_counter() - t0, dev)))
        e2e_value = float(np.median(e2e_runs))
        staged_ok = bool(torch.equal(s_hc[(k_s[0] - 1) % nfly], ref_c))
        hbm_reserved = nfly * sbytes
        del s_ws
        e2e = {"value": e2e_value, "unit": "TFLOP/s", "steps": e2e_steps,
               "h2d_bytes_per_step": int(world * 8 * (A["data"].size + B["data"].size)),
               "d2h_bytes_per_step": int(sum_over_ranks(8 * plan.out["size"], dev)),
               "path": "ytn_tensordot on page-locked host A, B, C with a staging workspace "
                       f"(ytn_workspace_size_staged): each call copies its inputs in and its result out with "
                       f"the copy engines; {nfly} calls in flight on {nfly} streams",
               "runs": e2e_runs, "hbm_reserved_bytes": int(hbm_reserved),
               "staged_result_equals_device_result": staged_ok, **e2e}
    else:
        del ws, da, db, dc
    torch.cuda.empty_cache()

    res = head["res"]
    out = {
        "value": head["value"], "ms_per_step": head["total_ms"] / steps, "total_flops": total_flops,
        "plan": plan, "head": head, "phases": ph, "roofline": roofline(prec, head), "e2e": e2e,
        "latency_ms": {"p50": float(np.percentile(head["step_ms"], 50)),
                       "p99": float(np.percentile(head["step_ms"], 99))},
        "data_movers": {"bytes_per_step": moved_bytes, "ms_per_step": mover_ms,
                        "GB_per_s": moved_bytes / (mover_ms * 1e-3) / 1e9 if mover_ms else None,
                        "peak_GB_per_s": peaks["hbm_gbs"]},
        "host": {"plan_s": t_plan, "plan_cached_s": t_plan_cached},
        "fp64": other,
    }
    if prec != ytn.YTN_FP64:
        out["split"] = {"slices": res["slices"],
                        "variant": {2: "fused and pipelined: slices straight from the blocks, each sector "
                                       "group's slicing beside the previous group's GEMM",
                                    1: "fused: slices straight from the blocks",
                                    0: "staged: FP64 sector matrices gathered first"}.get(res["split_variant"]),
                        "pipe_groups": plan.info["split_pipe_groups"],
                        "narrow_sector_tails": bool(res.get("narrow_tiles", 0)),
                        "a_priori_err_est": res["err_est"],
                        "err_est": report["err_est"], "split_err_est": report["split_err_est"],
                        "max_sector_est": report["max_sector_est"], "fp64_fallback_sectors": report["nfallback"],
                        "fp64_fallback_flops": report["fallback_flops"]}
        # the autotuner's record for this slice count: the candidates' times on the
        # plan's first call (ms, fastest of its rounds; 0 where not timed)
        tun = ytn.ytn_plan_tuning(plan, res["slices"])
        out["split"]["tuning_ms"] = {k: tun[k] for k in ("staged_ms", "fused_ms", "pipelined_ms", "wide_ms",
                                                         "narrow_ms")}
    return out


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
    if args.precision not in PREC:
        raise SystemExit("--precision auto applies to --serving only")
    prec = PREC[args.precision]
    extras = rank == 0 and world == 1 and not args.no_extras and args.workload == "cfg5"

    t_gen = time.perf_counter()
    cfg = make_workload(args.workload, 0)    # one problem, shared out over the ranks
    A, B = cfg["A"], cfg["B"]
    t_gen = time.perf_counter() - t_gen
    ctx = ytn.ytn_ctx_create(local)
    m = measure_contraction(args, ytn, ctx, dev, cfg, world, rank, local, prec, args.steps, args.warmup,
                            max(1, min(args.steps, args.e2e_steps)), args.fp64_steps)
    plan, ph = m["plan"], m["phases"]
    line = {
        "metric": METRIC, "value": m["value"], "unit": "TFLOP/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": m["ms_per_step"], "higher_is_better": True,
        "scaling": "strong", "vs_baseline": None,
        "dtype": "f64" if prec == ytn.YTN_FP64 else "bf16 slices, f32 accumulate, f64 recombine",
        "data": "synthetic", "precision": args.precision,
        "config": {"workload": WORKLOAD_DESC[args.workload], "useful_flops_per_step": m["total_flops"],
                   "parallelism": f"sector-sharded x{world}" if world > 1 else "one GPU",
                   "blocks": [int(A["t"].shape[0]), int(B["t"].shape[0]), int(plan.out["t"].shape[0])],
                   "sectors": plan.info["nsectors"],
                   "max_mnk": [plan.info["max_m"], plan.info["max_n"], plan.info["max_k"]],
                   "l2": "inputs larger than L2 (no flush)",
                   "rtol": args.rtol if prec != ytn.YTN_FP64 else None},
        "latency_ms": m["latency_ms"],
        "clocks": m["head"]["clocks"],
        "e2e": m["e2e"],
        # kernels of the library per timed region: one per phase call, plus the second
        # kernel of the split phase (exponents and slices, or row maxima and digits)
        # and the rest of the check phase (the FP64 recomputation; on the fused path
        # also the gathers of the recomputed sectors, two launches; the workloads here
        # have every block of a sector, so no zero fill); the pipelined variant adds,
        # inside its GEMM phase, one GEMM and two slicing launches per further group
        "gpu_launches": int(sum(v["calls"] for v in ph.values()) + ph.get("split", {}).get("calls", 0)
                            + ph.get("check", {}).get("calls", 0)
                            * (3 if m["head"]["res"].get("split_variant") in (1, 2) else 1)
                            + (ph.get("gemm", {}).get("calls", 0) * 3 * (m["split"]["pipe_groups"] - 1)
                               if m["head"]["res"].get("split_variant") == 2 else 0)),
        "roofline": m["roofline"],
        "phases_ms": ph,
        "data_movers": m["data_movers"],
        "host": dict(m["host"], generate_s=t_gen),
    }
    if "split" in m:
        line["split"] = m["split"]
    if m["fp64"] is not None:
        line["fp64"] = m["fp64"]
    del m, plan
    if extras:
        line["cfg5b"] = extra_cfg5b(args, ytn, ctx, dev, prec)
        line["serving"] = serving_summary(args, ytn, ctx, dev, prec, nruns=args.extra_serve_runs,
                                          nrequests=args.extra_serve_requests)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        f, s, desc = oracle_sample(cfg, args.cpu_budget)
        line["cpu_baseline"] = {"value": f / s / 1e12, "unit": "TFLOP/s", "cores": 1, "kind": "oracle",
                                "sample": desc}
        if not args.no_extras:
            pool = cpu_pool(cfg)
            try:
                line["cpu_baseline"]["all_cores"] = oracle_sample_parallel(pool, cfg, args.cpu_budget)
            finally:
                pool.close()
            line["cpu_workflow"] = cpu_workflow(cfg, args.cpu_budget, host_cores())
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()
    if rank == 0:
        print(json.dumps(line), flush=True)
    return 0


def extra_cfg5b(args, ytn, ctx, dev, prec):
    """The 25-sector reading of the large workload (D = 20 over 9 charges, 81 sectors up
    to 11388^3), a few steps: value, roofline and e2e on the same clock as the headline."""
    cfg = make_workload("cfg5b", 0)
    m = measure_contraction(args, ytn, ctx, dev, cfg, 1, 0, 0, prec, args.extra_steps, 3, args.extra_steps, 0,
                            nfly=2)
    out = {"workload": WORKLOAD_DESC["cfg5b"], "useful_flops_per_step": m["total_flops"], "value": m["value"],
           "unit": "TFLOP/s", "steps": args.extra_steps, "warmup": 3, "ms_per_step": m["ms_per_step"],
           "sectors": m["plan"].info["nsectors"],
           "max_mnk": [m["plan"].info["max_m"], m["plan"].info["max_n"], m["plan"].info["max_k"]],
           "clocks": m["head"]["clocks"], "roofline": m["roofline"], "e2e": m["e2e"], "phases_ms": m["phases"]}
    if "split" in m:
        out["split"] = m["split"]
    return out


# ------------------------------------------------------------------ serving (continuous batching)

def serving_summary(args, ytn, ctx, dev, prec, nruns, nrequests, slots=None, budget_gb=None):
    """Poisson stream of tensordot requests from independent U(1) iPEPS runs (D uniform
    in {4,6,8,10,12}, chi in [4D, 8D], random sector splits per run), tensors resident on
    the device, admission by an HBM budget, served by the library's continuous-batching
    server. First the saturation rate is measured (all requests at once), then the
    requests arrive as a Poisson stream at 0.8x that rate; latency = completion time -
    arrival time. Returns the summary fields."""
    import torch
    slots = slots or args.serve_slots
    budget_gb = budget_gb or args.serve_budget_gb
    runs = W.serving_runs(nruns=nruns)
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
    budget = int(budget_gb * 1e9)
    arena_bytes = (budget - resident) // 256 * 256
    arena = torch.empty(arena_bytes, dtype=torch.uint8, device=dev)
    rng = np.random.default_rng(4242)
    pick = rng.integers(0, len(res), size=nrequests)
    total_flops = float(sum(res[i]["flops"] for i in pick))

    def serve(arrivals):
        srv = ytn.Server(ctx, slots, arena)
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
    out = {
        "workload": f"{len(pick)} requests from {len(res)} independent U(1) iPEPS runs, D in {{4,6,8,10,12}}, "
                    f"chi in [4D,8D]; X2 . a over two legs",
        "precision": args.precision, "requests": len(pick), "slots": slots, "hbm_budget_gb": budget_gb,
        "resident_gb": resident / 1e9, "arena_gb": arena_bytes / 1e9, "requests_flops": total_flops,
        "value": total_flops / (span * 1e-3) / 1e12, "unit": "TFLOP/s",
        "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
        "saturation": {"requests_per_s": rate * 1e3, "tflops": total_flops / (span_sat * 1e-3) / 1e12,
                       "p50_ms": float(np.percentile(lat_sat, 50)), "p99_ms": float(np.percentile(lat_sat, 99))},
        "poisson": {"rate_per_s": lam * 1e3, "p50_ms": float(np.percentile(lat, 50)),
                    "p99_ms": float(np.percentile(lat, 99)), "mean_ms": float(lat.mean()), "span_ms": span},
    }
    del res, arena
    torch.cuda.empty_cache()
    return out


def run_serving(args):
    import torch

    from paper_2405_12196_gb300 import ytn
    dev = torch.device("cuda:0")
    prec = {"fp64": ytn.YTN_FP64, "split": ytn.YTN_SPLIT_BF16, "auto": ytn.YTN_AUTO}[args.precision]
    ctx = ytn.ytn_ctx_create(0)
    sm = serving_summary(args, ytn, ctx, dev, prec, args.serve_runs, args.serve_requests)
    line = {
        "metric": "serving: block-sparse tensordot requests, p50/p99 latency and useful TFLOP/s",
        "value": sm["value"], "unit": "TFLOP/s", "impl": "ours", "n_gpus": 1,
        "higher_is_better": True, "precision": args.precision, "data": "synthetic",
        "config": {k: sm[k] for k in ("workload", "slots", "hbm_budget_gb", "resident_gb", "arena_gb",
                                      "requests_flops")},
        "saturation": sm["saturation"], "poisson": sm["poisson"],
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
    ap.add_argument("--precision", default="split", choices=["fp64", "split", "auto"])
    ap.add_argument("--fp64-steps", type=int, default=2)
    ap.add_argument("--rtol", type=float, default=1e-10)
    ap.add_argument("--workload", default="cfg5", choices=sorted(WORKLOAD_DESC))
    ap.add_argument("--e2e-steps", type=int, default=20)
    ap.add_argument("--cpu-budget", type=float, default=15.0)
    ap.add_argument("--ref-budget", type=float, default=8.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the 25-sector workload and the serving stream of the default line")
    ap.add_argument("--extra-steps", type=int, default=5, help="timed steps of the 25-sector workload")
    ap.add_argument("--extra-serve-runs", type=int, default=32)
    ap.add_argument("--extra-serve-requests", type=int, default=600)
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
