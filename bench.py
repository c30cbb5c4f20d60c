"""Benchmark: NESA matrix-vector products per second on the r = 3 sphere workload.

Workload: PEC sphere of radius 3 wavelengths, icosphere subdivision 6 (81,920
triangles, 122,880 RWG unknowns), octree of 6 levels with 0.25-wavelength leaves,
one right-hand side.  One step = one full operator application (near field +
radiation, source transfer, translation, potential transfer, reception) through the
library's C ABI.

``value`` is the rate of the FP64 product (the paper's arithmetic: complex128 operator,
FP64 kernels).  The mixed-precision product (tensor-core BF16 hi/lo translations,
complex64 elsewhere; its error against the FP64 product is measured and reported) is
timed beside it (``mixed``), and GMRES solves to 1e-5 are timed for both: the plain
FP64 solve and FP64 iterative refinement around the mixed product (``solve``).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line on rank 0.  ``--impl reference`` times the CPU oracle instead, on
all host cores: each step is a stage-wise sample of one product (see
``oracle_sampled_product``) spread over a process pool.  Under torchrun (N > 1) every
rank runs an independent replica of the workload (the product of one operator does not
shard without a halo exchange, which is not built); ``value`` counts the products of
all ranks.
"""
import os

os.environ.setdefault("OPENBLAS_NUM_THREADS", "1")
os.environ.setdefault("OMP_NUM_THREADS", "1")
os.environ.setdefault("MKL_NUM_THREADS", "1")

import argparse  # noqa: E402
import json  # noqa: E402
import subprocess  # noqa: E402
import sys  # noqa: E402
import threading  # noqa: E402
import time  # noqa: E402

import numpy as np  # noqa: E402

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from workloads import get_config, plane_wave_directions, random_coefficients  # noqa: E402

CONFIG = "C2"
METRIC = "nesa_matvec_per_s"
UNIT = "matvec/s"
# GB300: 152 SMs at 2070 MHz; per SM and clock 2 FP64 FMA and 128 FP32 FMA
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.070e9 / 1e12
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.070e9 / 1e12
# DRAM traffic of the translation / potential-transfer GEMM launches of one product of
# the r = 3 sphere (ncu, dram__bytes_read.sum + dram__bytes_write.sum); null elsewhere
GEMM_DRAM_BYTES_C2 = 1.5083e9
# DRAM traffic of the FP64 translation launches (k_translate64) of one product of
# the r = 3 sphere (ncu: dram__bytes_read.sum + dram__bytes_write.sum of the 4 launches of one
# product, captured on the current kernel with `--profile-run fp64_C2`)
K_TRANSLATE64_DRAM_BYTES_C2 = 21.7700e9
SPEC = ("PEC sphere r=3 wavelengths, icosphere subdiv 6 (81,920 triangles, 122,880 RWG), "
        "6-level octree, leaf 0.25 wavelength, 1 RHS")


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except OSError:
        return {}


class ClockSampler:
    """nvidia-smi samples (every 200 ms) while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None
        time.sleep(0.3)
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc is not None:
            time.sleep(0.25)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for name, val in zip(names, f[5:9]):
                if val.lower() == "active":
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"], "samples": 0}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


class Ranks:
    """Barrier and max-over-ranks for the timing (no process group with one rank).
    backend "nccl" on the GPUs for the benchmark; "gloo" on the host for tests."""

    def __init__(self, world, backend="nccl", device="cuda"):
        import torch
        self.device = torch.device(device)
        self.pg = None
        if world > 1:
            import torch.distributed as dist
            if backend == "nccl":
                dist.init_process_group(backend, device_id=self.device)
            else:
                dist.init_process_group(backend)
            self.pg = dist

    def barrier(self):
        if self.pg is not None:
            self.pg.barrier()

    def max(self, v):
        import torch
        t = torch.tensor([float(v)], dtype=torch.float64, device=self.device)
        if self.pg is not None:
            self.pg.all_reduce(t, op=self.pg.ReduceOp.MAX)
        return float(t.item())

    def close(self):
        if self.pg is not None:
            self.pg.destroy_process_group()
            self.pg = None


def job_throughput(world, units_per_rank_step, ms_per_step_max):
    """Whole-job units per second: every rank processes units_per_rank_step per step,
    the step time is the slowest rank's."""
    return world * units_per_rank_step * 1e3 / ms_per_step_max


def oracle_sampled_product(o, x, n_leaves=12, n_boxes=12, n_rows=48, seed=0):
    """Seconds the oracle needs for one full product, estimated stage by stage on a
    bounded sample: every stage (channel sources, near rows, radiation, source
    transfer, translation per level, reception, testing) is timed on a random subset
    of its units (leaves, boxes or rows) and scaled by the number of units.  Inputs of
    the sampled stages are the true ones where cheap, else random vectors of the right
    shape (the cost of a stage does not depend on the values)."""
    rng = np.random.default_rng(seed)
    t = o.tree
    L, l0 = o.L, o.l0
    parts = {}

    def pick(seq, k):
        seq = list(seq)
        idx = rng.choice(len(seq), size=min(k, len(seq)), replace=False)
        return [seq[i] for i in idx]

    t0 = time.perf_counter()
    J = o.sources(x)
    parts["sources"] = time.perf_counter() - t0
    rows = np.sort(rng.choice(o.n, size=min(n_rows, o.n), replace=False))
    t0 = time.perf_counter()
    _ = o.near_rows(rows) @ x
    parts["near"] = (time.perf_counter() - t0) * o.n / len(rows)
    leaves = t.boxes[L]
    sample = pick(leaves, n_leaves)
    t0 = time.perf_counter()
    for b in sample:
        o.radiate(J, b)
    parts["radiation"] = (time.perf_counter() - t0) * len(leaves) / len(sample)
    up = 0.0
    for l in range(L, l0, -1):
        sample = pick(t.boxes[l], n_boxes)
        s = rng.standard_normal((o.Q[l], 4)) + 0j
        t0 = time.perf_counter()
        for b in sample:
            o.source_transfer(l, b, s)
        up += (time.perf_counter() - t0) * len(t.boxes[l]) / len(sample)
    parts["source_transfer"] = up
    tr = 0.0
    for l in range(l0, L + 1):
        sample = pick(t.boxes[l], n_boxes)
        srcs = {b for a in sample for b in t.interaction_list(l, a)}
        s = {b: rng.standard_normal((o.Q[l], 4)) + 0j for b in srcs}
        op = rng.standard_normal((o.Q[l - 1], 4)) + 0j if l > l0 else None
        o._D = {}
        t0 = time.perf_counter()
        for a in sample:
            o.translate(l, a, s, op)
        tr += (time.perf_counter() - t0) * len(t.boxes[l]) / len(sample)
        o._D = {}
    parts["translation"] = tr
    sample = pick(leaves, n_leaves)
    oL = rng.standard_normal((o.Q[L], 4)) + 0j
    t0 = time.perf_counter()
    for b in sample:
        o.receive(b, oL)
    parts["reception"] = (time.perf_counter() - t0) * len(leaves) / len(sample)
    F = np.zeros((len(t.points), 4), np.complex128)
    t0 = time.perf_counter()
    o.test(F, rows)
    parts["testing"] = (time.perf_counter() - t0) * o.n / len(rows)
    total = sum(parts.values())
    desc = ("stage-wise sample of one product: %d of %d leaves (radiation, reception), %d boxes per level "
            "(source transfer, translation with D built on the fly), %d of %d rows (near field, testing); "
            "each stage scaled by its unit count" % (min(n_leaves, len(leaves)), len(leaves), n_boxes,
                                                   len(rows), o.n))
    return total, parts, desc


# ------------------------------------------------------------------ all-core oracle timing
# Worker processes (spawned, so that no CUDA state is inherited) each build the oracle
# once; a sampled stage then runs as one task per worker, every task the size of the
# single-core sample (like the paper's OpenMP/SuperGlue tasks, Sec. 5.3, one unit group
# per task), and the stage's wall time is scaled by its unit count.
_W = {}


def _pool_init(cfg_name, seed):
    os.environ["OPENBLAS_NUM_THREADS"] = "1"
    o = build_oracle(get_config(cfg_name))
    x = random_coefficients(o.n, 1, seed=seed)[0]
    _W.update(o=o, x=x, J=o.sources(x))


def _pool_task(task):
    o, kind = _W["o"], task[0]
    rng = np.random.default_rng(task[-1])
    if kind == "near":
        _ = o.near_rows(task[1]) @ _W["x"]
    elif kind == "radiation":
        for b in task[1]:
            o.radiate(_W["J"], b)
    elif kind == "source_transfer":
        s = rng.standard_normal((o.Q[task[1]], 4)) + 0j
        for b in task[2]:
            o.source_transfer(task[1], b, s)
    elif kind == "translation":
        l, boxes = task[1], task[2]
        srcs = {b for a in boxes for b in o.tree.interaction_list(l, a)}
        s = {b: rng.standard_normal((o.Q[l], 4)) + 0j for b in srcs}
        op = rng.standard_normal((o.Q[l - 1], 4)) + 0j if l > o.l0 else None
        o._D = {}
        for a in boxes:
            o.translate(l, a, s, op)
        o._D = {}
    elif kind == "reception":
        oL = rng.standard_normal((o.Q[o.L], 4)) + 0j
        for b in task[1]:
            o.receive(b, oL)
    elif kind == "testing":
        F = np.zeros((len(o.tree.points), 4), np.complex128)
        o.test(F, task[1])
    return 0


class OraclePool:
    """A spawned process pool of `procs` workers, each holding the oracle of one workload."""

    def __init__(self, cfg_name, procs, seed=2024):
        import multiprocessing as mp
        self.procs = procs
        self.pool = mp.get_context("spawn").Pool(procs, initializer=_pool_init, initargs=(cfg_name, seed))
        self.pool.map(_pool_task, [("near", [0], i) for i in range(procs)])  # every worker is up

    def close(self):
        self.pool.terminate()
        self.pool.join()

    def sampled_product(self, o, n_leaves=12, n_boxes=12, n_rows=48, seed=0):
        """As oracle_sampled_product, with every stage's sample multiplied by the number of
        workers and run as one task per worker.  The channel sources (one pass over the
        triangles, under 1 % of the product) are timed on one core."""
        P = self.procs
        rng = np.random.default_rng(seed)
        t = o.tree
        L, l0 = o.L, o.l0
        parts = {}

        def run(tasks):
            t0 = time.perf_counter()
            self.pool.map(_pool_task, tasks, chunksize=1)
            return time.perf_counter() - t0

        def groups(seq, k):
            seq = list(seq)
            idx = rng.choice(len(seq), size=min(k * P, len(seq)), replace=False)
            picked = [seq[i] for i in idx]
            return [picked[i::P] for i in range(P) if picked[i::P]], len(picked)

        t0 = time.perf_counter()
        o.sources(random_coefficients(o.n, 1, seed=seed)[0])
        parts["sources"] = time.perf_counter() - t0
        rows = np.sort(rng.choice(o.n, size=min(n_rows * P, o.n), replace=False))
        chunks = [rows[i::P] for i in range(P)]
        parts["near"] = run([("near", c, i) for i, c in enumerate(chunks)]) * o.n / len(rows)
        g, m = groups(t.boxes[L], n_leaves)
        parts["radiation"] = run([("radiation", c, i) for i, c in enumerate(g)]) * len(t.boxes[L]) / m
        up = 0.0
        for l in range(L, l0, -1):
            g, m = groups(t.boxes[l], n_boxes)
            up += run([("source_transfer", l, c, i) for i, c in enumerate(g)]) * len(t.boxes[l]) / m
        parts["source_transfer"] = up
        tr = 0.0
        for l in range(l0, L + 1):
            g, m = groups(t.boxes[l], n_boxes)
            tr += run([("translation", l, c, i) for i, c in enumerate(g)]) * len(t.boxes[l]) / m
        parts["translation"] = tr
        g, m = groups(t.boxes[L], n_leaves)
        parts["reception"] = run([("reception", c, i) for i, c in enumerate(g)]) * len(t.boxes[L]) / m
        parts["testing"] = run([("testing", c, i) for i, c in enumerate(chunks)]) * o.n / len(rows)
        desc = ("stage-wise sample of one product on %d worker processes (one task per worker, each the size of "
                "the single-core sample: %d leaves, %d boxes per level, %d rows); each stage's wall time scaled by "
                "its unit count; channel sources on one core" % (P, n_leaves, n_boxes, n_rows))
        return sum(parts.values()), parts, desc


def host_cores():
    """Cores this process may run on (its affinity mask; os.cpu_count() counts the whole host)."""
    try:
        return max(1, len(os.sched_getaffinity(0)))
    except (AttributeError, OSError):
        return os.cpu_count() or 1


def build_oracle(cfg):
    from oracle.nesa import NesaOracle
    return NesaOracle(cfg["vertices"], cfg["triangles"], cfg["k"], cfg["leaf_size"], cfg["n_levels"])


def run_reference(args, world, rank):
    """The oracle, as it stands, on all host cores (rank 0 only)."""
    if rank != 0:
        return 0
    cfg = get_config(CONFIG)
    o = build_oracle(cfg)
    procs = host_cores()
    pool = OraclePool(CONFIG, procs)
    try:
        for _ in range(args.warmup):
            pool.sampled_product(o, seed=1)
        est, walls = [], []
        for s in range(args.steps):
            t0 = time.perf_counter()
            sec, parts, desc = pool.sampled_product(o, seed=100 + s)
            walls.append(time.perf_counter() - t0)
            est.append(sec)
    finally:
        pool.close()
    value = 1.0 / float(np.mean(est))
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * float(np.mean(walls)), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
        "config": {"workload": "%s: %s" % (CONFIG, SPEC), "parallelism": "%d host processes" % procs},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": procs, "kind": "oracle", "sample": desc,
                         "host_cpu_count": os.cpu_count()},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


def _time_products(g, x, y, parts, steps, warmup, stream, barrier):
    import torch
    with torch.cuda.stream(stream):
        for _ in range(max(3, warmup)):
            g.matvec(x, y, parts=parts)
    stream.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier()
    torch.cuda.synchronize()
    with torch.cuda.stream(stream):
        ev0.record(stream)
        for _ in range(steps):
            g.matvec(x, y, parts=parts)
        ev1.record(stream)
    stream.synchronize()
    torch.cuda.synchronize()
    barrier()
    # stage split: a second pass of the same products with per-stage events
    g.profile_enable(True)
    with torch.cuda.stream(stream):
        for _ in range(steps):
            g.matvec(x, y, parts=parts)
    stream.synchronize()
    prof = g.profile_read()
    g.profile_enable(False)
    return ev0.elapsed_time(ev1) / steps, prof


# the paper's CPU timings of the complete 2D product at N = 100,000 (Sec. 5, Tables 3
# and 7): context for the 2D block, other hardware
MODEL2D_PAPER_MS = {(300, 100): {"1 core (Table 3)": 1192.0, "64 cores (Table 7)": 127.0},
                    (400, 100): {"far field, 1 core (Table 1)": 95.0, "far field, 16 cores (Table 1)": 19.0,
                                 "near field, 1 core (Table 2)": 3848.0, "near field, 16 cores (Table 2)": 398.0},
                    (50, 10): {"1 core (Table 3)": 244.0, "16 cores (Table 3)": 156.0}}


def run_model2d(args, stream, world, barrier, max_over_ranks):
    """FP64 NESA products of the 2D model problem (Sec. 3) at the paper's size."""
    import torch

    import paper_1801_03589_gb300 as nesa
    from workloads.curve2d import charges, curve_points
    n = 100_000
    x = curve_points(n, seed=1)
    qd = torch.from_numpy(charges(n, seed=1)).cuda()
    y = torch.empty_like(qd)
    torch.cuda.synchronize()  # the copy above ran on torch's stream, the products run on `stream`
    out = {"workload": "N = 100,000 charges on a seeded closed curve (the paper's curve is not available); "
                       "phi = K q, K = -log|x_i - x_j|; FP64", "cases": []}
    peak = _peaks().get("hbm_gbs", 6790.0)
    for P, Q in ((300, 100), (400, 100), (50, 10)):
        t0 = time.perf_counter()
        g = nesa.Model2D(x, P, Q)
        build_s = time.perf_counter() - t0
        g.set_stream(stream)
        info = g.info()

        def timed(parts):
            for _ in range(max(3, args.warmup)):
                g.matvec(qd, y, parts=parts)
            stream.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            barrier()
            e0.record(stream)
            for _ in range(args.steps):
                g.matvec(qd, y, parts=parts)
            e1.record(stream)
            stream.synchronize()
            return max_over_ranks(e0.elapsed_time(e1) / args.steps)

        ms = timed(nesa.PART2D_ALL)
        ms_near, ms_far = timed(nesa.PART2D_NEAR), timed(nesa.PART2D_FAR)
        near_bytes = 8.0 * info["near_entries"] + 8.0 * 2 * n  # stored blocks once, charges in, potentials out
        out["cases"].append({"P": P, "Q": Q, "levels": [info["l0"], info["L"]], "leaves": info["n_boxes"][info["L"]],
                             "near_entries": info["near_entries"], "near_gb": 8e-9 * info["near_entries"],
                             "ms_per_matvec": ms, "matvec_per_s": job_throughput(world, 1, ms),
                             "near_only_ms": ms_near, "far_only_ms": ms_far,
                             "near_roofline": {"kernel": "k2_near (+ the two permutations)", "bound": "hbm",
                                               "achieved_gbs": near_bytes / (ms_near * 1e-3) / 1e9, "peak_gbs": peak,
                                               "frac": near_bytes / (ms_near * 1e-3) / 1e9 / peak},
                             "build_s": build_s, "paper_cpu_ms": MODEL2D_PAPER_MS[(P, Q)]})
        g.close()
    return out


def run_large(args, stream, world, barrier, max_over_ranks, name):
    """A large workload at full size: the r = 16 sphere (C5: 1,966,080 RWG, 9 levels, Q up
    to 4,096, 16 right-hand sides) or the aircraft body scaled to 52 wavelengths (C4L:
    516,413 RWG, Q up to 12,544, 8 right-hand sides).  Build, the mixed product of all
    right-hand sides, the FP64 product of one, and the mixed product's error against it.
    The coarse far levels whose FP64 tables would exceed 6 GB are generated when used."""
    import torch

    import paper_1801_03589_gb300 as nesa
    cfg = get_config(name)
    nrhs = cfg["nrhs"]
    t0 = time.perf_counter()
    g = nesa.Nesa(cfg["vertices"], cfg["triangles"], cfg["k"], leaf_size=cfg["leaf_size"],
                  n_levels=cfg["n_levels"], precision=nesa.MIXED, translate=nesa.TRANSLATE_TENSOR)
    build_s = time.perf_counter() - t0
    g.set_stream(stream)
    info = g.info()
    mixed = nesa.PART_ALL | nesa.PART_MIXED
    x = torch.from_numpy(random_coefficients(g.n, nrhs, seed=2024)).cuda()
    y = torch.empty_like(x)
    torch.cuda.synchronize()

    def timed(xx, yy, parts, reps):
        with torch.cuda.stream(stream):
            g.matvec(xx, yy, parts=parts)  # warm-up (allocations, tile tuning)
        stream.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        barrier()
        with torch.cuda.stream(stream):
            e0.record(stream)
            for _ in range(reps):
                g.matvec(xx, yy, parts=parts)
            e1.record(stream)
        stream.synchronize()
        return max_over_ranks(e0.elapsed_time(e1) / reps)

    ms_mx = timed(x, y, mixed, 3)
    g.profile_enable(True)
    with torch.cuda.stream(stream):
        g.matvec(x, y, parts=mixed)
    stream.synchronize()
    prof = g.profile_read()
    g.profile_enable(False)
    x1, y1 = x[:1].contiguous(), torch.empty_like(x[:1])
    ms64 = timed(x1, y1, nesa.PART_ALL, 1)
    y64 = y1.clone()
    ym = g.matvec(x1, parts=mixed)
    torch.cuda.synchronize()
    err = float((ym - y64).abs().pow(2).sum().sqrt() / y64.abs().pow(2).sum().sqrt())
    gemm = prof["translation_tensor_gemm"]
    gemm_tf = gemm["flops"] / (gemm["ms"] * 1e-3) / 1e12 if gemm["ms"] > 0 else None
    l0, L = info["l0"], info["n_levels"] - 1
    generated = [l for l in range(l0, L + 1) if 16.0 * info["n_offsets"][l] * info["q"][l] ** 2 > 6e9]
    out = {"workload": "%s: %s; %d right-hand sides" % (name, cfg["description"], nrhs),
           "n_unknowns": g.n, "levels": info["n_levels"], "l0": l0, "q": info["q"][l0:],
           "near_nnz": info["near_nnz"], "device_gb": g.info()["device_bytes"] / 1e9, "build_s": build_s,
           "build_split_s": info["build_split"],
           "generated_levels": generated,
           "mixed": {"ms_per_product": ms_mx, "nrhs": nrhs, "matvec_per_s": job_throughput(world, nrhs, ms_mx),
                     "tensor_gemm_ms": gemm["ms"], "tensor_gemm_tflops": gemm_tf,
                     "tensor_gemm_frac_of_bf16_burst": (gemm_tf / _peaks().get("bf16_tflops", 1901.0))
                     if gemm_tf else None,
                     "stages_ms": {k: v["ms"] for k, v in prof.items()}},
           "fp64": {"ms_per_product": ms64, "nrhs": 1, "matvec_per_s": job_throughput(world, 1, ms64)},
           "mixed_rel_err_vs_fp64": err}
    g.close()
    del g
    torch.cuda.empty_cache()
    return out


def _stages(prof, steps):
    return {k: {"launches": v["launches"], "ms_per_step": v["ms"] / steps,
                "tflops": (v["flops"] / (v["ms"] * 1e-3) / 1e12) if v["ms"] > 0 else None,
                "gbs": (v["bytes"] / (v["ms"] * 1e-3) / 1e9) if v["ms"] > 0 else None}
            for k, v in prof.items()}


def run_ours(args, world, rank, local):
    import torch

    import paper_1801_03589_gb300 as nesa

    torch.cuda.set_device(local)
    ranks = Ranks(world, "nccl", torch.device("cuda", local))
    cfg = get_config(args.workload)
    g = nesa.Nesa(cfg["vertices"], cfg["triangles"], cfg["k"], leaf_size=cfg["leaf_size"], n_levels=cfg["n_levels"],
                  precision=nesa.MIXED, translate=nesa.TRANSLATE_TENSOR, tile_n=args.tile_n)
    info = g.info()
    stream = torch.cuda.Stream()
    g.set_stream(stream)
    n = g.n
    nrhs = 1
    x = torch.from_numpy(random_coefficients(n, nrhs, seed=2024 + rank)).cuda()
    y = torch.empty_like(x)
    torch.cuda.synchronize()

    barrier, max_over_ranks = ranks.barrier, ranks.max

    mixed = nesa.PART_ALL | nesa.PART_MIXED
    with ClockSampler(local) as clk:
        ms64, prof64 = _time_products(g, x, y, nesa.PART_ALL, args.steps, args.warmup, stream, barrier)
        ms_mx, prof_mx = _time_products(g, x, y, mixed, args.steps, args.warmup, stream, barrier)
    ms64, ms_mx = max_over_ranks(ms64), max_over_ranks(ms_mx)
    value = job_throughput(world, nrhs, ms64)  # the FP64 product: the paper's arithmetic
    # accuracy of the mixed product against the FP64 product on this input
    y64 = g.matvec(x)
    ymx = g.matvec(x, parts=mixed)
    mixed_err = float((ymx - y64).abs().pow(2).sum().sqrt() / y64.abs().pow(2).sum().sqrt())

    # end to end through the host-pointer entry point: H2D of x, product, D2H of y
    # (FP64 product for the headline, the mixed product beside it)
    xh = torch.from_numpy(random_coefficients(n, nrhs, seed=7 + rank)).pin_memory()
    yh = torch.empty_like(xh).pin_memory()

    def e2e(parts):
        for _ in range(3):
            g.matvec_host_ptr(xh.data_ptr(), yh.data_ptr(), nrhs, parts)
        barrier()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            g.matvec_host_ptr(xh.data_ptr(), yh.data_ptr(), nrhs, parts)
        return max_over_ranks((time.perf_counter() - t0) * 1e3 / args.steps)

    e2e_ms = e2e(nesa.PART_ALL)
    e2e_mx_ms = e2e(mixed)

    # solves to 1e-5 (x-polarised plane wave along +z): the plain FP64 GMRES(100) with the
    # overlapping block-Jacobi preconditioner (the comparator of the metric), and FP64
    # refinement around GMRES(100) on the mixed product (inner tolerance 3e-3), without
    # and with that preconditioner; optionally the unpreconditioned FP64 solve
    solve = None
    if not args.no_solve:
        b = g.rhs_planewave([[0.0, 0.0, 1.0]], [[1.0, 0.0, 0.0]])
        torch.cuda.synchronize()
        barrier()

        def one(**kw):
            _, si = g.solve(b, tol=1e-5, restart=100, max_iters=4000, check=False, **kw)
            return {"seconds": max_over_ranks(si["seconds"]), "status": si["status"],
                    "iterations": si["iterations"], "refinements": si["refinements"],
                    "fp64_products": si["fp64_matvecs"], "true_rel_residual": si["rel_residual"][0]}

        t0 = time.perf_counter()
        g.precond_apply(b, nesa.PRECOND_OVERLAP)
        torch.cuda.synchronize()
        setup_s = time.perf_counter() - t0
        solve = {"tol": 1e-5,
                 "fp64_overlap": one(precond=nesa.PRECOND_OVERLAP),
                 "mixed_none": one(mixed=True, inner_tol=3e-3),
                 "mixed_overlap": one(mixed=True, inner_tol=3e-3, precond=nesa.PRECOND_OVERLAP),
                 "overlap_setup_seconds": setup_s,
                 "method": "fp64_*: GMRES(100) on the FP64 product; mixed_*: FP64 iterative refinement, inner "
                           "GMRES(100) on the mixed product to 3e-3; overlapping block-Jacobi = near-field "
                           "restricted additive Schwarz over touching leaves (setup reported apart)"}
        if args.fp64_solve:
            solve["fp64_none"] = one()

    # learned preconditioner on the aircraft-like body: trained on the GMRES vectors of
    # two plane waves, measured by iterations and true residual on six held-out ones
    learned = None
    if not args.no_learned:
        cf = get_config("C4")
        ga = nesa.Nesa(cf["vertices"], cf["triangles"], cf["k"], leaf_size=cf["leaf_size"],
                       n_levels=cf["n_levels"], precision=nesa.MIXED, translate=nesa.TRANSLATE_TENSOR)
        ga.set_stream(stream)
        kh, pol = plane_wave_directions(8, seed=180103589)
        B8 = ga.rhs_planewave(kh, pol)
        held = B8[2:].contiguous()
        torch.cuda.synchronize()

        def lsolve(bb, **kw):
            _, si = ga.solve(bb, tol=1e-5, restart=100, max_iters=3000, check=False, **kw)
            return {"seconds": si["seconds"], "status": si["status"], "iterations": si["iterations"],
                    "converged": si["converged"], "true_rel_residual_max": max(si["rel_residual"][:bb.shape[0]])}

        ga.precond_apply(held[:1], nesa.PRECOND_OVERLAP)  # setup outside the timed solves
        learned = {"workload": "C4: %s; 8 plane waves (seed 180103589), trained on 2, solved together on the "
                               "other 6 to 1e-5" % cf["description"],
                   "n_unknowns": ga.n,
                   "mixed_none": lsolve(held, mixed=True, inner_tol=3e-3),
                   "mixed_block_jacobi": lsolve(held, mixed=True, inner_tol=3e-3,
                                                precond=nesa.PRECOND_BLOCK_JACOBI),
                   "mixed_overlap": lsolve(held, mixed=True, inner_tol=3e-3, precond=nesa.PRECOND_OVERLAP)}
        learned["training"] = ga.precond_train(B8[:2].contiguous(), samples=48, steps=300)
        learned["mixed_learned"] = lsolve(held, mixed=True, inner_tol=3e-3, precond=nesa.PRECOND_LEARNED)
        # the plain FP64 form with block-Jacobi on one of them, capped at 300 steps
        _, si = ga.solve(held[:1].contiguous(), tol=1e-5, restart=100, max_iters=300, check=False,
                         precond=nesa.PRECOND_BLOCK_JACOBI)
        learned["fp64_block_jacobi_1rhs_300_steps"] = {"seconds": si["seconds"], "iterations": si["iterations"],
                                                        "true_rel_residual": si["rel_residual"][0]}
        del ga

    # batched sweep: three meshes of uneven size with 64 right-hand sides each, one CUDA
    # graph launch per pass over all of them (mixed product, autotuned tile widths)
    batch = None
    if not args.no_batch:
        names = ("C3a", "C3b", "C3c")
        t0 = time.perf_counter()
        members = []
        for nm in names:
            cf = get_config(nm)
            members.append(nesa.Nesa(cf["vertices"], cf["triangles"], cf["k"], leaf_size=cf["leaf_size"],
                                     n_levels=cf["n_levels"], precision=nesa.MIXED,
                                     translate=nesa.TRANSLATE_TENSOR))
        bx = [torch.from_numpy(random_coefficients(m.n, 64, seed=300 + i)).cuda() for i, m in enumerate(members)]
        by = [torch.empty_like(v) for v in bx]
        bt = nesa.Batch(members, bx, by, parts=mixed)
        build_s = time.perf_counter() - t0
        for _ in range(max(3, args.warmup)):
            bt.launch(stream)
        stream.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        barrier()
        e0.record(stream)
        for _ in range(args.steps):
            bt.launch(stream)
        e1.record(stream)
        stream.synchronize()
        pass_ms = max_over_ranks(e0.elapsed_time(e1) / args.steps)
        # per-stage device times of one eager 64-RHS product per member (outside the
        # timed region; the graph's branches overlap, so these add up to more than a pass)
        stages_ms = {}
        for m, v, w in zip(members, bx, by):
            m.profile_enable(True)
            m.matvec(v, w, parts=mixed)
            torch.cuda.synchronize()
            for k_, d_ in m.profile_read().items():
                stages_ms[k_] = stages_ms.get(k_, 0.0) + d_["ms"]
            m.profile_enable(False)
        batch = {"workload": "sphere r=2 (30,720 RWG), 3:1 spheroid (60,750 RWG), 4x4 plate (42,960 RWG); "
                             "64 right-hand sides each; mixed product",
                 "pass_ms": pass_ms, "matvec_per_s": job_throughput(world, 3 * 64, pass_ms),
                 "graph_kernel_nodes": bt.kernel_nodes, "launches_per_pass": 1, "build_and_capture_s": build_s,
                 "stages_ms_eager": {k_: round(v_, 4) for k_, v_ in stages_ms.items()},
                 "tile_n": [{l: t["tile_n"] for l, t in m.tuning().items()} for m in members]}
        bt.close()

    # the r = 16 sphere and the 52-wavelength aircraft at full size (generated coarse
    # translations); a failure here is reported in the block and leaves the rest of the
    # line intact
    large = None
    if not args.no_large:
        large = {}
        for name in ("C5", "C4L"):
            try:
                large[name] = run_large(args, stream, world, barrier, max_over_ranks, name)
            except Exception as e:  # noqa: BLE001
                large[name] = {"error": "%s: %s" % (type(e).__name__, e)}

    # the paper's 2D model problem at its size (a separate library path; a failure here
    # is reported in the block and leaves the rest of the line intact)
    model2d = None
    if not args.no_model2d:
        try:
            model2d = run_model2d(args, stream, world, barrier, max_over_ranks)
        except Exception as e:  # noqa: BLE001
            model2d = {"error": "%s: %s" % (type(e).__name__, e)}

    if rank != 0:
        ranks.close()
        return 0

    peaks = _peaks()
    hbm_peak = peaks.get("hbm_gbs", 6790.0)
    bf16_peak = peaks.get("bf16_tflops", 1901.0)

    # roofline of the headline (FP64) product: its dominant kernel is the translation
    # (k_translate64, Eqs. 12-13), bound by the FP64 pipe.  Achieved counts the
    # algorithmic 8 flops per complex multiply-add; the kernel's 3M form issues 12 FP64
    # FMAs per matrix entry and right-hand side (3 per channel, with the sums Re + Im of
    # the matrix stored) where that count has 16, so "issued_frac" is frac x 12/16
    tr64 = prof64["translation"]
    ach64 = tr64["flops"] / (tr64["ms"] * 1e-3) / 1e12
    roof = {"kernel": "k_translate64", "bound": "alu", "achieved": ach64, "peak": FP64_PEAK_TFLOPS,
            "unit": "TFLOP/s", "frac": ach64 / FP64_PEAK_TFLOPS, "issued_frac": ach64 / FP64_PEAK_TFLOPS * 12 / 16,
            "peak_note": "FP64 pipe: 152 SMs x 2 DFMA/clk x 2 flop x 2070 MHz (derived from unit counts and the "
                         "maximum clock); achieved counts 8 flops per complex multiply-add, the 3M form issues "
                         "12/16 of them",
            "traffic": (K_TRANSLATE64_DRAM_BYTES_C2 if (args.workload == CONFIG and nrhs == 1) else None),
            "traffic_unit": "bytes per product (all launches of the kernel in one product)",
            "share_of_product": tr64["ms"] / sum(v["ms"] for k, v in prof64.items() if k != "translation_tensor_gemm"),
            "ms_per_step": tr64["ms"] / args.steps}

    # roofline of the dominant kernel of the mixed product (largest device time); the
    # tensor-core GEMMs are timed alone (stage 4), the rest of the translation stage is
    # their split and reduction kernels
    gemm = prof_mx["translation_tensor_gemm"]
    rest = {"ms": max(0.0, prof_mx["translation"]["ms"] - gemm["ms"]), "flops": 0.0,
            "bytes": max(0.0, prof_mx["translation"]["bytes"] - gemm["bytes"])}
    kernels = {"k_tc_gemm": (gemm, "tensor"), "k_perm_x + k_near_receive_v": (prof_mx["near_reception"], "hbm"),
               "k_split + k_tc_gemm + k_pair_reduce (source transfer)": (prof_mx["source_transfer"], "tensor"),
               "k_radiate2": (prof_mx["radiation"], "hbm"),
               "k_split + k_pair_reduce": (rest, "hbm")}
    kernel = max(kernels, key=lambda k: kernels[k][0]["ms"])
    d, bound = kernels[kernel]
    sec = d["ms"] * 1e-3
    if bound == "tensor":
        roof_mx = {"bound": "tensor", "achieved": d["flops"] / sec / 1e12, "unit": "TFLOP/s", "peak": bf16_peak,
                   "peak_note": "BF16 dense, burst, measured (MEASURED_PEAKS.json; 1901 when absent); achieved "
                                "counts 8 flops per complex multiply-add of the translations and potential transfers, "
                                "the BF16 hi/lo split executes 3x that"}
    else:
        roof_mx = {"bound": "hbm", "achieved": d["bytes"] / sec / 1e9, "unit": "GB/s", "peak": hbm_peak,
                   "peak_note": "HBM copy bandwidth, measured"}
    # DRAM bytes (read + written) per product of the stage-4 launches, from the ncu capture
    # (r = 3 sphere, 1 RHS, this kernel version)
    traffic = GEMM_DRAM_BYTES_C2 if (kernel == "k_tc_gemm" and args.workload == CONFIG and nrhs == 1) else None
    roof_mx.update({"kernel": kernel, "frac": roof_mx["achieved"] / roof_mx["peak"], "traffic": traffic,
                    "traffic_unit": "bytes per product (all launches of the kernel in one product)",
                    "ms_per_step": d["ms"] / args.steps})
    # kernels launched in the timed region: one product captured into a CUDA graph by the
    # library's batch API, its kernel nodes counted, times the timed products
    counts = {}
    for name, parts in (("fp64", nesa.PART_ALL), ("mixed", mixed)):
        b1 = nesa.Batch([g], [x], [y], parts=parts)
        counts[name] = b1.kernel_nodes
        b1.close()
    launches = counts["fp64"] * args.steps

    cpu = None
    if not args.no_cpu_baseline:
        o = build_oracle(cfg)
        xo = random_coefficients(n, 1, seed=2024)[0]
        sec1, parts1, desc1 = oracle_sampled_product(o, xo, seed=3)
        procs = host_cores()
        pool = OraclePool(CONFIG if args.workload == CONFIG else args.workload, procs)
        try:
            secp, partsp, descp = pool.sampled_product(o, seed=3)
        finally:
            pool.close()
        cpu = {"value": 1.0 / secp, "unit": UNIT, "cores": procs, "kind": "oracle", "sample": descp,
               "seconds_per_matvec": secp, "stage_seconds": partsp, "host_cpu_count": os.cpu_count(),
               "single_core": {"value": 1.0 / sec1, "cores": 1, "seconds_per_matvec": sec1,
                               "stage_seconds": parts1, "sample": desc1}}

    solve_fp64 = solve["fp64_overlap"]["seconds"] if solve else None
    solve_mx = solve["mixed_overlap"]["seconds"] if solve else None
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": max(3, args.warmup), "ms_per_step": ms64, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": ("%s: %s" % (CONFIG, SPEC)) if args.workload == CONFIG else args.workload,
                   "nrhs": nrhs, "n_unknowns": n,
                   "product": "FP64: complex128 operator, FP64 kernels (the paper's arithmetic)",
                   "levels": info["n_levels"], "l0": info["l0"], "q": info["q"][info["l0"]:],
                   "near_nnz": info["near_nnz"], "device_gb": info["device_bytes"] / 1e9,
                   "build_s": info["build_seconds"], "build_split_s": info["build_split"],
                   "l2": "operator data %.1f GB (FP64) / %.1f GB (mixed) per product > 129 MB L2, no flush needed" % (
                       sum(v["bytes"] for v in prof64.values()) / args.steps / 1e9,
                       sum(v["bytes"] for v in prof_mx.values()) / args.steps / 1e9),
                   "parallelism": "replicas" if world > 1 else "single GPU"},
        "clocks": clk.summary(),
        "e2e": {"value": job_throughput(world, nrhs, e2e_ms), "unit": UNIT, "h2d_bytes_per_step": 16 * n * nrhs,
                "d2h_bytes_per_step": 16 * n * nrhs, "ms_per_step": e2e_ms},
        "gpu_launches": launches,
        "roofline": roof,
        "fp64_value": value,
        "mixed_value": job_throughput(world, nrhs, ms_mx),
        "mixed_vs_fp64": ms64 / ms_mx,
        "solve_fp64_s": solve_fp64,
        "solve_mixed_s": solve_mx,
        "solve_mixed_vs_fp64": (solve_fp64 / solve_mx) if solve else None,
        "stages": _stages(prof64, args.steps),
        "mixed": {"value": job_throughput(world, nrhs, ms_mx), "unit": UNIT, "ms_per_step": ms_mx, "dtype": "f32",
                  "product": "mixed precision: translations on tcgen05 tensor cores (BF16 hi/lo, 3 products, FP32 "
                             "accumulate), other stages complex64; rel err vs FP64 product %.1e" % mixed_err,
                  "rel_err_vs_fp64": mixed_err,
                  "e2e": {"value": job_throughput(world, nrhs, e2e_mx_ms), "unit": UNIT, "ms_per_step": e2e_mx_ms},
                  "gpu_launches_per_product": counts["mixed"],
                  "roofline": roof_mx, "stages": _stages(prof_mx, args.steps),
                  "tensor_tiles": {str(l): t for l, t in g.tuning().items()}},
        "solve": solve,
        "learned": learned,
        "batch": batch,
        "large": large,
        "model2d": model2d,
        "cpu_baseline": cpu,
    }
    print(json.dumps(line))
    ranks.close()
    return 0


def large_solve(name, max_iters, restart, nrhs=0):
    """Mixed solve with FP64 refinement to 1e-5 of a large workload, all its right-hand
    sides (plane waves, seed 180103589) in lock step, overlapping block-Jacobi.  Prints
    one JSON line (setup, solve time, iterations, refinements, true FP64 residuals)."""
    import torch

    import paper_1801_03589_gb300 as nesa
    c = get_config(name)
    nrhs = nrhs or c["nrhs"]
    t0 = time.perf_counter()
    g = nesa.Nesa(c["vertices"], c["triangles"], c["k"], leaf_size=c["leaf_size"], n_levels=c["n_levels"],
                  precision=nesa.MIXED, translate=nesa.TRANSLATE_TENSOR)
    out = {"workload": "%s: %s" % (name, c["description"]), "n_unknowns": g.n, "nrhs": nrhs,
           "build_s": time.perf_counter() - t0}
    kh, pol = plane_wave_directions(nrhs, seed=180103589)
    b = g.rhs_planewave(kh, pol)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    g.precond_apply(b[:1].contiguous(), nesa.PRECOND_OVERLAP)
    torch.cuda.synchronize()
    out["overlap_setup_s"] = time.perf_counter() - t0
    _, si = g.solve(b, tol=1e-5, restart=restart, max_iters=max_iters, check=False, mixed=True, inner_tol=3e-3,
                    precond=nesa.PRECOND_OVERLAP, max_refine=6)
    out["solve"] = {k: si[k] for k in ("status", "seconds", "iterations", "refinements", "fp64_matvecs", "matvecs")}
    out["solve"]["restart"] = restart
    out["solve"]["true_rel_residual"] = si["rel_residual"][:nrhs]
    out["device_gb"] = g.info()["device_bytes"] / 1e9
    print(json.dumps(out))
    return 0


PROFILE_RUNS = ("fp64_C2", "fp64_C3a", "tensor_C3a_generated", "tensor_C3a_stored", "tensor_C3a_64rhs",
                "batch_C3", "model2d_N1e5_P300_Q100")


def profile_run(name):
    """A small fixed workload for profiler captures: build, two products, exit 0."""
    import torch

    import paper_1801_03589_gb300 as nesa
    if name.startswith("fp64_"):
        c = get_config(name.split("_")[1])
        g = nesa.Nesa(c["vertices"], c["triangles"], c["k"], leaf_size=c["leaf_size"], n_levels=c["n_levels"])
        x = torch.from_numpy(random_coefficients(g.n, 1, seed=5)).cuda()
        for _ in range(2):
            g.matvec(x)
    elif name == "batch_C3":  # the batched sweep: three meshes x 64 RHS, one graph launch per pass
        members = []
        for nm in ("C3a", "C3b", "C3c"):
            cf = get_config(nm)
            members.append(nesa.Nesa(cf["vertices"], cf["triangles"], cf["k"], leaf_size=cf["leaf_size"],
                                     n_levels=cf["n_levels"], precision=nesa.MIXED, translate=nesa.TRANSLATE_TENSOR,
                                     tile_n=128))
        bx = [torch.from_numpy(random_coefficients(m.n, 64, seed=300 + i)).cuda() for i, m in enumerate(members)]
        by = [torch.empty_like(v) for v in bx]
        bt = nesa.Batch(members, bx, by, parts=nesa.PART_ALL | nesa.PART_MIXED)
        for _ in range(2):
            bt.launch()
        torch.cuda.synchronize()
        bt.close()
    elif name.startswith("tensor_"):
        c = get_config("C3a")
        tables = nesa.TABLES_GENERATED if name.endswith("generated") else nesa.TABLES_STORED
        g = nesa.Nesa(c["vertices"], c["triangles"], c["k"], leaf_size=c["leaf_size"], n_levels=c["n_levels"],
                      precision=nesa.MIXED, translate=nesa.TRANSLATE_TENSOR, tile_n=128, translation_tables=tables)
        x = torch.from_numpy(random_coefficients(g.n, 64 if name.endswith("64rhs") else 1, seed=5)).cuda()
        for _ in range(2):
            g.matvec(x, parts=nesa.PART_ALL | nesa.PART_MIXED)
    else:
        from workloads.curve2d import charges, curve_points
        n = 100_000
        g = nesa.Model2D(curve_points(n, seed=1), 300, 100)
        q = torch.from_numpy(charges(n, seed=1)).cuda()
        for _ in range(2):
            g.matvec(q)
    torch.cuda.synchronize()
    print("profile run %s: ok" % name)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-solve", action="store_true")
    ap.add_argument("--no-batch", action="store_true")
    ap.add_argument("--no-model2d", action="store_true", help="skip the 2D model problem block")
    ap.add_argument("--no-large", action="store_true",
                    help="skip the r = 16 sphere and 52-wavelength aircraft blocks (about 5 minutes)")
    ap.add_argument("--no-learned", action="store_true", help="skip the learned-preconditioner block (aircraft body)")
    ap.add_argument("--fp64-solve", action="store_true", help="also time the unpreconditioned FP64 solve (about 2.5 minutes)")
    ap.add_argument("--workload", default=CONFIG, help="workload name (smaller ones are for profiling runs)")
    ap.add_argument("--tile-n", type=int, default=0, choices=[0, 64, 128, 256],
                    help="fixed column-tile width of the tensor GEMMs (0: autotune); for runs under a profiler")
    ap.add_argument("--profile-run", choices=PROFILE_RUNS,
                    help="build one small fixed workload, run two products and exit (for ncu captures)")
    ap.add_argument("--large-solve", choices=["C5", "C4L"],
                    help="only a mixed solve to 1e-5 of a large workload (tens of minutes), one JSON line")
    ap.add_argument("--large-solve-iters", type=int, default=2500)
    ap.add_argument("--large-solve-restart", type=int, default=50)
    ap.add_argument("--large-solve-nrhs", type=int, default=0, help="right-hand sides (0: the workload's)")
    args = ap.parse_args()
    if args.profile_run:
        return profile_run(args.profile_run)
    if args.large_solve:
        return large_solve(args.large_solve, args.large_solve_iters, args.large_solve_restart, args.large_solve_nrhs)
    world, rank, local = dist_setup()
    if args.impl == "reference":
        return run_reference(args, world, rank)
    return run_ours(args, world, rank, local)


if __name__ == "__main__":
    sys.exit(main())
