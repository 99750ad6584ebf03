"""Benchmark of the sector product y = H x on the GPU (one JSON line on stdout).

Default workload: the spin-1/2 J1-J2 Heisenberg model on the periodic 6x5 square lattice
(site = x + 6y; 60 nearest bonds J1 = 1, 60 next-nearest bonds J2 = 0.5), N = 15 up spins,
D = 155,117,520, split into n_sub = 2 subsystems of 15 sites, FP64 vectors, one right-hand
side. One step is one full product (row enumeration, diagonal, every hop, rank, gather, store)
over the whole sector, x drawn from the seeded generator (U[-1,1], normalised).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--workload j1j2|chain|bose|xxz|batched|diff|rank] [--n-sub K] [--dtype f64|f32] [--nrhs R]
                    [--N n]   (another particle number of the same lattice, for small profiling cases)

``--impl reference`` times the CPU oracle (plain numpy, as it stands) on a bounded sample of
rows of the same workload, on this machine's host cores; under torchrun only rank 0 runs it.
Multi-GPU runs are independent replicas (the product is not sharded): every rank runs the whole
workload and ``value`` counts the rows of all ranks over the slowest rank's time.
"""

from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "H·v sector elements/s"
PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")
FALLBACK_HBM = 6800.0

# DRAM traffic per launch of the panel kernel from one ncu capture, keyed by the SHA-256 of the
# panel kernel's sources (PANEL_SOURCES) it was taken on; reported only while they are unchanged.
NCU_TRAFFIC = {
    # ncu --metrics dram__bytes_read.sum,dram__bytes_write.sum,gpu__time_duration.sum (one pass),
    # the fourth k_panel launch of the full-size J1-J2 6x5 N = 15 product with FP64 vectors:
    # 17.458 GB read + 1.236 GB written
    ("j1j2_square_6x5_N15", 2, "f64", 1, "8e33e958ae977eb0"): 18.694668544e9,
    # the same capture with FP32 vectors: 6.361 GB read + 0.613 GB written
    ("j1j2_square_6x5_N15", 2, "f32", 1, "8e33e958ae977eb0"): 6.973293568e9,
}

WORKLOADS = {
    "j1j2": 2,
    "chain": 1,
    "bose": 3,
    "xxz": 5,
    "batched": 4,
    "diff": 5,
    "rank": 0,
    "lanczos": 2,
}


# Sources the panel kernel is built from (kernel, plan, fixed-point helpers, shared structures).
PANEL_SOURCES = ("dq_panel.cu", "dq_panel.cpp", "dq_fixed.cuh", "dq_internal.h")


def kernel_source_hash() -> str:
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2407_14591_gb300", "csrc")
    for fn in PANEL_SOURCES:
        with open(os.path.join(csrc, fn), "rb") as f:
            h.update(fn.encode())
            h.update(f.read())
    return h.hexdigest()[:16]


def hbm_peak():
    try:
        with open(PEAKS_FILE) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM, "fallback"


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons while the timed region runs."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.dev = device_index
        self.proc = None
        self.path = os.path.join("/tmp", f"dq_clocks_{os.getpid()}.csv")

    def __enter__(self):
        try:
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits", "-lms", "100",
                 "-i", str(self.dev)], stdout=self.fh, stderr=subprocess.DEVNULL)
            time.sleep(0.3)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.fh.close()

    def summary(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        rows = []
        try:
            with open(self.path) as f:
                for line in f:
                    p = [v.strip() for v in line.split(",")]
                    if len(p) >= 9 and p[1].isdigit():
                        rows.append(p)
            os.remove(self.path)
        except Exception:
            pass
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [int(r[1]) for r in rows]
        mx = max(int(r[2]) for r in rows)
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({n for r in rows for n, v in zip(names, r[5:9]) if v.lower() == "active"})
        load = [v for v in sm if v >= 0.5 * mx] or sm
        return {"sm_mhz": int(statistics.median(load)), "sm_max_mhz": mx, "reasons": reasons, "samples": len(rows)}


def build_workload(number: int, n_sub, N=None):
    from paper_2407_14591_gb300 import binding as b
    from paper_2407_14591_gb300 import workloads as wl

    w, _ = wl.workload(number, n_sub=n_sub, draw_vector=False)
    if N is not None:
        w.N = N
        w.name = f"{w.name}_as_N{N}"
    s = b.make_sector(w.L, w.Q, w.N, w.n_sub)
    w2, x = wl.workload(number, n_sub=n_sub, D=s.dim)  # x first, then any disorder, one generator
    w.terms = w2.terms
    return w, s, x


def aggregate(ms_local: float, rows_local: int, steps: int, reduce_max=None, reduce_sum=None):
    """Whole-job throughput over ranks: rows of all ranks / slowest rank's time.

    reduce_max / reduce_sum reduce a float over ranks (identity on one rank)."""
    ms = reduce_max(ms_local) if reduce_max else ms_local
    rows = reduce_sum(float(rows_local)) if reduce_sum else float(rows_local)
    return ms, rows * steps / (ms / 1e3)


def _shm_put(arr):
    from multiprocessing import shared_memory

    shm = shared_memory.SharedMemory(create=True, size=max(1, arr.nbytes))
    view = np.ndarray(arr.shape, dtype=arr.dtype, buffer=shm.buf)
    view[...] = arr
    return shm, (shm.name, arr.shape, arr.dtype.str)


def _oracle_worker(task):
    """Worker process of the all-cores oracle timing: attach the shared sector and x, and run the
    oracle's gather form on this worker's rows. Returns (rows done, seconds)."""
    from multiprocessing import shared_memory

    from oracle import OracleSector, matvec_rows

    (L, Q, N, part, terms, descs, rows) = task
    shms, arrs = [], []
    for name, shape, dt in descs:
        shm = shared_memory.SharedMemory(name=name)
        shms.append(shm)
        arrs.append(np.ndarray(shape, dtype=np.dtype(dt), buffer=shm.buf))
    basis, keys, x = arrs
    o = OracleSector.from_arrays(L, Q, N, part, basis, keys)
    t0 = time.perf_counter()
    matvec_rows(o, terms, x, rows)
    el = time.perf_counter() - t0
    del o, basis, keys, x, arrs
    for shm in shms:
        shm.close()
    return len(rows), el


def oracle_rows_rate(w, partition, x, seconds: float, steps: int | None = None, warmup: int = 0,
                     all_cores: bool = True):
    """Time the oracle's gather form (as it stands) on bounded random-row samples of the workload:
    on one core, and (all_cores) on all host cores, the same sample size per core split into
    row-disjoint ranges over spawned worker processes that share the sector and x through shared
    memory. Returns a dict with the rates (rows/s), the rows timed and the untimed build time."""
    import multiprocessing as mp

    from oracle import OracleSector, matvec_rows

    t0 = time.perf_counter()
    o = OracleSector(w.L, w.Q, w.N, partition=partition)
    setup = time.perf_counter() - t0
    rng = np.random.default_rng(12345)
    rows_per = 1 << 12
    # calibrate the sample size so one step takes about `seconds / steps`
    t0 = time.perf_counter()
    matvec_rows(o, w.terms, x, rng.choice(o.dim, rows_per, replace=False))
    dt = time.perf_counter() - t0
    n_steps = steps if steps is not None else 4
    target = seconds / n_steps
    rows_per = int(min(o.dim, max(1 << 10, rows_per * target / max(dt, 1e-6))))
    for _ in range(warmup):
        matvec_rows(o, w.terms, x, rng.choice(o.dim, rows_per, replace=False))
    done = 0
    t0 = time.perf_counter()
    for _ in range(n_steps):
        matvec_rows(o, w.terms, x, rng.choice(o.dim, rows_per, replace=False))
        done += rows_per
    el = time.perf_counter() - t0
    out = {"rate1": done / el, "rows1": done, "s1": el, "setup": setup, "rows_per_step": rows_per,
           "steps": n_steps, "cores": 1}
    ncores = os.cpu_count() or 1
    if all_cores and ncores > 1:
        shms, descs = [], []
        try:
            for arr in (o.basis, o.keys, np.ascontiguousarray(x)):
                shm, d = _shm_put(arr)
                shms.append(shm)
                descs.append(d)
            ctx = mp.get_context("spawn")
            with ctx.Pool(ncores) as pool:
                # one untimed round so that every worker has imported the oracle
                pool.map(_oracle_worker, [(w.L, w.Q, w.N, partition, w.terms, descs,
                                           np.arange(c, o.dim, max(1, o.dim // 64))[:64]) for c in range(ncores)])
                done_all = 0
                t0 = time.perf_counter()
                for _ in range(n_steps):
                    rows = np.sort(rng.choice(o.dim, min(o.dim, rows_per * ncores), replace=False))
                    chunks = np.array_split(rows, ncores)  # row-disjoint ranges, one per worker
                    res = pool.map(_oracle_worker, [(w.L, w.Q, w.N, partition, w.terms, descs, c) for c in chunks])
                    done_all += sum(r[0] for r in res)
                el_all = time.perf_counter() - t0
            out.update({"rate_all": done_all / el_all, "rows_all": done_all, "s_all": el_all, "cores": ncores})
        finally:
            for shm in shms:
                shm.close()
                shm.unlink()
    return out


def lanczos_check(b, torch):
    """Workload 1 (periodic Heisenberg chain L=20, N=10): 100 Lanczos steps through the library
    with FP64 and FP32 vectors from the seeded start vector, with FP64 passes over the basis and
    with their double-single form, against the oracle's E0 stored in
    tests/golden/lanczos_workload1.txt. Wall-clock time of the synchronous call."""
    from paper_2407_14591_gb300 import workloads as wl

    ref = {}
    with open(os.path.join(ROOT, "tests", "golden", "lanczos_workload1.txt")) as f:
        for line in f:
            line = line.split("#", 1)[0].split()
            if line:
                ref[line[0]] = line[1]
    e_ref, steps = float(ref["E0"]), int(ref["steps"])
    w, _ = wl.workload(1, draw_vector=False)
    s = b.make_sector(w.L, w.Q, w.N, w.n_sub)
    w, x = wl.workload(1, D=s.dim)
    t = b.make_terms(s, w.terms)
    out = {"workload": w.name, "D": s.dim, "steps": steps, "E0_oracle": e_ref, "reorth": True}
    for dt, ds, name in ((torch.float64, False, "f64"), (torch.float32, False, "f32"),
                         (torch.float64, True, "f64_double_single"), (torch.float32, True, "f32_double_single")):
        v0 = torch.from_numpy(x).to("cuda", dt)
        b.lanczos(s, t, v0, steps, double_single=ds)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        r = b.lanczos(s, t, v0, steps, double_single=ds)
        el = time.perf_counter() - t0
        # the same number of products alone (CUDA events), for the cost of the rest of the step
        y = torch.empty_like(v0)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(r["steps_done"]):
            b.matvec(s, t, v0, y)
        e1.record()
        torch.cuda.synchronize()
        out[name] = {"E0": r["E0"], "rel_err": abs(r["E0"] - e_ref) / abs(e_ref), "ms": 1e3 * el,
                     "steps_done": r["steps_done"], "products_ms": e0.elapsed_time(e1)}
    return out


def run_reference(args, world, rank):
    if rank != 0:
        return
    number = WORKLOADS[args.workload]
    from paper_2407_14591_gb300 import workloads as wl
    from oracle import OracleSector, most_equal_partition, sector_dim

    w, _ = wl.workload(number, n_sub=args.n_sub, draw_vector=False)
    part = most_equal_partition(w.L, w.n_sub, w.Q)
    D = sector_dim(w.L, w.Q, w.N)
    w, x = wl.workload(number, n_sub=args.n_sub, D=D)
    r = oracle_rows_rate(w, part, x, seconds=max(8.0, 1.0 * args.steps), steps=args.steps, warmup=args.warmup)
    rate = r.get("rate_all", r["rate1"])
    el = r.get("s_all", r["s1"])
    line = {
        "impl": "reference", "metric": METRIC, "value": rate, "unit": "elements/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * el / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": w.name, "D": D, "n_sub": w.n_sub, "partition": part, "nrhs": 1},
        "cpu_baseline": {"value": rate, "unit": "elements/s", "cores": r["cores"], "kind": "oracle",
                         "sample": f"{r.get('rows_all', r['rows1']) // args.steps} random rows per step (gather form), "
                                   f"{args.steps} steps over {r['cores']} processes with row-disjoint ranges, "
                                   f"after a {r['setup']:.0f} s untimed sector build (enumerate + sort)",
                         "single_core": {"value": r["rate1"], "cores": 1, "rows": r["rows1"]}},
        "e2e": {"value": rate, "unit": "elements/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def run_batched(args, world, rank, local, dist, torch):
    """Workload 4: 64 disordered XXZ chains (L 16..26), 8 right-hand sides, one persistent launch
    per step, tuned once, replayed from a CUDA graph."""
    from paper_2407_14591_gb300 import binding as b
    from paper_2407_14591_gb300 import workloads as wl

    tdtype = torch.float64 if args.dtype == "f64" else torch.float32
    esize = 8 if args.dtype == "f64" else 4
    ws = wl.batched_chains(64, 8)
    secs = [b.make_sector(w.L, 2, w.N, 0) for w in ws]
    terms = [b.make_terms(s, w.terms) for s, w in zip(secs, ws)]
    xs = [torch.from_numpy(x).to("cuda", tdtype) for x in wl.batched_vectors([s.dim for s in secs], 8)]
    ys = [torch.empty_like(x) for x in xs]
    batch = b.make_batch(secs, terms, 8, tdtype)
    choice = batch.tune(xs, ys)
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        batch.matvec(xs, ys)
    torch.cuda.current_stream().wait_stream(side)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        batch.matvec(xs, ys)
    for _ in range(args.warmup):
        g.replay()
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()
        ev0.record(stream)
        for _ in range(args.steps):
            g.replay()
        ev1.record(stream)
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()
    rows = sum(s.dim for s in secs) * 8
    ms, value = aggregate(ev0.elapsed_time(ev1), rows, args.steps)
    ms_step = ms / args.steps
    alg_bytes = rows * 2 * esize
    peak, peak_kind = hbm_peak()
    # the main kernel alone, timed by the library's hooks on eager (not graph) launches
    b.timing_enable(True)
    for _ in range(args.steps):
        batch.matvec(xs, ys)
    kern_ms, kern_calls, kernels = b.timing_read()
    b.timing_enable(False)
    kern_ms_launch = kern_ms / max(kern_calls, 1)
    kernels_per_step = kernels // max(kern_calls, 1)
    achieved = alg_bytes / (kern_ms_launch / 1e3) / 1e9
    # the same products as 64 separate launches, for comparison
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for s, t, x, y in zip(secs, terms, xs, ys):
        b.matvec(s, t, x, y)
    e1.record(stream)
    torch.cuda.synchronize()
    seq_ms = e0.elapsed_time(e1)

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "elements/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": args.dtype, "data": "synthetic",
            "config": {"workload": "xxz_chains_64_L16to26_nrhs8", "sectors": len(secs),
                       "D_total": sum(s.dim for s in secs), "nrhs": 8, "launch_shape": choice,
                       "graph": True, "L2": "inputs larger than L2"},
            "effective_GBps": alg_bytes / (ms_step / 1e3) / 1e9,
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                         "traffic": None, "peak_source": peak_kind, "algorithmic_bytes_per_launch": alg_bytes,
                         "kernel": "k_batch",
                         "kernel_ms_per_launch": kern_ms_launch},
            "separate_launches_ms": seq_ms,
            "clocks": clk.summary(),
            "gpu_launches": args.steps * kernels_per_step,
        }
        print(json.dumps(line), flush=True)


def run_diff(args, world, rank, local, dist, torch):
    """Workload 5 as a training step: y = H(theta) x forward and the hand-written adjoint
    (dx = H dy, dtheta_k = <dy, T_k x>) backward, theta = 24 couplings + 24 fields."""
    from paper_2407_14591_gb300 import autograd as ag
    from paper_2407_14591_gb300 import binding as b
    from paper_2407_14591_gb300 import workloads as wl

    tdtype = torch.float64 if args.dtype == "f64" else torch.float32
    esize = 8 if args.dtype == "f64" else 4
    s = b.make_sector(24, 2, 12, 2)
    w, x_np = wl.workload(5, D=s.dim)
    params = []
    for bnd, (i, j) in enumerate(wl.chain_bonds(24)):
        params.append(("XY", i, j, bnd, 1.0))
        params.append(("ZZ", i, j, bnd, 1.0))
    for i in range(24):
        params.append(("Z", i, -1, 24 + i, 1.0))
    op = ag.ParamOperator(s, params, n_params=48)
    theta = torch.tensor([t[3] for t in w.terms if t[0] == "XY"] + [t[3] for t in w.terms if t[0] == "Z"],
                         dtype=torch.float64, requires_grad=True)
    x = torch.from_numpy(x_np).to("cuda", tdtype).requires_grad_(True)
    r = torch.ones_like(x)

    def step():
        theta.grad = None
        x.grad = None
        y = ag.matvec(op, x, theta)
        y.backward(r)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        torch.cuda.synchronize()
        b.timing_enable(True)
        ev0.record(stream)
        for _ in range(args.steps):
            step()
        ev1.record(stream)
        torch.cuda.synchronize()
    kern_ms, kern_calls, kernels = b.timing_read()
    b.timing_enable(False)
    ms, value = aggregate(ev0.elapsed_time(ev1), s.dim, args.steps)
    ms_step = ms / args.steps
    # forward product, backward product, per-term reduction: x, y, dy, dx and x again
    alg_bytes = s.dim * esize * 6
    peak, peak_kind = hbm_peak()
    achieved = alg_bytes / (ms_step / 1e3) / 1e9

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "elements/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": args.dtype, "data": "synthetic",
            "config": {"workload": "disordered_xxz_L24_N12_forward_backward", "D": s.dim, "params": 48,
                       "step": "y = H(theta) x, then dx and dtheta"},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                         "traffic": None, "peak_source": peak_kind, "algorithmic_bytes_per_launch": alg_bytes,
                         "kernel": {"panel": "k_panel", "panel_pb": "k_panel_pb", "panel_w": "k_panel_w", "panel_q": "k_panel_q"}.get(
                             op.compile(theta.detach()).path,
                             "k_matvec_q2_fx" if args.dtype == "f64" else "k_matvec_q2_f32x") + " + k_term_grads",
                         "main_kernels_ms_per_step": kern_ms / args.steps},
            "clocks": clk.summary(),
            "gpu_launches": kernels,
        }
        print(json.dumps(line), flush=True)


RANK_SWEEP = [  # (L, Q, N, n_sub): Fig. 4-6 analogue; half filling unless stated
    (20, 2, 10, 1), (20, 2, 10, 2), (20, 2, 10, 4), (20, 2, 10, 20),
    (24, 2, 12, 1), (24, 2, 12, 2), (24, 2, 12, 3), (24, 2, 12, 6), (24, 2, 12, 24),
    (28, 2, 14, 2), (28, 2, 14, 3), (28, 2, 14, 4), (28, 2, 14, 7),
    (32, 2, 16, 2), (32, 2, 16, 3), (32, 2, 16, 4), (32, 2, 16, 8), (32, 2, 16, 32),
    (32, 2, 4, 2), (32, 2, 4, 4),
    (12, 4, 18, 1), (12, 4, 18, 2), (12, 4, 18, 3), (16, 4, 24, 2), (16, 4, 24, 4),
]


def run_rank(args, world, rank, local, dist, torch):
    """Function (i) throughput: index_of_batch on 2^24 random valid states per configuration
    (states from state_at_batch on random indices), one JSON line per configuration."""
    from paper_2407_14591_gb300 import binding as b

    n = 1 << 24
    g = torch.Generator(device="cpu").manual_seed(20240719)
    for (L, Q, N, n_sub) in RANK_SWEEP:
        s = b.make_sector(L, Q, N, n_sub)
        idx = (torch.rand(n, generator=g, dtype=torch.float64) * s.dim).long().clamp_(max=s.dim - 1).to("cuda")
        st = s.state_at_batch(idx)
        out = torch.empty_like(idx)
        for _ in range(max(1, args.warmup)):
            s.index_of_batch(st, out)
        torch.cuda.synchronize()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record()
        for _ in range(args.steps):
            s.index_of_batch(st, out)
        ev1.record()
        torch.cuda.synchronize()
        s.check_device()
        ok = bool(torch.equal(out, idx))
        ms = ev0.elapsed_time(ev1) / args.steps
        nb = (Q - 1).bit_length()
        table_bytes = sum(4 << (nb * Lk) for Lk in set(s.partition))
        if rank == 0:
            print(json.dumps({"metric": "ranks/s", "value": n / (ms / 1e3), "unit": "ranks/s", "L": L, "Q": Q,
                              "N": N, "n_sub": s.n_sub, "partition": s.partition, "D": s.dim,
                              "rank_table_bytes": table_bytes, "ms": ms, "states": n, "roundtrip_ok": ok}),
                  flush=True)


def run_lanczos(args, world, rank, local, dist, torch):
    """The Lanczos form of workload 2 (J1-J2 6x5, N = 15, D = 155,117,520) or, with
    --lanczos-workload bose, workload 3 (Bose-Hubbard Q = 4, L = 14, N = 14, D = 6,472,168), at
    full size: the same seeded start vector with FP64 vectors and with FP32 vectors (FP64
    recurrence, dot products and updates in both; then both again with the double-single passes
    over the basis), full re-orthogonalisation (classical Gram-Schmidt, a second pass when the
    DGKS criterion asks for it). One JSON line: E0 of each, the FP32/FP64 relative difference, the
    residual ||H psi - E0 psi|| / |E0| of each Ritz vector (FP64), time per Lanczos step, and the
    product's share of it."""
    from paper_2407_14591_gb300 import binding as b

    steps = args.lanczos_steps
    number = {"j1j2": 2, "bose": 3}[args.lanczos_workload]
    w, s, x_np = build_workload(number, args.n_sub if number == 2 else None, args.N if number == 2 else None)
    t = b.make_terms(s, w.terms)
    out = {}
    for dt, ds, name in ((torch.float64, False, "f64"), (torch.float32, False, "f32"),
                         (torch.float64, True, "f64_double_single"), (torch.float32, True, "f32_double_single")):
        v0 = torch.from_numpy(x_np).to("cuda", dt)
        b.lanczos(s, t, v0, 3, reorth=True, double_single=ds)  # warm-up (scratch, tables)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        r = b.lanczos(s, t, v0, steps, reorth=True, want_vector=True, double_single=ds)
        el = time.perf_counter() - t0
        psi = r.pop("psi")
        hpsi = b.matvec(s, t, psi)
        res = (torch.linalg.norm(hpsi.double() - r["E0"] * psi.double()) / abs(r["E0"])).item()
        del hpsi, psi
        # the products alone: `steps` products of the same vector, CUDA events
        y = torch.empty_like(v0)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(r["steps_done"]):
            b.matvec(s, t, v0, y)
        e1.record()
        torch.cuda.synchronize()
        prod_ms = e0.elapsed_time(e1)
        out[name] = {"E0": r["E0"], "steps_done": r["steps_done"], "ms_per_step": 1e3 * el / max(r["steps_done"], 1),
                     "residual": res, "products_ms_per_step": prod_ms / max(r["steps_done"], 1),
                     "total_s": el}
        del v0, y
    rel = abs(out["f32"]["E0"] - out["f64"]["E0"]) / abs(out["f64"]["E0"])
    if rank == 0:
        print(json.dumps({"metric": "Lanczos E0, FP32 vectors vs FP64 vectors", "value": rel, "unit": "relative",
                          "higher_is_better": False, "n_gpus": world, "steps": steps, "data": "synthetic",
                          "config": {"workload": w.name, "D": s.dim, "n_sub": s.n_sub, "reorth": True},
                          **out}), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="j1j2", choices=sorted(WORKLOADS))
    ap.add_argument("--n-sub", type=int, default=None)
    ap.add_argument("--dtype", default="f64", choices=["f64", "f32"])
    ap.add_argument("--nrhs", type=int, default=1)
    ap.add_argument("--N", type=int, default=None, help="override the particle number (smaller profiling cases)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-lanczos", action="store_true", help="skip the workload-1 Lanczos E0 check")
    ap.add_argument("--lanczos-steps", type=int, default=100, help="steps of --workload lanczos")
    ap.add_argument("--lanczos-workload", default="j1j2", choices=["j1j2", "bose"],
                    help="sector of --workload lanczos: workload 2 (j1j2) or workload 3 (bose)")
    ap.add_argument("--graph", type=int, default=0,
                    help="also time this many products captured in one CUDA graph (launch-free rate)")
    args = ap.parse_args()

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))

    if args.impl == "reference":
        run_reference(args, world, rank)
        return

    import torch

    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    from paper_2407_14591_gb300 import binding as b

    if args.workload in ("batched", "diff", "rank", "lanczos"):
        {"batched": run_batched, "diff": run_diff, "rank": run_rank,
         "lanczos": run_lanczos}[args.workload](args, world, rank, local, dist, torch)
        if dist is not None:
            dist.barrier()
            dist.destroy_process_group()
        return
    number = WORKLOADS[args.workload]
    w, s, x_np = build_workload(number, args.n_sub, args.N)
    tdtype = torch.float64 if args.dtype == "f64" else torch.float32
    esize = 8 if args.dtype == "f64" else 4
    if args.nrhs > 1:
        rng = np.random.default_rng(777)
        x_np = np.repeat(x_np[:, None], args.nrhs, axis=1) * rng.uniform(0.5, 1.5, size=(1, args.nrhs))
    x = torch.from_numpy(np.ascontiguousarray(x_np)).to("cuda", tdtype)
    y = torch.empty_like(x)
    t = b.make_terms(s, w.terms)
    stream = torch.cuda.current_stream()

    for _ in range(args.warmup):
        b.matvec(s, t, x, y)
    torch.cuda.synchronize()
    s.check_device()

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    path = t.path if args.nrhs == 1 else "general"
    general = (("k_matvec_q2_fx" if args.dtype == "f64" else "k_matvec_q2_f32x") if w.Q == 2 else
               ("k_matvec_qg_fx" if args.dtype == "f64" else "k_matvec_qg_f32x"))
    kernel_name = {"panel": "k_panel", "panel_pb": "k_panel_pb", "panel_w": "k_panel_w", "panel_q": "k_panel_q",
                   "cluster": "k_matvec_cl"}.get(path, general)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        barrier()
        b.timing_enable(True)  # CUDA events around the main kernel of every product, on its stream
        ev0.record(stream)
        for _ in range(args.steps):
            b.matvec(s, t, x, y)
        ev1.record(stream)
        barrier()
    kern_ms, kern_calls, kernels = b.timing_read()
    b.timing_enable(False)

    graph = None
    if args.graph:
        # launch-free rate: args.graph products captured once in a CUDA graph, replayed
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, capture_error_mode="relaxed"):
            for _ in range(args.graph):
                b.matvec(s, t, x, y)
        for _ in range(2):
            g.replay()
        torch.cuda.synchronize()
        reps = 5
        g0, g1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        g0.record(stream)
        for _ in range(reps):
            g.replay()
        g1.record(stream)
        torch.cuda.synchronize()
        gms = g0.elapsed_time(g1) / (reps * args.graph)
        graph = {"products_per_graph": args.graph, "replays": reps, "ms_per_product": gms,
                 "elements_per_s": world * s.dim * args.nrhs / (gms / 1e3)}
        del g

    def red(op):
        def f(v):
            if dist is None:
                return v
            tt = torch.tensor([v], device="cuda", dtype=torch.float64)
            dist.all_reduce(tt, op=op)
            return float(tt.item())
        return f

    rows = s.dim * args.nrhs
    ms, value = aggregate(ev0.elapsed_time(ev1), rows, args.steps,
                          red(dist.ReduceOp.MAX) if dist else None, red(dist.ReduceOp.SUM) if dist else None)
    s.check_device()
    ms_step = ms / args.steps
    alg_bytes = s.dim * args.nrhs * 2 * esize
    peak, peak_kind = hbm_peak()
    kern_ms_launch = kern_ms / max(kern_calls, 1)  # average duration of the main kernel
    achieved = alg_bytes / (kern_ms_launch / 1e3) / 1e9
    src_hash = kernel_source_hash()
    traffic = NCU_TRAFFIC.get((w.name, s.n_sub, args.dtype, args.nrhs, src_hash))

    e2e = None
    if not args.no_e2e:
        # End to end through the public product call with pinned host buffers: every step copies
        # its x host->device and its y device->host. Pipelined: the copy of step k+1's x (copy
        # stream) and of step k-1's y (second copy stream) overlap step k's product; two device
        # buffer pairs, ordered by events. The serial form (copy, product, copy on one stream) is
        # reported beside it.
        xh = torch.empty(x.shape, dtype=tdtype, pin_memory=True)
        xh.copy_(x)
        yh = [torch.empty(x.shape, dtype=tdtype, pin_memory=True) for _ in range(2)]
        xb, yb = [x, torch.empty_like(x)], [y, torch.empty_like(y)]
        k_e2e = max(2, min(args.steps, 50))  # the timed steps themselves (bounded run time)
        h2d, d2h = torch.cuda.Stream(), torch.cuda.Stream()

        def ev():
            return torch.cuda.Event()

        barrier()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        ev_in, ev_done, ev_out = [], [], []
        for k in range(k_e2e):
            i = k % 2
            if k == 0:
                h2d.wait_event(e0)
            elif k >= 2:
                h2d.wait_event(ev_done[k - 2])  # the product of step k-2 has read x buffer i
            with torch.cuda.stream(h2d):
                xb[i].copy_(xh, non_blocking=True)
            ev_in.append(ev())
            ev_in[k].record(h2d)
            stream.wait_event(ev_in[k])
            if k >= 2:
                stream.wait_event(ev_out[k - 2])  # y buffer i read back
            b.matvec(s, t, xb[i], yb[i])
            ev_done.append(ev())
            ev_done[k].record(stream)
            d2h.wait_event(ev_done[k])
            with torch.cuda.stream(d2h):
                yh[i].copy_(yb[i], non_blocking=True)
            ev_out.append(ev())
            ev_out[k].record(d2h)
        stream.wait_event(ev_out[-1])
        e1.record(stream)
        barrier()
        ems = e0.elapsed_time(e1)
        # the last read-back equals the device-timed product (the same x, deterministic sums)
        same = bool(torch.equal(yh[(k_e2e - 1) % 2], y.cpu()))
        # serial form for comparison
        s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        s0.record(stream)
        for _ in range(k_e2e):
            x.copy_(xh, non_blocking=True)
            b.matvec(s, t, x, y)
            yh[0].copy_(y, non_blocking=True)
        s1.record(stream)
        barrier()
        sms_ = s0.elapsed_time(s1)
        if dist is not None:
            tt = torch.tensor([ems, sms_], device="cuda", dtype=torch.float64)
            dist.all_reduce(tt, op=dist.ReduceOp.MAX)
            ems, sms_ = float(tt[0].item()), float(tt[1].item())
        e2e = {"value": world * rows * k_e2e / (ems / 1e3), "unit": "elements/s",
               "h2d_bytes_per_step": int(x.numel() * esize), "d2h_bytes_per_step": int(y.numel() * esize),
               "steps": k_e2e, "ms_per_step": ems / k_e2e, "pipelined": True, "output_checked": same,
               "serial_ms_per_step": sms_ / k_e2e}
        del xb[1], yb[1]

    cpu = None
    if rank == 0 and not args.no_cpu_baseline and args.nrhs == 1:
        r = oracle_rows_rate(w, s.partition, x_np if x_np.ndim == 1 else x_np[:, 0], seconds=8.0)
        rate = r.get("rate_all", r["rate1"])
        cpu = {"value": rate, "unit": "elements/s", "cores": r["cores"], "kind": "oracle",
               "sample": f"{r.get('rows_all', r['rows1']) // r['steps']} random rows per step, {r['steps']} steps (gather form, "
                         f"numpy), over {r['cores']} spawned processes with row-disjoint ranges, after a "
                         f"{r['setup']:.0f} s untimed sector build",
               "single_core": {"value": r["rate1"], "cores": 1, "rows": r["rows1"], "seconds": r["s1"]}}

    lz = lanczos_check(b, torch) if rank == 0 and not args.no_lanczos else None

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "elements/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": args.dtype, "data": "synthetic",
            "config": {"workload": w.name, "D": s.dim, "n_sub": s.n_sub, "partition": s.partition,
                       "nrhs": args.nrhs, "L2": "inputs larger than L2" if alg_bytes > 129e6 else "inputs fit in L2",
                       "parallelism": f"replicas{world}" if world > 1 else "single"},
            "effective_GBps": alg_bytes / (ms_step / 1e3) / 1e9,
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": traffic, "peak_source": peak_kind,
                         "algorithmic_bytes_per_launch": alg_bytes, "kernel": kernel_name,
                         "kernel_ms_per_launch": kern_ms_launch, "source_hash": src_hash},
            "clocks": clk.summary(),
            "gpu_launches": kernels,
            "e2e": e2e,
            "cpu_baseline": cpu,
            "lanczos": lz,
            "graph": graph,
        }
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
