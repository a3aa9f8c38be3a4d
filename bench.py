"""Benchmark of the batched small-matrix hot path on GB300.

One step = one pass over every cell of the placement sweep at the largest
sweep batch: the six operations {gemm, posv (potrf+potrs), trsm, getrf+getrs,
rotation-chain compose, SE(3) apply} at n in {3,6,7,12,14,24,32,64} on 16384
independent problems each (48 launches), every launch with the placement the
library's measured table selects ("tuned").  The same step with one fixed
placement (one thread per problem where feasible, else one warp: "plain") is
timed beside it.

Reported (one compact JSON line on stdout; the per-cell rows and the full
records of the other configurations go to a detail file, a per-cell table
to stderr):
  value       batched matrices/s of the tuned step, inputs resident in HBM,
              the K timed steps replayed as one CUDA graph (the library's
              calls are capture-safe) that forks into --streams streams, the
              independent cells spread over them; per-cell times from a
              graph of each cell alone;
  e2e         the same through host buffers (pinned H2D of every input and
              D2H of every result inside the timed region);
  roofline    of the dominant kernel (largest share of the step), from CUDA
              events around its launches;
  cpu_baseline  the FP64 C oracle on a bounded sample, all host cores (and
              the same sample on one core);
  accuracy    the worst per-problem relative error of the tuned and the
              plain results of every cell against the oracle's results on
              the same problems (the oracle's sample of the CPU baseline);
  plain       the plain step and the tuned/plain speedup;
  extras      headline numbers of the other configurations (mixed sizes,
              tensor-core GEMM, refinement, learned placement).
`--impl reference` times the oracle (the reference arm of this task) on the
same workload, one bounded sample per step.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "batched matrices/s and % of HBM/FP32 roofline, tuned vs plain at 1e-4 rel error"
BATCH = 16384


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return {"hbm_gbs": float(d["hbm_gbs"]), "src": "measured", "sm_max_mhz": float(d.get("sm_max_mhz", 2070.0))}
    return {"hbm_gbs": 6800.0, "src": "fallback", "sm_max_mhz": 2070.0}


def fp32_peak_tflops(sms: int, mhz: float) -> float:
    """FP32 SIMT peak: SMs x 128 FP32 lanes x 2 flop (FFMA) x clock."""
    return sms * 128 * 2 * mhz * 1e6 / 1e12


# ----------------------------------------------------------------- clocks
class ClockSampler:
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = None

    def __enter__(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
            time.sleep(0.3)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        if self.proc is None or not self.path or not os.path.exists(self.path):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx = float(parts[2])
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx, "samples": len(sm),
                "reasons": sorted(reasons)}


# ------------------------------------------------------------------ setup
def cell_list(ops, sizes, batch):
    return [(op, n, batch) for op in ops for n in sizes]


def plain_placement(cell):
    import paper_2609_28179_gb300 as g
    for scope in (g.GLASS_SCOPE_THREAD, g.GLASS_SCOPE_WARP):
        if cell.feasible(scope, 1):
            return scope, 1
    return g.GLASS_SCOPE_BLOCK, 1


def resolved_placement(cell):
    import paper_2609_28179_gb300 as g
    from paper_2609_28179_gb300.cells import OP_ID
    nn = cell.n if cell.op not in ("rot3", "se3") else (3 if cell.op == "rot3" else 4)
    s, pl = g.glass_get_placement(OP_ID[cell.op], nn, cell.k, cell.batch)
    g.check(s, "get_placement")
    return pl


def stream_assignment(per_ms, nstreams):
    """Longest-processing-time-first assignment of cells to streams by their
    measured times: cell index -> stream index."""
    load = [0.0] * nstreams
    out = [0] * len(per_ms)
    for i in sorted(range(len(per_ms)), key=lambda i: -per_ms[i]):
        j = min(range(nstreams), key=lambda j: load[j])
        out[i] = j
        load[j] += per_ms[i]
    return out


def time_steps(cells, placements, steps, warmup, barrier=None, nstreams=1):
    """Warm up with `warmup` eager passes, then time `steps` passes of the
    step captured in one CUDA graph (the library's calls never allocate,
    synchronise or read device memory on the host, so a step records as a
    graph and replays without host launch gaps).  The cells are independent
    problems: with nstreams > 1 the graph forks into that many streams, each
    cell's launches on one of them (assigned by measured time), so that
    latency-bound cells overlap others.  Every destructive cell reads its
    own fresh input copy in each pass; the copies are restored, untimed,
    before the replay.  Per-cell times come from a graph of that cell's
    `steps` launches alone.  Returns (total_ms, per-cell ms)."""
    import torch
    import paper_2609_28179_gb300 as g
    for w in range(warmup):
        for c, (s, p) in zip(cells, placements):
            g.check(c.launch(w, s, p), f"{c.op} n={c.n}")
    torch.cuda.synchronize()

    def restore_all():
        for c in cells:
            c.restore()
        torch.cuda.synchronize()

    def replay_ms(graph):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        graph.replay()
        b.record()
        torch.cuda.synchronize()
        return a.elapsed_time(b)

    cap = torch.cuda.Stream()
    per = []
    for c, (s, p) in zip(cells, placements):
        gr = torch.cuda.CUDAGraph()
        with torch.cuda.graph(gr, stream=cap):
            for st in range(steps):
                c.launch(warmup + st, s, p)
        c.restore()
        torch.cuda.synchronize()
        per.append(replay_ms(gr) / steps)
        del gr
    step = torch.cuda.CUDAGraph()
    branches = [torch.cuda.Stream() for _ in range(nstreams)] if nstreams > 1 else [cap]
    owner = stream_assignment(per, nstreams) if nstreams > 1 else [0] * len(cells)
    with torch.cuda.graph(step, stream=cap):
        if nstreams > 1:
            fork = torch.cuda.Event()
            fork.record(cap)
            for b in branches:
                b.wait_event(fork)
        for st in range(steps):
            for i, (c, (s, p)) in enumerate(zip(cells, placements)):
                c.launch(warmup + st, s, p, stream=branches[owner[i]])
        if nstreams > 1:
            for b in branches:
                join = torch.cuda.Event()
                join.record(b)
                cap.wait_event(join)
    restore_all()
    replay_ms(step)          # first replay uploads the graph; not timed
    restore_all()
    if barrier:
        barrier()
    torch.cuda.synchronize()
    total = replay_ms(step)  # ends with a synchronize
    if barrier:
        barrier()
    del step
    return total, per


def e2e_steps(cells, steps, warmup):
    """End to end through the public API with host buffers: per step, pinned
    H2D of every cell's inputs, the launches, D2H of every result.  Three
    streams by role -- uploads, launches, downloads -- so the two copy
    engines and the SMs stay busy at once: a cell's launch waits for its
    upload, its download for its launch, and its next upload (the buffers
    are reused in place) for its download."""
    import torch
    pinned_in, pinned_out, outs = [], [], []
    h2d = d2h = 0
    for c in cells:
        pin = {k: torch.from_numpy(v).pin_memory() for k, v in c.host.items()}
        pinned_in.append(pin)
        h2d += sum(t.numel() * 4 for t in pin.values())
        res = []
        w = c.work[0]
        if c.op in ("gemm", "rot3", "se3"):
            res.append(c.out)
        elif c.op == "posv":
            res += [w["A"], w["B"], c.info]
        elif c.op == "trsm":
            res.append(w["B"])
        else:
            res += [w["A"], w["B"], c.ipiv, c.info]
        outs.append(res)
        po = [torch.empty(r.shape, dtype=r.dtype).pin_memory() for r in res]
        pinned_out.append(po)
        d2h += sum(r.numel() * r.element_size() for r in res)

    up, run, down = torch.cuda.Stream(), torch.cuda.Stream(), torch.cuda.Stream()
    main = torch.cuda.current_stream()
    ev_in = [torch.cuda.Event() for _ in cells]
    ev_run = [torch.cuda.Event() for _ in cells]
    ev_out = [None] * len(cells)

    def one_step():
        for i, (c, pin) in enumerate(zip(cells, pinned_in)):
            with torch.cuda.stream(up):
                if ev_out[i] is not None:
                    up.wait_event(ev_out[i])
                w = c.work[0]
                for k, t in pin.items():
                    w[k].copy_(t, non_blocking=True)
                ev_in[i].record(up)
        for i, c in enumerate(cells):
            run.wait_event(ev_in[i])
            c.launch(0, stream=run)
            ev_run[i].record(run)
        for i, (res, po) in enumerate(zip(outs, pinned_out)):
            with torch.cuda.stream(down):
                down.wait_event(ev_run[i])
                for r, p in zip(res, po):
                    p.copy_(r, non_blocking=True)
                ev = torch.cuda.Event()
                ev.record(down)
                ev_out[i] = ev

    for _ in range(warmup):
        one_step()
    torch.cuda.synchronize()
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t0.record(main)
    for s in (up, run, down):
        s.wait_stream(main)
    for _ in range(steps):
        one_step()
    for s in (up, run, down):
        main.wait_stream(s)
    t1.record(main)
    torch.cuda.synchronize()
    return t0.elapsed_time(t1), h2d, d2h


# ------------------------------------------------------------ cpu oracle
def oracle_cell(op, n, host, batch, sample):
    """The FP64 oracle on the first `sample` problems of a cell: (seconds,
    problems, outputs) -- the outputs keyed like gpu_outputs'."""
    import numpy as np
    import oracle
    from paper_2609_28179_gb300.cells import NPTS, rhs_of
    k = rhs_of(op, n)
    s = min(sample, batch)
    f64 = lambda key, per: host[key][: s * per].astype(np.float64)
    t = time.perf_counter()
    if op == "gemm":
        out = {"X": oracle.gemm(n, n, n, f64("A", n * n), f64("B", n * n), s)}
    elif op == "posv":
        L, X, _ = oracle.posv(n, 1, f64("A", n * n), f64("B", n), s)
        out = {"X": X, "L": L}
    elif op == "trsm":
        out = {"X": oracle.trsm(n, k, f64("A", n * n), f64("B", n * k), s)}
    elif op == "getrf_getrs":
        LU, piv, X, _ = oracle.getrf_getrs(n, 1, f64("A", n * n), f64("B", n), s)
        out = {"X": X, "LU": LU, "ipiv": piv}
    elif op == "rot3":
        out = {"X": oracle.rot3_compose(k, f64("A", 9 * k), s)}
    else:
        out = {"X": oracle.se3_apply(k, f64("A", 16 * k), NPTS, f64("B", 3 * NPTS), s)}
    return time.perf_counter() - t, s, out


def oracle_cell_time(op, n, host, batch, sample):
    """Seconds the FP64 oracle takes for `sample` problems of a cell."""
    dt, s, _ = oracle_cell(op, n, host, batch, sample)
    return dt, s


def gpu_outputs(cell, placement, count):
    """Outputs of one eager launch of `cell` at `placement` on its pristine
    input (work set 0, restored first), first `count` problems, as float64
    host arrays keyed X (solution / product / composed result), L (posv
    factor, lower triangle), LU and ipiv (getrf)."""
    import numpy as np
    import torch
    import paper_2609_28179_gb300 as g
    scope, pack = placement
    cell.restore()
    g.check(cell.launch(0, scope, pack), f"check {cell.op} n={cell.n}")
    torch.cuda.synchronize()
    n, k = cell.n, cell.k
    s = min(count, cell.batch)
    w = cell.work[0]
    h = lambda t, per: t[: s * per].double().cpu().numpy()
    out = {"count": s}
    if cell.op == "gemm":
        out["X"] = h(cell.out, n * n)
    elif cell.op == "posv":
        out.update(X=h(w["B"], n), L=h(w["A"], n * n))
    elif cell.op == "trsm":
        out["X"] = h(w["B"], n * k)
    elif cell.op == "getrf_getrs":
        out.update(X=h(w["B"], n), LU=h(w["A"], n * n), ipiv=cell.ipiv[: s * n].cpu().numpy())
    elif cell.op == "rot3":
        out["X"] = h(cell.out, 9)
    else:
        from paper_2609_28179_gb300.cells import NPTS
        out["X"] = h(cell.out, 3 * NPTS)
    return out


def cell_errors(op, n, gpu, ref, s_ref, s):
    """Largest per-problem relative error max|y - y*| / max|y*| over the first
    s problems (the oracle's outputs hold s_ref >= s problems), over every
    floating output (posv: only L's lower triangle is defined), and the
    number of pivot indices that differ from the oracle's."""
    import numpy as np
    err = 0.0
    for key in ("X", "L", "LU"):
        if key not in gpu or key not in ref:
            continue
        per = ref[key].size // s_ref
        yy = gpu[key].reshape(-1)[: s * per].reshape(s, per)
        rr = ref[key].reshape(-1)[: s * per].reshape(s, per)
        if key == "L":
            lower = np.tril(np.ones((n, n), dtype=bool)).T.reshape(-1)  # column-major lower triangle
            yy, rr = yy[:, lower], rr[:, lower]
        num = np.abs(yy - rr).max(1)
        den = np.maximum(np.abs(rr).max(1), 1e-300)
        err = max(err, float((num / den).max()))
    piv = 0
    if "ipiv" in gpu and "ipiv" in ref:
        m = s * n
        piv = int((gpu["ipiv"][:m] != ref["ipiv"][:m]).sum())
    return err, piv


def cpu_baseline(hosts, ops_sizes, batch, budget_s=12.0, gpu=None):
    """Oracle matrices/s over the step's cells, each on an adaptively sized
    sample (scaled to the full batch).  When `gpu` maps a label ("tuned",
    "plain") to the GPU outputs of each cell's first problems, the oracle's
    results on the same problems also give each cell's error (the second
    value: label -> [(rel_err, pivot mismatches, problems compared)])."""
    import oracle
    oracle.build()
    per_cell = budget_s / max(1, len(ops_sizes))
    full_time, samples, refs = 0.0, [], []
    for (op, n), host in zip(ops_sizes, hosts):
        sample = 16
        while True:
            dt, s, out = oracle_cell(op, n, host, batch, sample)
            if dt >= per_cell * 0.5 or s >= batch:
                break
            sample = min(batch, sample * max(2, int(per_cell * 0.6 / max(dt, 1e-4))))
        full_time += dt / s * batch
        samples.append(f"{op}{n}:{s}")
        refs.append((s, out))
    value = len(ops_sizes) * batch / full_time
    cores = oracle.max_threads()
    # the same samples on one core
    one_time = 0.0
    oracle.set_threads(1)
    try:
        for (op, n), host, tag in zip(ops_sizes, hosts, samples):
            s = int(tag.split(":")[1])
            dt, s = oracle_cell_time(op, n, host, batch, s)
            one_time += dt / s * batch
    finally:
        oracle.set_threads(cores)
    errs = {}
    for label, outs in (gpu or {}).items():
        errs[label] = []
        for (op, n), (s, ref), got in zip(ops_sizes, refs, outs):
            cnt = min(s, got["count"])
            e, piv = cell_errors(op, n, got, ref, s, cnt)
            errs[label].append((e, piv, cnt))
    sizes = [int(t.split(":")[1]) for t in samples]
    return {"value": value, "unit": "matrices/s", "cores": cores, "kind": "oracle",
            "value_1core": len(ops_sizes) * batch / one_time,
            "sample": f"per cell an adaptive prefix of its {batch} problems ({min(sizes)}..{max(sizes)} problems, "
                      f"about {budget_s / max(1, len(ops_sizes)):.2f} s of oracle work each; per-cell sizes in the "
                      f"detail file), scaled to the full batch; value_1core: the same samples on one core",
            "per_cell_sample": samples}, errs


# ------------------------------------------------------------- reference
def run_reference(args, rank, world):
    if rank != 0:
        return 0
    import oracle
    from paper_2609_28179_gb300.cells import make_inputs
    oracle.build()
    ops_sizes = [(op, n) for op, n, _ in cell_list(args.ops, args.sizes, args.batch)]
    sample = max(1, args.batch // args.ref_sample_div)
    hosts = [make_inputs(op, n, sample, 1002) for op, n in ops_sizes]
    times = []
    for st in range(args.warmup + args.steps):
        t = 0.0
        for (op, n), h in zip(ops_sizes, hosts):
            dt, _ = oracle_cell_time(op, n, h, sample, sample)
            t += dt
        if st >= args.warmup:
            times.append(t)
    per_step = statistics.mean(times)
    problems = sample * len(ops_sizes)
    value = problems / per_step
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "matrices/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": per_step * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": config_of(args, sample_note=f"oracle sample of {sample} problems per cell"),
            "cpu_baseline": {"value": value, "unit": "matrices/s", "cores": oracle.max_threads(), "kind": "oracle",
                             "sample": f"{sample} of {args.batch} problems per cell, every cell, each step"},
            "e2e": {"value": value, "unit": "matrices/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


def config_of(args, sample_note=None):
    c = {"workload": f"placement sweep: {len(args.ops)} ops x n in {args.sizes} (chain length for rot3/se3, "
                     f"1024 points for se3), batch {args.batch} per cell, tuned placements",
         "ops": args.ops, "sizes": args.sizes, "batch": args.batch,
         "rhs": "posv/getrs 1, trsm n, gemm square n x n x n",
         "l2": "step working set > 1 GB >> 129 MB L2; destructive cells read a fresh input copy every step",
         "streams": getattr(args, "streams", 1)}
    if sample_note:
        c["sample"] = sample_note
    return c


def max_over_ranks(x: float, world: int, device: str = "cuda") -> float:
    """The job's time is the slowest replica's (replicas share no data; the
    only collective is this reduction, outside the timed region)."""
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_value(problems_per_rank: int, world: int, steps: int, ms_max: float) -> float:
    """Whole-job matrices/s: every rank's problems over the slowest rank's time."""
    return problems_per_rank * world * steps / (ms_max / 1e3)


# Source files each operation's kernels are built from: a committed DRAM
# traffic figure stays valid while these files are unchanged.
KERNEL_SOURCES = {
    "gemm": ["common.cuh", "k_gemm.cu", "k_gemm_tc.cu", "dev_umma.cuh"],
    "posv": ["common.cuh", "k_chol_impl.cuh", "k_chol_posv.cu", "dev_chol.cuh", "dev_chol_tc.cuh",
             "dev_rows.cuh", "dev_trsm_tc.cuh"],
    "trsm": ["common.cuh", "k_chol_impl.cuh", "k_chol_trsm.cu", "dev_chol.cuh", "dev_chol_tc.cuh",
             "dev_rows.cuh", "dev_trsm_tc.cuh"],
    "getrf_getrs": ["common.cuh", "k_lu.cu", "dev_lu.cuh", "dev_lu_tc.cuh", "dev_lu_tc2.cuh", "dev_chol_tc.cuh",
                    "dev_rows.cuh"],
    "rot3": ["common.cuh", "k_geom.cu"],
    "se3": ["common.cuh", "k_geom.cu"],
}


def sources_hash(op):
    """Hash of the kernel sources of one operation (KERNEL_SOURCES)."""
    h = hashlib.sha1()
    csrc = os.path.join(ROOT, "paper_2609_28179_gb300", "csrc")
    for f in sorted(KERNEL_SOURCES[op]):
        with open(os.path.join(csrc, f), "rb") as fh:
            h.update(f.encode())
            h.update(fh.read())
    return h.hexdigest()[:12]


def traffic_for(kernel_key):
    """DRAM bytes per launch of a cell's kernel from the committed ncu
    summary (profiles/ncu_traffic.json), or None when that operation's kernel
    sources changed since the capture."""
    p = os.path.join(ROOT, "profiles", "ncu_traffic.json")
    if not os.path.exists(p):
        return None
    with open(p) as f:
        d = json.load(f)
    e = d.get("cells", {}).get(kernel_key)
    if not isinstance(e, dict) or e.get("sources_hash") != sources_hash(kernel_key.split(":")[0]):
        return None
    return e.get("bytes")


# ------------------------------------------------------------ other configs
def _graph_time(fn, reps, iters=5, setup=None):
    """Median ms of `reps` back-to-back calls of fn captured in one graph."""
    import torch
    if setup:
        setup()
    fn()  # warm (module load, attributes) outside capture
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    s = torch.cuda.Stream()
    with torch.cuda.graph(graph, stream=s):
        for _ in range(reps):
            fn()
    out = []
    for _ in range(iters):
        if setup:
            setup()
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        graph.replay()
        b.record()
        torch.cuda.synchronize()
        out.append(a.elapsed_time(b) / reps)
    return statistics.median(out)


def extra_plain_posv(peaks):
    """Plain batched Cholesky factor+solve: 1024 SPD systems, n = 6, one RHS,
    one thread per matrix (no tuning)."""
    import torch
    import paper_2609_28179_gb300 as g
    from paper_2609_28179_gb300 import workloads as W
    from paper_2609_28179_gb300.cells import bytes_flops
    n, batch = 6, 1024
    A = torch.from_numpy(W.spd(n, batch, 1000)).cuda()
    b = torch.from_numpy(W.gaussian(n * batch, 1001)).cuda()
    sets = 64
    As = [A.clone() for _ in range(sets)]
    bs = [b.clone() for _ in range(sets)]
    info = torch.zeros(batch, dtype=torch.int32, device="cuda")
    o = g.make_opts(scope=g.GLASS_SCOPE_THREAD, pack=1)
    k = [0]

    def fn():
        i = k[0] % sets
        k[0] += 1
        g.glass_batched_posv(n, 1, As[i], n, n * n, bs[i], n, n, info, batch, o)

    def setup():
        for x, y in zip(As, bs):
            x.copy_(A)
            y.copy_(b)
    ms = _graph_time(fn, sets, setup=setup)
    by = bytes_flops("posv", n, 1)[0] * batch
    return {"workload": "posv n=6 batch 1024 nrhs 1, one thread per matrix", "us": ms * 1e3,
            "matrices_per_s": batch / (ms / 1e3), "gbs": by / (ms / 1e3) / 1e9,
            "frac_hbm": by / (ms / 1e3) / 1e9 / peaks["hbm_gbs"],
            "note": "3.5 kB per launch: launch/latency bound, not bandwidth bound"}


def extra_varsize(peaks, wpcs=(0, 2, 4, 8)):
    """8192 SPD systems, n ~ U{6..64}, 4 RHS, one persistent launch (with its
    binning kernel) per graph node, replayed."""
    import torch
    import paper_2609_28179_gb300 as g
    from paper_2609_28179_gb300 import workloads as W
    from paper_2609_28179_gb300.cells import bytes_flops
    batch, nrhs = 8192, 4
    sizes = W.varsize_sizes(batch, 1003)
    A, B, offA, offB = W.varsize_pack(sizes, nrhs, 1004)
    dn = torch.from_numpy(sizes).cuda()
    doA, doB = torch.from_numpy(offA).cuda(), torch.from_numpy(offB).cuda()
    A0, B0 = torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda()
    sets = 8
    As = [A0.clone() for _ in range(sets)]
    Bs = [B0.clone() for _ in range(sets)]
    info = torch.zeros(batch, dtype=torch.int32, device="cuda")
    wsb = g.glass_posv_varsize_workspace(batch)
    ws = torch.empty(wsb, dtype=torch.uint8, device="cuda")
    by = sum(bytes_flops("posv", int(n), nrhs)[0] for n in sizes)
    out = {"workload": "8192 SPD systems, n ~ U{6..64}, 4 RHS, persistent posv in a CUDA graph",
           "bytes_per_launch": by, "schedules": {}}

    def setup():
        for x, y in zip(As, Bs):
            x.copy_(A0)
            y.copy_(B0)
    for wpc in wpcs:
        o = g.make_opts(scope=g.GLASS_SCOPE_WARP if wpc else g.GLASS_SCOPE_AUTO, pack=wpc)
        k = [0]

        def fn():
            i = k[0] % sets
            k[0] += 1
            g.glass_posv_varsize(batch, dn, doA, doB, nrhs, As[i], Bs[i], info, ws, wsb, o)
        ms = _graph_time(fn, sets, setup=setup)
        out["schedules"][f"warps_per_cta={wpc or 8}"] = {"us": ms * 1e3, "matrices_per_s": batch / (ms / 1e3),
                                                         "gbs": by / (ms / 1e3) / 1e9,
                                                         "frac_hbm": by / (ms / 1e3) / 1e9 / peaks["hbm_gbs"]}
    best = min(out["schedules"].items(), key=lambda kv: kv[1]["us"])
    out["best"] = {"schedule": best[0], **best[1]}
    return out


def extra_tc_gemm(peaks, batch=65536):
    """Tensor-core batched GEMM, n in {16, 32, 64}, batch 65536, inputs N(0,1);
    fp32_table is the FP32 call at the table's placement (SIMT kernels for
    n = 16, 32; the tcgen05 3xTF32 kernel for n = 64)."""
    import torch
    import paper_2609_28179_gb300 as g
    out = {}
    gen = torch.Generator(device="cuda")
    gen.manual_seed(1004)
    for n in (16, 32, 64):
        A = torch.randn(batch * n * n, generator=gen, device="cuda")
        B = torch.randn(batch * n * n, generator=gen, device="cuda")
        C = torch.empty_like(A)
        Ab, Bb = A.to(torch.bfloat16), B.to(torch.bfloat16)
        for name, math_, dt, a, b, bpe in (("bf16", g.GLASS_MATH_BF16_TC, g.GLASS_BF16, Ab, Bb, 2),
                                           ("tf32", g.GLASS_MATH_TF32_TC, g.GLASS_F32, A, B, 4),
                                           ("3xtf32", g.GLASS_MATH_3XTF32_TC, g.GLASS_F32, A, B, 4),
                                           ("fp32_table", g.GLASS_MATH_FP32, g.GLASS_F32, A, B, 4)):
            o = g.make_opts(dtype=dt, math=math_)
            fn = lambda: g.glass_batched_gemm(n, n, n, a, n, n * n, b, n, n * n, C, n, n * n, batch, o)
            g.check(fn(), f"tc gemm {name}")
            ms = _graph_time(fn, 4)
            by = (2 * bpe + 4) * n * n * batch
            fl = 2 * n ** 3 * batch
            out[f"{name}_n{n}"] = {"us": ms * 1e3, "matrices_per_s": batch / (ms / 1e3),
                                   "gbs": by / (ms / 1e3) / 1e9, "tflops": fl / (ms / 1e3) / 1e12,
                                   "frac_hbm": by / (ms / 1e3) / 1e9 / peaks["hbm_gbs"]}
    return out


def extra_refine(peaks, batch=16384):
    """Refined SPD solve: n in {32, 64}, kappa swept 1e1..1e6 by decades, one refinement
    step with the FP64 residual (x1) and with the compensated FP32 one (x1d);
    forward error of x0, x1 and x1d against the FP64 solution (numpy/LAPACK)
    of the same FP32-rounded systems on a sample, and time at full batch."""
    import numpy as np
    import torch
    import paper_2609_28179_gb300 as g
    from paper_2609_28179_gb300 import workloads as W
    from paper_2609_28179_gb300.cells import bytes_flops
    out = {}
    sample = 128
    for n in (32, 64):
        for kappa in (1e1, 1e2, 1e3, 1e4, 1e5, 1e6):
            A = W.kappa_spd(n, sample, kappa, 1005)
            b = W.gaussian(n * sample, 1006)
            Am = W.from_colmajor(A, sample, n, n).astype(np.float64)
            # FP64 reference solution of the FP32-rounded system (LAPACK via numpy)
            Xs = np.linalg.solve(Am, b.reshape(sample, n, 1).astype(np.float64)).reshape(-1)
            row = {}
            for tag, refine, resid in (("x0", 0, g.GLASS_RESIDUAL_FP64), ("x1", 1, g.GLASS_RESIDUAL_FP64),
                                       ("x1d", 1, g.GLASS_RESIDUAL_DOT2)):
                dA, dB = torch.from_numpy(A).cuda(), torch.from_numpy(b).cuda()
                info = torch.zeros(sample, dtype=torch.int32, device="cuda")
                o = g.make_opts(scope=g.GLASS_SCOPE_WARP, pack=1, refine_steps=refine, fp64_diag=refine,
                                residual=resid)
                g.check(g.glass_batched_posv(n, 1, dA, n, n * n, dB, n, n, info, sample, o))
                X = dB.cpu().numpy().astype(np.float64)
                inf = info.cpu().numpy()
                ok = inf == 0
                fwd = (np.abs(X - Xs).reshape(sample, n).max(1) / np.abs(Xs).reshape(sample, n).max(1))[ok]
                Xm = X.reshape(sample, n, 1)
                bm = b.reshape(sample, n, 1).astype(np.float64)
                R = bm - Am @ Xm
                be = (np.abs(R).max((1, 2)) / (np.abs(Am).sum(2).max(1) * np.abs(Xm).max((1, 2)) +
                                               np.abs(bm).max((1, 2))))[ok]
                row[tag] = {"fwd_err_median": float(np.median(fwd)) if ok.any() else None,
                                     "fwd_err_max": float(fwd.max()) if ok.any() else None,
                                     "bwd_err_max": float(be.max()) if ok.any() else None,
                                     "failed": int((~ok).sum()),
                                     "within_1e-4_fwd": int((fwd <= 1e-4).sum())}
            out[f"n{n}_kappa{kappa:.0e}"] = row
    # time at full batch (kappa 1e3 inputs), refined and plain
    for n in (32, 64):
        A = torch.from_numpy(W.kappa_spd(n, 256, 1e3, 1007)).cuda().repeat(batch // 256)
        b = torch.from_numpy(W.gaussian(n * batch, 1008)).cuda()
        sets = 4
        As = [A.clone() for _ in range(sets)]
        bs = [b.clone() for _ in range(sets)]
        info = torch.zeros(batch, dtype=torch.int32, device="cuda")

        def setup():
            for x, y in zip(As, bs):
                x.copy_(A)
                y.copy_(b)
        for refine, fp64d, resid in ((0, 0, 0), (1, 1, 0), (1, 0, 0), (0, 1, 0), (1, 1, g.GLASS_RESIDUAL_DOT2)):
            o = g.make_opts(refine_steps=refine, fp64_diag=fp64d, residual=resid)
            k = [0]

            def fn():
                i = k[0] % sets
                k[0] += 1
                g.glass_batched_posv(n, 1, As[i], n, n * n, bs[i], n, n, info, batch, o)
            ms = _graph_time(fn, sets, setup=setup)
            by = bytes_flops("posv", n, 1)[0] * batch + (4 * n * batch if refine else 0)
            key = f"time_n{n}_refine{refine}" + ("" if fp64d == refine else f"_fp64diag{fp64d}") + \
                ("_dot2" if resid == g.GLASS_RESIDUAL_DOT2 else "")
            out[key] = {"us": ms * 1e3, "matrices_per_s": batch / (ms / 1e3), "gbs": by / (ms / 1e3) / 1e9}
    return out


def extra_learned():
    """Median / p90 regret of the learned placement model on held-out measured
    points, against nearest-grid table lookup and the best fixed placement
    (the model is trained here, on the GPU, from the committed measurements)."""
    import paper_2609_28179_gb300.learned as Lm
    tdir = os.path.join(ROOT, "paper_2609_28179_gb300", "tuning")
    tr, ho = os.path.join(tdir, "sm103_random_train.jsonl"), os.path.join(tdir, "sm103_random_heldout.jsonl")
    if not (os.path.exists(tr) and os.path.exists(ho)):
        return {"unavailable": "no committed random-point measurements"}
    train_pts, held = Lm.load_points(tr), Lm.load_points(ho)
    t0 = time.perf_counter()
    w, mu, sd, losses = Lm.train(train_pts, epochs=300)
    res = Lm.evaluate(w, mu, sd, train_pts, held)
    res["train_seconds"] = time.perf_counter() - t0
    res["final_loss"] = losses[-1]
    return res


def measure_peaks():
    """Measured pipe peaks (TFLOP/s) from the library's throughput probes:
    FP32 FFMA, FP64 DFMA, TF32 m16n8k8 and BF16 m16n8k16 mma.sync; each
    launch sized to about 2 ms, the best of 5 launches."""
    import torch
    import paper_2609_28179_gb300 as g
    sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    blocks, threads = sms * 8, 256
    sink = torch.empty(blocks * threads, dtype=torch.float64, device="cuda")
    out = {}

    def once(kind, iters):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        st, fl = g.glass_peak_probe(kind, iters, blocks, threads, sink)
        b.record()
        torch.cuda.synchronize()
        g.check(st, "peak probe")
        return a.elapsed_time(b), fl
    for kind, name in ((0, "fp32_ffma"), (1, "fp64_dfma"), (2, "tf32_mma_m16n8k8"), (3, "bf16_mma_m16n8k16")):
        iters = 16
        for _ in range(4):
            ms, _ = once(kind, iters)
            if ms >= 1.0:
                break
            iters = int(min(1 << 22, max(iters * 2, iters * 2.0 / max(ms, 1e-3))))
        best = min(once(kind, iters) for _ in range(5))
        out[name] = {"tflops": best[1] / (best[0] / 1e3) / 1e12, "ms": best[0], "iters": iters,
                     "grid": f"{blocks}x{threads}"}
    return out


def extra_latency(ops=None, sizes=(6, 64), batches=(1, 1024, 16384)):
    """Per-call latency: one launch on a cold L2 (a 512 MB buffer written
    between calls), timed with events; the median of 5."""
    import torch
    import paper_2609_28179_gb300 as g
    from paper_2609_28179_gb300.cells import OPS, Cell
    flush = torch.empty(512 << 20, dtype=torch.uint8, device="cuda")
    out = {}
    for op in ops or OPS:
        for n in sizes:
            for batch in batches:
                cell = Cell(op, n, batch, sets=1, device_inputs=True, seed=2000 + n)
                g.check(cell.launch(0), f"latency {op} {n}")
                ts = []
                for _ in range(5):
                    cell.restore()
                    flush.fill_(1)
                    torch.cuda.synchronize()
                    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    a.record()
                    cell.launch(0)
                    b.record()
                    torch.cuda.synchronize()
                    ts.append(a.elapsed_time(b) * 1e3)
                out[f"{op}:n{n}:b{batch}"] = round(statistics.median(ts), 2)
                del cell
        torch.cuda.empty_cache()
    return {"unit": "us per call (cold L2, single launch, table placement)", "cells": out}


def extra_batch_scaling(peaks, ops=("gemm", "posv", "getrf_getrs"), sizes=(16, 64),
                        batches=(16384, 65536, 262144, 1048576)):
    """Where the HBM roofline becomes reachable: the matrix operations at
    batches up to 2^20 (table placement; inputs restored between launches,
    untimed)."""
    import torch
    from paper_2609_28179_gb300.cells import Cell
    out = {}
    for op in ops:
        for n in sizes:
            for batch in batches:
                cell = Cell(op, n, batch, sets=1, device_inputs=True, seed=3000 + n)
                ms = _graph_time(lambda: cell.launch(0), 1, iters=5, setup=cell.restore)
                out[f"{op}:n{n}:b{batch}"] = {"us": round(ms * 1e3, 2), "matrices_per_s": batch / (ms / 1e3),
                                              "gbs": cell.bytes / (ms / 1e3) / 1e9,
                                              "frac_hbm": cell.bytes / (ms / 1e3) / 1e9 / peaks["hbm_gbs"]}
                del cell
                torch.cuda.empty_cache()
    return out


def extra_riccati(peaks, batches=(64, 16384)):
    """LQR feedback gain K = (R + B^T P B)^{-1} B^T P A at the workload's
    (nx, nu) pairs: the fused kernel at every feasible placement against the
    composition of primitive calls, and what the table resolves."""
    import paper_2609_28179_gb300 as g
    from paper_2609_28179_gb300 import workloads as W
    from paper_2609_28179_gb300.tune import COMPOSED, RiccatiCell
    out = {}
    for nx, nu in W.RICCATI_SIZES:
        for batch in batches:
            cell = RiccatiCell(nx, nu, batch)
            times = {}
            for scope, pack in cell.placements():
                g.check(cell.launch(scope, pack), "riccati")
                times[f"{g.SCOPE_NAMES[scope]}x{pack}"] = _graph_time(lambda: cell.launch(scope, pack), 8) * 1e3
            auto_us = _graph_time(lambda: cell.launch(), 8) * 1e3
            fused = {k: v for k, v in times.items() if not k.startswith("composed")}
            bf = min(fused, key=fused.get)
            out[f"{nx}x{nu}:b{batch}"] = {
                "fused_best": bf, "fused_us": round(fused[bf], 2), "composed_us": round(times["composedx1"], 2),
                "composed_over_fused": times["composedx1"] / fused[bf], "auto_us": round(auto_us, 2),
                "auto_placement": "{}x{}".format(*(lambda s: (g.SCOPE_NAMES[s[1][0]], s[1][1]))(
                    g.glass_riccati_placement(nx, nu, batch, True))),
                "matrices_per_s_auto": batch / (auto_us / 1e6),
                "gbs_auto": cell.bytes / (auto_us / 1e6) / 1e9}
            del cell
    return out


def extra_robo(peaks, batches=(4096, 1 << 20)):
    """Robotics operations of the placement table (quaternion/SE(3)
    retractions and error, motion cross product, eig3, svd3, closest
    rotation, argmax and softmax at n = 16): ns per problem at the best
    placement of each scope, as the paper tabulates them, and the table's."""
    import paper_2609_28179_gb300 as g
    from paper_2609_28179_gb300.tune import ROBO_N, RoboCell
    out = {}
    for op, name in enumerate(g.ROBO_OPS):
        for batch in batches:
            cell = RoboCell(op, batch)
            per_scope = {}
            for scope in (0, 1, 2):
                best = None
                for pack in (1, 2, 4, 8):
                    if not g.glass_robo_feasible(op, ROBO_N, scope, pack):
                        continue
                    g.check(cell.launch(scope, pack), name)
                    us = _graph_time(lambda: cell.launch(scope, pack), 16) * 1e3
                    if best is None or us < best[0]:
                        best = (us, pack)
                if best is not None:  # element-wise operations are thread scope only
                    per_scope[g.SCOPE_NAMES[scope]] = {"ns_per_problem": best[0] * 1e3 / batch, "pack": best[1]}
            us = _graph_time(lambda: cell.launch(), 16) * 1e3
            out[f"{name}:b{batch}"] = {"scopes": per_scope, "table_ns_per_problem": us * 1e3 / batch,
                                       "table_gbs": cell.bytes / (us / 1e6) / 1e9,
                                       "table_frac_hbm": cell.bytes / (us / 1e6) / 1e9 / peaks["hbm_gbs"]}
            del cell
    return out


def extra_blas(peaks):
    """Batched dot and GEMV, and the block-tridiagonal matvec and solve of
    trajectory optimization (symmetric, N blocks of nb x nb: N = horizon,
    nb = state size), table/auto placements, inputs restored untimed."""
    import numpy as np
    import torch
    import paper_2609_28179_gb300 as g
    out = {}
    gen = torch.Generator(device="cuda")
    gen.manual_seed(1010)
    for n, batch in ((16, 1 << 20), (64, 1 << 20)):
        x = torch.randn(batch * n, generator=gen, device="cuda")
        y = torch.randn(batch * n, generator=gen, device="cuda")
        o = torch.empty(batch, device="cuda")
        ms = _graph_time(lambda: g.glass_batched_dot(n, x, n, y, n, o, batch), 8)
        by = 4 * batch * (2 * n + 1)
        out[f"dot:n{n}:b{batch}"] = {"us": ms * 1e3, "gbs": by / (ms / 1e3) / 1e9,
                                     "frac_hbm": by / (ms / 1e3) / 1e9 / peaks["hbm_gbs"]}
    for n, batch in ((16, 1 << 18), (64, 1 << 16)):
        A = torch.randn(batch * n * n, generator=gen, device="cuda")
        x = torch.randn(batch * n, generator=gen, device="cuda")
        y = torch.empty(batch * n, device="cuda")
        ms = _graph_time(lambda: g.glass_batched_gemv(0, n, n, 1.0, A, n, n * n, x, n, 0.0, y, n, batch), 8)
        by = 4 * batch * (n * n + 2 * n)
        out[f"gemv:n{n}:b{batch}"] = {"us": ms * 1e3, "gbs": by / (ms / 1e3) / 1e9,
                                      "frac_hbm": by / (ms / 1e3) / 1e9 / peaks["hbm_gbs"]}
    for nb, N, batch in ((6, 32, 4096), (12, 32, 4096), (16, 64, 4096)):
        r = np.random.default_rng(1011)
        M = r.standard_normal((batch, N, nb, nb)).astype(np.float32)
        D0 = torch.from_numpy(np.ascontiguousarray(
            (M @ M.transpose(0, 1, 3, 2) + (2 * nb + 2) * np.eye(nb, dtype=np.float32)).transpose(0, 1, 3, 2))).cuda()
        O0 = torch.randn(batch * (N - 1) * nb * nb, generator=gen, device="cuda")
        b0 = torch.randn(batch * N * nb, generator=gen, device="cuda")
        D, O, b = D0.clone().reshape(-1), O0.clone(), b0.clone()
        info = torch.empty(batch, dtype=torch.int32, device="cuda")
        y = torch.empty_like(b0)

        def setup():
            D.copy_(D0.reshape(-1))
            O.copy_(O0)
            b.copy_(b0)
        ms_mv = _graph_time(lambda: g.glass_batched_btd_matvec(nb, N, D0, O0, b0, y, batch), 8)
        ms_sv = _graph_time(lambda: g.glass_batched_btd_posv(nb, N, D, O, b, info, batch), 1, setup=setup)
        by = 4 * batch * ((2 * N - 1) * nb * nb + 2 * N * nb)
        out[f"btd:nb{nb}:N{N}:b{batch}"] = {
            "matvec_us": ms_mv * 1e3, "matvec_gbs": by / (ms_mv / 1e3) / 1e9,
            "posv_us": ms_sv * 1e3, "posv_systems_per_s": batch / (ms_sv / 1e3),
            "posv_gbs": 2 * by / (ms_sv / 1e3) / 1e9}
    return out


def extra_fp64(peaks, sizes=(6, 32, 64), batch=16384):
    """FP64 storage variants at the table's placement: time, GB/s and the
    fraction of the measured FP64 FMA peak (glass_peak_probe kind 1)."""
    from paper_2609_28179_gb300.cells import bytes_flops
    from paper_2609_28179_gb300.tune import F64_OPS, F64Cell
    pk = measure_peaks()["fp64_dfma"]["tflops"]
    out = {"fp64_peak_tflops": pk}
    for op in F64_OPS:
        for n in sizes:
            cell = F64Cell(op, n, batch, sets=4)
            k = [0]

            def fn():
                cell.launch(k[0] % 4)
                k[0] += 1
            ms = _graph_time(fn, 4, setup=cell.restore)
            fl = bytes_flops(op, n)[1] * batch
            out[f"{op}:n{n}:b{batch}"] = {"us": round(ms * 1e3, 2), "gbs": cell.bytes / (ms / 1e3) / 1e9,
                                          "frac_hbm": cell.bytes / (ms / 1e3) / 1e9 / peaks["hbm_gbs"],
                                          "gflops": fl / (ms / 1e3) / 1e9, "frac_fp64": fl / (ms / 1e3) / 1e12 / pk}
            del cell
    return out


def run_extras(peaks, which):
    out = {}
    for name, fn in (("plain_posv_n6", lambda: extra_plain_posv(peaks)), ("mixed_size", lambda: extra_varsize(peaks)),
                     ("tensor_core_gemm", lambda: extra_tc_gemm(peaks)), ("refined_posv", lambda: extra_refine(peaks)),
                     ("learned_placement", extra_learned), ("latency", extra_latency),
                     ("batch_scaling", lambda: extra_batch_scaling(peaks)),
                     ("riccati_gain", lambda: extra_riccati(peaks)), ("robotics_ops", lambda: extra_robo(peaks)),
                     ("blas_block_tridiagonal", lambda: extra_blas(peaks)), ("fp64_storage", lambda: extra_fp64(peaks))):
        if which != "all" and name not in which.split(","):
            continue
        try:
            out[name] = fn()
        except Exception as e:  # report, do not hide: the line says what failed
            out[name] = {"error": f"{type(e).__name__}: {e}"}
    return out


# ------------------------------------------------------------------ main
def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="glass", choices=["glass", "reference"])
    ap.add_argument("--batch", type=int, default=BATCH)
    ap.add_argument("--ops", nargs="+", default=None)
    ap.add_argument("--sizes", nargs="+", type=int, default=None)
    ap.add_argument("--no-cpu", action="store_true", help="skip the oracle CPU baseline")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--ref-sample-div", type=int, default=64)
    ap.add_argument("--extras", default="all", help="comma list of extra configs, 'all' or 'none'")
    ap.add_argument("--detail", default=None, help="file for the per-cell rows and the extra configs' records")
    ap.add_argument("--streams", type=int, default=3,
                    help="streams the step graph forks into (the cells are independent; 3 measured best of 1-8)")
    args = ap.parse_args()
    from paper_2609_28179_gb300.cells import OPS, SWEEP_N
    args.ops = args.ops or OPS
    args.sizes = args.sizes or SWEEP_N
    args.warmup = max(3, args.warmup)

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        return run_reference(args, rank, world)

    import torch
    import torch.distributed as dist
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    from paper_2609_28179_gb300 import _build
    if rank == 0 or world == 1:
        _build.build()
    if world > 1:
        dist.barrier()
    import paper_2609_28179_gb300 as g
    from paper_2609_28179_gb300.cells import Cell
    g.lib()

    sets = args.steps + args.warmup
    cells = [Cell(op, n, b, sets=sets) for op, n, b in cell_list(args.ops, args.sizes, args.batch)]
    tuned = [resolved_placement(c) for c in cells]
    plain = [plain_placement(c) for c in cells]

    def barrier():
        if world > 1:
            dist.barrier()

    # tuned step (the headline), clocks sampled during the timed region
    barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as cs:
        t_tuned, per_tuned = time_steps(cells, tuned, args.steps, args.warmup, barrier, args.streams)
    clocks = cs.summary()
    barrier()
    for c in cells:
        c.restore()
    torch.cuda.synchronize()
    t_plain, per_plain = time_steps(cells, plain, args.steps, args.warmup, barrier, args.streams)
    t_e2e = h2d = d2h = None
    if not args.no_e2e:
        t_e2e, h2d, d2h = e2e_steps(cells, args.steps, args.warmup)

    t_tuned, t_plain = max_over_ranks(t_tuned, world), max_over_ranks(t_plain, world)
    if t_e2e is not None:
        t_e2e = max_over_ranks(t_e2e, world)
    problems = len(cells) * args.batch * world
    ms_step = t_tuned / args.steps
    value = replica_value(len(cells) * args.batch, world, args.steps, t_tuned)

    peaks = load_peaks()
    sms = torch.cuda.get_device_properties(local).multi_processor_count
    pipes = measure_peaks()
    fp32_peak = pipes["fp32_ffma"]["tflops"]
    rows = []
    for c, (s, p), us_t, (ps, pp), us_p in zip(cells, tuned, per_tuned, plain, per_plain):
        t_bw = c.bytes / (peaks["hbm_gbs"] * 1e9)
        t_fl = c.flops / (fp32_peak * 1e12)  # measured FFMA peak
        bound = "hbm" if t_bw >= t_fl else "alu"
        t_roof = max(t_bw, t_fl)
        rows.append({"op": c.op, "n": c.n, "placement": f"{g.SCOPE_NAMES[s]}x{p}", "us": round(us_t * 1e3, 2),
                     "matrices_per_s": c.batch / (us_t / 1e3), "gbs": c.bytes / (us_t / 1e3) / 1e9,
                     "gflops": c.flops / (us_t / 1e3) / 1e9, "bound": bound,
                     "frac": t_roof / (us_t / 1e3), "plain": f"{g.SCOPE_NAMES[ps]}x{pp}",
                     "plain_us": round(us_p * 1e3, 2), "speedup_vs_plain": us_p / us_t})
    dom = max(range(len(cells)), key=lambda i: per_tuned[i])
    dc, dr = cells[dom], rows[dom]
    dur = per_tuned[dom] / 1e3
    if dr["bound"] == "hbm":
        roof = {"bound": "hbm", "achieved": dc.bytes / dur / 1e9, "peak": peaks["hbm_gbs"], "unit": "GB/s"}
    else:
        roof = {"bound": "alu", "achieved": dc.flops / dur / 1e12, "peak": fp32_peak, "unit": "TFLOP/s"}
    roof["frac"] = roof["achieved"] / roof["peak"]
    roof["peak_src"] = (f"{peaks['src']} HBM copy" if roof["bound"] == "hbm" else
                        "measured FP32 FFMA probe (glass_peak_probe)")
    key = f"{dc.op}:{dc.n}:{dr['placement']}"
    roof["kernel"] = key
    roof["traffic"] = traffic_for(key)
    roof["algorithmic_bytes"] = dc.bytes
    roof["us_per_launch"] = round(per_tuned[dom] * 1e3, 2)
    roof["step_share"] = per_tuned[dom] / sum(per_tuned)
    line = {"metric": METRIC, "value": value, "unit": "matrices/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": config_of(args), "roofline": roof, "gpu_launches": len(cells) * args.steps,
            "clocks": clocks,
            "plain": {"value": problems * args.steps / (t_plain / 1e3), "ms_per_step": t_plain / args.steps,
                      "speedup_tuned_over_plain": t_plain / t_tuned},
            "hbm_weighted_frac": sum(r["frac"] * r["us"] for r in rows) / sum(r["us"] for r in rows)}
    if t_e2e is not None:
        line["e2e"] = {"value": problems * args.steps / (t_e2e / 1e3), "unit": "matrices/s",
                       "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                       "ms_per_step": t_e2e / args.steps}
    detail = {"cells": rows, "peaks": {"hbm_gbs": peaks["hbm_gbs"], "hbm_src": peaks["src"], **pipes,
                                       "fp32_nominal_tflops": fp32_peak_tflops(sms, peaks["sm_max_mhz"])}}
    if rank == 0 and not args.no_cpu:
        outs = {lab: [gpu_outputs(c, pl, CHECK_PROBLEMS) for c, pl in zip(cells, pls)]
                for lab, pls in (("tuned", tuned), ("plain", plain))}
        cb, errs = cpu_baseline([c.host for c in cells], [(c.op, c.n) for c in cells], args.batch, gpu=outs)
        detail["cpu_baseline_samples"] = cb.pop("per_cell_sample")
        line["cpu_baseline"] = cb
        for lab, es in errs.items():
            for r, (e, piv, cnt) in zip(rows, es):
                r[f"err_{lab}"] = e
                r[f"ipiv_mismatch_{lab}"] = piv
                r["err_problems"] = cnt
        line["accuracy"] = accuracy_summary(rows)
    if rank == 0 and args.extras != "none":
        detail["extras"] = run_extras(peaks, args.extras)
        line["extras"] = summarize_extras(detail["extras"])
    if rank == 0:
        line["top_cells"] = [f"{r['op']}:{r['n']} {r['placement']} {r['us']}us frac {r['frac']:.2f}"
                             for r in sorted(rows, key=lambda r: -r["us"])[:6]]
        path = write_detail(args, detail)
        line["detail_file"] = path
        for r in sorted(rows, key=lambda r: -r["us"]):
            print(f"  {r['op']:>12} n={r['n']:<3} {r['placement']:>7} {r['us']:9.2f} us  {r['gbs']:7.0f} GB/s  "
                  f"frac {r['frac']:.3f}  plain {r['plain_us']:9.2f} us  err {r.get('err_tuned', float('nan')):.1e}",
                  file=sys.stderr)
        print(json.dumps(line))
    if world > 1:
        dist.destroy_process_group()
    return 0


CHECK_PROBLEMS = 256   # problems per cell compared with the oracle (a prefix of the batch)
ERR_BAR = 1e-4


def accuracy_summary(rows):
    """Worst per-problem relative error of the tuned and plain results over
    every cell, against the FP64 oracle on the same inputs."""
    out = {"bar": ERR_BAR, "cells": len(rows),
           "sample": f"first min({CHECK_PROBLEMS}, oracle sample) problems of every cell, every output"}
    for lab in ("tuned", "plain"):
        es = [(r.get(f"err_{lab}"), r) for r in rows if r.get(f"err_{lab}") is not None]
        if not es:
            continue
        worst = max(es, key=lambda x: x[0])
        out[f"{lab}_max_rel_err"] = worst[0]
        out[f"{lab}_worst_cell"] = f"{worst[1]['op']}:{worst[1]['n']}"
        out[f"{lab}_cells_within_bar"] = sum(1 for e, _ in es if e <= ERR_BAR)
        out[f"{lab}_ipiv_mismatches"] = sum(r.get(f"ipiv_mismatch_{lab}", 0) for _, r in es)
    return out


def summarize_extras(ex):
    """A few headline numbers of the other configurations for the result
    line (the full records go to the detail file)."""
    out = {}

    def pick(name, fn):
        try:
            v = fn(ex[name])
            if v is not None:
                out[name] = v
        except Exception as e:  # report, do not hide
            out[name] = {"error": f"{type(e).__name__}: {e}"[:200]}
    pick("plain_posv_n6", lambda d: {"us": round(d["us"], 2), "matrices_per_s": d["matrices_per_s"]})
    pick("mixed_size", lambda d: {k: d["best"][k] for k in ("schedule", "us", "matrices_per_s", "frac_hbm")})
    pick("tensor_core_gemm", lambda d: {k: {"us": round(v["us"], 1), "frac_hbm": round(v["frac_hbm"], 3)}
                                        for k, v in d.items() if k.endswith("n64")})
    pick("refined_posv", lambda d: {
        **{f"n{n}_refined_over_plain": d[f"time_n{n}_refine1"]["us"] / d[f"time_n{n}_refine0"]["us"]
           for n in (32, 64)},
        **{f"n{n}_refined_fp32diag_over_plain": d[f"time_n{n}_refine1_fp64diag0"]["us"] / d[f"time_n{n}_refine0"]["us"]
           for n in (32, 64)},
        **{f"n{n}_refined_dot2_over_plain": d[f"time_n{n}_refine1_dot2"]["us"] / d[f"time_n{n}_refine0"]["us"]
           for n in (32, 64)},
        **{k: {"x0_fwd_med": v["x0"]["fwd_err_median"], "x1_fwd_med": v["x1"]["fwd_err_median"],
               "x1d_fwd_med": v["x1d"]["fwd_err_median"], "x1_bwd_max": v["x1"]["bwd_err_max"],
               "x1d_bwd_max": v["x1d"]["bwd_err_max"], "x1_failed": v["x1"]["failed"]}
           for k, v in d.items() if k.startswith("n64_kappa")}})
    pick("learned_placement", lambda d: {k: {"median_regret": round(d[k]["median"], 4), "p90_regret": round(d[k]["p90"], 4)}
                                         for k in ("learned", "nearest_grid_table", "fixed_placement")})
    return out


def write_detail(args, detail):
    """Per-cell rows and the full records of the other configurations go to
    a JSON file (--detail, default gpurun_out/bench_detail.json under the
    repository if that folder exists, else the system's temporary folder)."""
    path = args.detail
    if not path:
        d = os.path.join(ROOT, "gpurun_out")
        path = os.path.join(d if os.path.isdir(d) else tempfile.gettempdir(), "bench_detail.json")
    try:
        with open(path, "w") as f:
            json.dump(detail, f)
        return path
    except OSError as e:
        return f"unwritten: {e}"


if __name__ == "__main__":
    sys.exit(main())
