"""Offline autotuner and placement-table code generator (Sec. III-A: the
library "benchmarks ... offline on a target GPU and stores the resulting
choices in architecture-specific tables"; Sec. IV-A sweep protocol).

Measurement of one (cell, placement): R back-to-back launches are captured
in one CUDA graph (so host launch overhead is not measured), the graph is
replayed `iters` times with CUDA events on the launching stream, and the
median per-launch time is kept together with every raw sample.  R is large
enough that R launches stream at least twice the L2 size for large cells
(or at least 16 launches), and destructive operations read a fresh copy of
their input on every launch of the graph (restored untimed between
replays).  Placement order is shuffled per cell.

Selection: the fastest placement, except that any placement within the
5 % dispatch margin of it (Sec. IV-A) that uses fewer resources wins --
thread < warp < block, then the smaller pack.

Usage (on the GPU):
  python -m paper_2609_28179_gb300.tune sweep   [--out FILE]   # placement grid
  python -m paper_2609_28179_gb300.tune random  --count N --seed S --out FILE
  python -m paper_2609_28179_gb300.tune codegen [--inp FILE]   # -> csrc/placement_table.h
  python -m paper_2609_28179_gb300.tune launch  --cells op:n:batch[:scope:pack] ...
      (one launch of each cell, for profilers; default placement = the table's)
"""
from __future__ import annotations

import argparse
import json
import math
import os
import random
import statistics
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
TUNING = os.path.join(HERE, "tuning")
GRID_FILE = os.path.join(TUNING, "sm103_grid.jsonl")
TABLE_H = os.path.join(HERE, "csrc", "placement_table.h")
L2_BYTES = 126 * 1024 * 1024
MARGIN = 0.05


def _reps(cell_bytes: int) -> int:
    return int(min(64, max(16, math.ceil(2 * L2_BYTES / max(1, cell_bytes)))))


def measure(cell, placements, iters: int = 5, rng: random.Random | None = None):
    """Median per-launch microseconds of each feasible placement of `cell`."""
    import torch
    import paper_2609_28179_gb300 as g
    out = {}
    order = list(placements)
    (rng or random).shuffle(order)
    R = _reps(cell.bytes)
    stream = torch.cuda.Stream()
    for scope, pack in order:
        if not cell.feasible(scope, pack):
            continue
        # warm (loads the module, sets smem attributes) outside capture
        g.check(cell.launch(0, scope, pack), f"{cell.op} n={cell.n} {scope}x{pack}")
        cell.restore()
        torch.cuda.synchronize()
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph, stream=stream):
            for r in range(R):
                cell.launch(r, scope, pack)
        samples = []
        for _ in range(iters):
            cell.restore()
            torch.cuda.synchronize()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            graph.replay()
            b.record()
            torch.cuda.synchronize()
            samples.append(a.elapsed_time(b) * 1e3 / R)
        del graph
        out[(scope, pack)] = {"us": statistics.median(samples), "samples": samples, "reps": R}
    return out


def choose(meas: dict):
    """Best placement with the dispatch-margin tie-break; meas keyed by (scope, pack)."""
    best = min(v["us"] for v in meas.values())
    ok = [k for k, v in meas.items() if v["us"] <= best * (1 + MARGIN)]
    return min(ok, key=lambda k: (k[0], k[1]))


def _sets_for(op, n, batch):
    from paper_2609_28179_gb300.cells import DESTRUCTIVE, bytes_flops
    if op not in DESTRUCTIVE:
        return 1
    return _reps(bytes_flops(op, n)[0] * batch)


def sweep(out_path: str, ops=None, sizes=None, batches=None, seed: int = 7, iters: int = 5):
    import torch
    import paper_2609_28179_gb300 as g
    from paper_2609_28179_gb300.cells import OPS, SWEEP_B, SWEEP_N, Cell
    g.lib()
    rng = random.Random(seed)
    os.makedirs(os.path.dirname(out_path) or ".", exist_ok=True)
    with open(out_path, "w") as f:
        for op in ops or OPS:
            for n in sizes or SWEEP_N:
                for batch in batches or SWEEP_B:
                    cell = Cell(op, n, batch, sets=_sets_for(op, n, batch), device_inputs=True, seed=seed + n)
                    meas = measure(cell, g.PLACEMENTS, iters=iters, rng=rng)
                    for (s, p), v in meas.items():
                        f.write(json.dumps({"op": op, "n": n, "k": cell.k, "batch": batch, "scope": s, "pack": p,
                                            **v}) + "\n")
                    f.flush()
                    del cell
                    torch.cuda.empty_cache()
                    best = choose(meas)
                    print(f"{op:12s} n={n:3d} B={batch:6d} best={g.SCOPE_NAMES[best[0]]}x{best[1]} "
                          f"{meas[best]['us']:.2f}us", flush=True)


def random_points(out_path: str, count: int, seed: int, iters: int = 3):
    """Measure all 12 placements at `count` random (op, n, batch) points of
    the four matrix operations: n ~ U{3..64}, batch log-uniform in
    [1, 65536].  Points are grouped by (op, n) so that one device pool of
    inputs serves all batches of that pair."""
    import torch
    import paper_2609_28179_gb300 as g
    from paper_2609_28179_gb300.cells import Cell
    g.lib()
    rng = random.Random(seed)
    ops = ["gemm", "posv", "trsm", "getrf_getrs"]
    pts = [(rng.choice(ops), rng.randint(3, 64), int(round(2 ** rng.uniform(0, 16)))) for _ in range(count)]
    groups = {}
    for i, (op, n, b) in enumerate(pts):
        groups.setdefault((op, n), []).append((i, b))
    rows = [None] * count
    for (op, n), items in sorted(groups.items()):
        bmax = max(b for _, b in items)
        pool = Cell(op, n, bmax, sets=1, device_inputs=True, seed=seed * 1000 + n)
        for i, b in items:
            cell = _prefix_cell(pool, b)
            meas = measure(cell, g.PLACEMENTS, iters=iters, rng=rng)
            rows[i] = {"op": op, "n": n, "k": cell.k, "batch": b,
                       "us": {f"{s}x{p}": v["us"] for (s, p), v in meas.items()}}
            del cell
        del pool
        torch.cuda.empty_cache()
    with open(out_path, "w") as f:
        for r in rows:
            f.write(json.dumps(r) + "\n")


def _prefix_cell(pool, batch):
    """A cell over the first `batch` problems of a pool, with its own fresh
    copies for destructive operations."""
    import torch
    from paper_2609_28179_gb300.cells import DESTRUCTIVE, Cell, bytes_flops
    c = Cell.__new__(Cell)
    c.op, c.n, c.batch, c.k, c.dev = pool.op, pool.n, batch, pool.k, pool.dev
    c.host = None
    per = {key: v.numel() // pool.batch for key, v in pool.pristine.items()}
    c.pristine = {key: v[: per[key] * batch] for key, v in pool.pristine.items()}
    sets = _reps(bytes_flops(c.op, c.n)[0] * batch) if c.op in DESTRUCTIVE else 1
    c.sets = sets
    c.work = [{key: v.clone() for key, v in c.pristine.items()} for _ in range(sets)] \
        if c.op in DESTRUCTIVE else [c.pristine]
    c.out = None if pool.out is None else torch.empty(pool.out.numel() // pool.batch * batch,
                                                      dtype=torch.float32, device=c.dev)
    c.info = torch.zeros(max(1, batch), dtype=torch.int32, device=c.dev)
    c.ipiv = torch.zeros(max(1, batch * c.n), dtype=torch.int32, device=c.dev)
    c.bytes, c.flops = bytes_flops(c.op, c.n)
    c.bytes *= batch
    c.flops *= batch
    return c


def load_grid(path: str = GRID_FILE):
    cells = {}
    with open(path) as f:
        for line in f:
            r = json.loads(line)
            cells.setdefault((r["op"], r["n"], r["batch"]), {})[(r["scope"], r["pack"])] = r
    return cells


def codegen(inp: str = GRID_FILE, out: str = TABLE_H):
    from paper_2609_28179_gb300.cells import OPS, SWEEP_B, SWEEP_N
    cells = load_grid(inp)
    rows = []
    for op in OPS:
        per_n = []
        for n in SWEEP_N:
            codes = []
            for b in SWEEP_B:
                meas = cells[(op, n, b)]
                s, p = choose(meas)
                codes.append(str(s * 4 + int(math.log2(p))))
            per_n.append("{" + ", ".join(codes) + "}")
        rows.append(f"    /* {op} */ {{" + ", ".join(per_n) + "},")
    text = f"""// placement_table.h -- GENERATED by paper_2609_28179_gb300/tune.py; do not edit.
// Placement per (op, n, batch) cell: code = scope * 4 + log2(pack), scope
// 0 thread / 1 warp / 2 block (Sec. III-A: offline-measured, compile-time
// resolved placement tables).  For the geometry ops n is the chain length.
// source: {os.path.relpath(inp, os.path.dirname(HERE))} (GB300 measurements, 5 % dispatch margin)
#pragma once
namespace glass {{
static const int kTableNumN = {len(SWEEP_N)};
static const int kTableN[{len(SWEEP_N)}] = {{{", ".join(map(str, SWEEP_N))}}};
static const int kTableNumB = {len(SWEEP_B)};
static const int kTableB[{len(SWEEP_B)}] = {{{", ".join(map(str, SWEEP_B))}}};
static const unsigned char kTable[{len(OPS)}][{len(SWEEP_N)}][{len(SWEEP_B)}] = {{
{chr(10).join(rows)}
}};
}}  // namespace glass
"""
    with open(out, "w") as f:
        f.write(text)
    return out


def launch_cells(specs):
    """One launch of each cell 'op:n:batch[:scope:pack]' (device inputs)."""
    import torch
    import paper_2609_28179_gb300 as g
    from paper_2609_28179_gb300.cells import Cell
    g.lib()
    for spec in specs:
        parts = spec.split(":")
        op, n, batch = parts[0], int(parts[1]), int(parts[2])
        scope, pack = (int(parts[3]), int(parts[4])) if len(parts) == 5 else (g.GLASS_SCOPE_AUTO, 0)
        cell = Cell(op, n, batch, sets=1, device_inputs=True)
        g.check(cell.launch(0, scope, pack), spec)
        torch.cuda.synchronize()
        del cell
        torch.cuda.empty_cache()
        print("launched", spec, flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("cmd", choices=["sweep", "random", "codegen", "launch"])
    ap.add_argument("--cells", nargs="+", default=[])
    ap.add_argument("--out", default=None)
    ap.add_argument("--inp", default=GRID_FILE)
    ap.add_argument("--count", type=int, default=5000)
    ap.add_argument("--seed", type=int, default=11)
    ap.add_argument("--ops", nargs="+", default=None)
    args = ap.parse_args()
    if args.cmd == "sweep":
        sweep(args.out or GRID_FILE, ops=args.ops)
    elif args.cmd == "random":
        random_points(args.out or os.path.join(TUNING, f"sm103_random_{args.seed}.jsonl"), args.count, args.seed)
    elif args.cmd == "launch":
        launch_cells(args.cells)
    else:
        print(codegen(args.inp))


if __name__ == "__main__":
    sys.exit(main())
