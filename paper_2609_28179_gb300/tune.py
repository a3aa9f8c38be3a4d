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
  python -m paper_2609_28179_gb300.tune riccati [--out FILE]   # LQR gain: fused vs composed
  python -m paper_2609_28179_gb300.tune riccati-codegen        # -> csrc/riccati_table.h
  python -m paper_2609_28179_gb300.tune robo [--out FILE]      # robotics ops (Table II)
  python -m paper_2609_28179_gb300.tune robo-codegen           # -> csrc/robo_table.h
  python -m paper_2609_28179_gb300.tune fp64 [--out FILE]      # FP64 storage variants
  python -m paper_2609_28179_gb300.tune fp64-codegen           # -> csrc/fp64_table.h
"""
from __future__ import annotations

import argparse
import json
import math
import os
import random
import statistics
import sys

import numpy as np

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
    from paper_2609_28179_gb300.cells import OPS, SWEEP_B, TABLE_N, Cell
    g.lib()
    rng = random.Random(seed)
    os.makedirs(os.path.dirname(out_path) or ".", exist_ok=True)
    with open(out_path, "w") as f:
        for op in ops or OPS:
            for n in sizes or TABLE_N:
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
    from paper_2609_28179_gb300.cells import OPS, SWEEP_B, TABLE_N as SWEEP_N
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


RICCATI_FILE = os.path.join(TUNING, "sm103_riccati.jsonl")
RICCATI_H = os.path.join(HERE, "csrc", "riccati_table.h")
COMPOSED = 3


class RiccatiCell:
    """Device inputs of the LQR gain at one (nx, nu) and batch, with a
    launcher per placement (fused scope x pack, or the composition)."""

    def __init__(self, nx, nu, batch, seed=4000, pool=None):
        import torch
        import paper_2609_28179_gb300 as g
        from paper_2609_28179_gb300 import workloads as W
        self.nx, self.nu, self.batch = nx, nu, batch
        if pool is None:
            host = W.riccati_inputs(nx, nu, batch, seed + nx * 100 + nu)
            self.A, self.B, self.P, self.R = (torch.from_numpy(x).cuda() for x in host)
        else:
            self.A, self.B, self.P, self.R = (x[: n * batch] for x, n in
                                              zip((pool.A, pool.B, pool.P, pool.R),
                                                  (nx * nx, nx * nu, nx * nx, nu * nu)))
        self.K = torch.empty(batch * nu * nx, device="cuda")
        self.info = torch.empty(max(1, batch), dtype=torch.int32, device="cuda")
        self.wsb = g.glass_riccati_workspace(nx, nu, batch)
        self.ws = torch.empty(max(1, self.wsb), dtype=torch.uint8, device="cuda")
        # bytes the method must touch: A, B, P, R in, K out
        self.bytes = 4 * batch * (2 * nx * nx + nx * nu + nu * nu + nu * nx)

    def placements(self):
        import paper_2609_28179_gb300 as g
        out = [(s, p) for s in (1, 2) for p in (1, 2, 4, 8) if g.glass_riccati_feasible(self.nx, self.nu, s, p)]
        return out + [(COMPOSED, 1)]

    def launch(self, scope=-1, pack=0):
        import paper_2609_28179_gb300 as g
        nx, nu = self.nx, self.nu
        return g.glass_riccati_gain(nx, nu, self.A, nx * nx, self.B, nx * nu, self.P, nx * nx, self.R, nu * nu,
                                    self.K, nu * nx, self.info, self.batch, self.ws, self.wsb,
                                    g.make_opts(scope=scope, pack=pack))


def riccati_sweep(out_path: str = RICCATI_FILE, iters: int = 5, seed: int = 17):
    """Every placement of the LQR gain (fused scopes and packs, and the
    composition) at each (nx, nu) of the workload and each sweep batch."""
    import torch
    import paper_2609_28179_gb300 as g
    from paper_2609_28179_gb300 import workloads as W
    from paper_2609_28179_gb300.cells import SWEEP_B
    g.lib()
    rng = random.Random(seed)
    stream = torch.cuda.Stream()
    with open(out_path, "w") as f:
        for nx, nu in W.RICCATI_SIZES:
            pool = RiccatiCell(nx, nu, max(SWEEP_B))
            for batch in SWEEP_B:
                cell = RiccatiCell(nx, nu, batch, pool=pool)
                R = _reps(cell.bytes)
                order = cell.placements()
                rng.shuffle(order)
                meas = {}
                for scope, pack in order:
                    g.check(cell.launch(scope, pack), f"riccati {nx}x{nu} {scope}x{pack}")
                    torch.cuda.synchronize()
                    graph = torch.cuda.CUDAGraph()
                    with torch.cuda.graph(graph, stream=stream):
                        for _ in range(R):
                            cell.launch(scope, pack)
                    samples = []
                    for _ in range(iters):
                        torch.cuda.synchronize()
                        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                        a.record()
                        graph.replay()
                        b.record()
                        torch.cuda.synchronize()
                        samples.append(a.elapsed_time(b) * 1e3 / R)
                    del graph
                    meas[(scope, pack)] = statistics.median(samples)
                    f.write(json.dumps({"nx": nx, "nu": nu, "batch": batch, "scope": scope, "pack": pack,
                                        "us": meas[(scope, pack)], "samples": samples, "reps": R}) + "\n")
                f.flush()
                best = choose({k: {"us": v} for k, v in meas.items()})
                print(f"riccati {nx:2d}x{nu:2d} B={batch:6d} best={g.SCOPE_NAMES[best[0]]}x{best[1]} "
                      f"{meas[best]:.2f}us composed={meas[(COMPOSED, 1)]:.2f}us", flush=True)
                del cell
            del pool
            torch.cuda.empty_cache()


def riccati_codegen(inp: str = RICCATI_FILE, out: str = RICCATI_H):
    from paper_2609_28179_gb300 import workloads as W
    from paper_2609_28179_gb300.cells import SWEEP_B
    cells = {}
    with open(inp) as f:
        for line in f:
            r = json.loads(line)
            cells.setdefault((r["nx"], r["nu"], r["batch"]), {})[(r["scope"], r["pack"])] = r
    rows = []
    for nx, nu in W.RICCATI_SIZES:
        codes = []
        for b in SWEEP_B:
            s, p = choose(cells[(nx, nu, b)])  # the composition ranks last on ties (scope 3)
            codes.append(str(12 if s == COMPOSED else s * 4 + int(math.log2(p))))
        rows.append("    {" + ", ".join(codes) + "},")
    sizes = W.RICCATI_SIZES
    text = f"""// riccati_table.h -- GENERATED by paper_2609_28179_gb300/tune.py; do not edit.
// Placement of the LQR gain per ((nx, nu), batch) cell: code = scope * 4 +
// log2(pack) for the fused kernel (scope 1 warp / 2 block), 12 = the
// composition of primitive calls (Sec. IV-E: fusion granularity measured as
// a placement).
// source: {os.path.relpath(inp, os.path.dirname(HERE))} (GB300 measurements, 5 % dispatch margin)
#pragma once
namespace glass {{
static const int kRicNum = {len(sizes)};
static const int kRicNx[{len(sizes)}] = {{{", ".join(str(a) for a, _ in sizes)}}};
static const int kRicNu[{len(sizes)}] = {{{", ".join(str(b) for _, b in sizes)}}};
static const int kRicNumB = {len(SWEEP_B)};
static const int kRicB[{len(SWEEP_B)}] = {{{", ".join(map(str, SWEEP_B))}}};
static const unsigned char kRicTable[{len(sizes)}][{len(SWEEP_B)}] = {{
{chr(10).join(rows)}
}};
}}  // namespace glass
"""
    with open(out, "w") as f:
        f.write(text)
    return out


ROBO_FILE = os.path.join(TUNING, "sm103_robo.jsonl")
ROBO_H = os.path.join(HERE, "csrc", "robo_table.h")
ROBO_N = 16  # argmax / softmax length of the placement table (Table II)


class RoboCell:
    """Device inputs and outputs of one robotics operation at one batch."""

    def __init__(self, op: int, batch: int, seed: int = 5000):
        import torch
        from paper_2609_28179_gb300 import workloads as W
        self.op, self.batch = op, batch
        dev = lambda x: torch.from_numpy(np.ascontiguousarray(x, dtype=np.float32)).cuda()
        empty = lambda n: torch.empty(max(1, n), device="cuda")
        r = W.rng(seed + op)
        if op in (0, 1):
            self.a = dev(W.unit_quaternions(batch, seed))
            self.b = dev(W.rotation_vectors(batch, seed + 1)) if op == 0 else dev(W.unit_quaternions(batch, seed + 2))
            self.outs = [empty(4 * batch if op == 0 else 3 * batch)]
            self.bytes = 4 * batch * (4 + 3 + (4 if op == 0 else 4 + 3 - 3))
        elif op == 2:
            self.a, self.b = dev(W.se3_transforms(batch, seed)), dev(W.twists(batch, seed + 1))
            self.outs = [empty(16 * batch)]
            self.bytes = 4 * batch * (16 + 6 + 16)
        elif op == 3:
            self.a, self.b = dev(r.standard_normal(6 * batch)), dev(r.standard_normal(6 * batch))
            self.outs = [empty(6 * batch)]
            self.bytes = 4 * batch * 18
        elif op == 4:
            self.a, self.b = dev(W.sym3(batch, seed)), None
            self.outs = [empty(3 * batch), empty(9 * batch)]
            self.bytes = 4 * batch * (9 + 12)
        elif op in (5, 6):
            self.a, self.b = dev(r.standard_normal(9 * batch)), None
            self.outs = [empty(9 * batch), empty(3 * batch), empty(9 * batch)] if op == 5 else [empty(9 * batch)]
            self.bytes = 4 * batch * (9 + (21 if op == 5 else 9))
        else:
            self.a, self.b = dev(r.standard_normal(ROBO_N * batch)), None
            self.outs = [torch.empty(max(1, batch), dtype=torch.int32, device="cuda")] if op == 7 else \
                [empty(ROBO_N * batch)]
            self.bytes = 4 * batch * (ROBO_N + (1 if op == 7 else ROBO_N))

    def launch(self, scope=-1, pack=0):
        import paper_2609_28179_gb300 as g
        o, B, a, b, out = g.make_opts(scope=scope, pack=pack), self.batch, self.a, self.b, self.outs
        f = [g.glass_batched_quat_retract, g.glass_batched_quat_error, g.glass_batched_se3_retract,
             g.glass_batched_motion_cross]
        if self.op < 4:
            return f[self.op](a, b, out[0], B, o)
        if self.op == 4:
            return g.glass_batched_eig3(a, out[0], out[1], B, o)
        if self.op == 5:
            return g.glass_batched_svd3(a, out[0], out[1], out[2], B, o)
        if self.op == 6:
            return g.glass_batched_closest_rotation(a, out[0], B, o)
        if self.op == 7:
            return g.glass_batched_argmax(ROBO_N, a, ROBO_N, out[0], B, o)
        return g.glass_batched_softmax(ROBO_N, a, ROBO_N, out[0], ROBO_N, B, o)


def robo_sweep(out_path: str = ROBO_FILE, iters: int = 5, seed: int = 19):
    """Every placement of every robotics operation at each sweep batch."""
    import torch
    import paper_2609_28179_gb300 as g
    from paper_2609_28179_gb300.cells import SWEEP_B
    g.lib()
    rng = random.Random(seed)
    stream = torch.cuda.Stream()
    with open(out_path, "w") as f:
        for op, name in enumerate(g.ROBO_OPS):
            for batch in SWEEP_B:
                cell = RoboCell(op, batch)
                R = _reps(cell.bytes)
                order = [pl for pl in g.PLACEMENTS if g.glass_robo_feasible(op, ROBO_N, *pl)]
                rng.shuffle(order)
                meas = {}
                for scope, pack in order:
                    g.check(cell.launch(scope, pack), f"{name} {scope}x{pack}")
                    torch.cuda.synchronize()
                    graph = torch.cuda.CUDAGraph()
                    with torch.cuda.graph(graph, stream=stream):
                        for _ in range(R):
                            cell.launch(scope, pack)
                    samples = []
                    for _ in range(iters):
                        torch.cuda.synchronize()
                        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                        a.record()
                        graph.replay()
                        b.record()
                        torch.cuda.synchronize()
                        samples.append(a.elapsed_time(b) * 1e3 / R)
                    del graph
                    meas[(scope, pack)] = {"us": statistics.median(samples)}
                    f.write(json.dumps({"op": name, "batch": batch, "scope": scope, "pack": pack,
                                        "us": meas[(scope, pack)]["us"], "samples": samples, "reps": R,
                                        "bytes": cell.bytes}) + "\n")
                f.flush()
                best = choose(meas)
                print(f"{name:17s} B={batch:6d} best={g.SCOPE_NAMES[best[0]]}x{best[1]} "
                      f"{meas[best]['us']:.2f}us", flush=True)
                del cell
                torch.cuda.empty_cache()


def robo_codegen(inp: str = ROBO_FILE, out: str = ROBO_H):
    import paper_2609_28179_gb300 as g
    from paper_2609_28179_gb300.cells import SWEEP_B
    cells = {}
    with open(inp) as f:
        for line in f:
            r = json.loads(line)
            cells.setdefault((r["op"], r["batch"]), {})[(r["scope"], r["pack"])] = r
    rows = []
    for name in g.ROBO_OPS:
        codes = []
        for b in SWEEP_B:
            s, p = choose(cells[(name, b)])
            codes.append(str(s * 4 + int(math.log2(p))))
        rows.append(f"    /* {name} */ {{" + ", ".join(codes) + "},")
    text = f"""// robo_table.h -- GENERATED by paper_2609_28179_gb300/tune.py; do not edit.
// Placement of each robotics operation (glass_robo_op order) per batch
// bucket: code = scope * 4 + log2(pack) (Sec. IV-E, Table II placements);
// argmax and softmax measured at n = {ROBO_N}.
// source: {os.path.relpath(inp, os.path.dirname(HERE))} (GB300 measurements, 5 % dispatch margin)
#pragma once
namespace glass {{
static const int kRoboNumB = {len(SWEEP_B)};
static const int kRoboB[{len(SWEEP_B)}] = {{{", ".join(map(str, SWEEP_B))}}};
static const unsigned char kRoboTable[{len(g.ROBO_OPS)}][{len(SWEEP_B)}] = {{
{chr(10).join(rows)}
}};
}}  // namespace glass
"""
    with open(out, "w") as f:
        f.write(text)
    return out


F64_FILE = os.path.join(TUNING, "sm103_fp64.jsonl")
F64_H = os.path.join(HERE, "csrc", "fp64_table.h")
F64_OPS = ["gemm", "posv", "trsm", "getrf_getrs"]


class F64Cell:
    """FP64 device inputs of one (op, n, batch) cell; destructive operations
    get `sets` copies restored (untimed) between replays."""

    def __init__(self, op, n, batch, sets=1, seed=6000):
        import torch
        self.op, self.n, self.batch = op, n, batch
        gen = torch.Generator(device="cuda")
        gen.manual_seed(seed + n)
        dd = dict(dtype=torch.float64, device="cuda")
        eye = torch.eye(n, **dd)
        if op == "gemm":
            A, B = torch.randn(batch, n, n, generator=gen, **dd), torch.randn(batch, n, n, generator=gen, **dd)
        elif op == "posv":
            M = torch.randn(batch, n, n, generator=gen, **dd)
            A, B = M @ M.transpose(1, 2) + n * eye, torch.randn(batch, n, 1, generator=gen, **dd)
        elif op == "trsm":
            A, B = torch.tril(torch.randn(batch, n, n, generator=gen, **dd)) + n * eye, \
                torch.randn(batch, n, n, generator=gen, **dd)
        else:
            A, B = torch.randn(batch, n, n, generator=gen, **dd) + n * eye, torch.randn(batch, n, 1, generator=gen, **dd)
        self.pristine = {"A": A.transpose(1, 2).contiguous().reshape(-1), "B": B.transpose(1, 2).contiguous().reshape(-1)}
        self.k = n if op in ("gemm", "trsm") else 1
        self.sets = sets if op != "gemm" else 1
        self.work = [{k: v.clone() for k, v in self.pristine.items()} for _ in range(self.sets)] if op != "gemm" \
            else [self.pristine]
        self.out = torch.empty(batch * n * n, **dd) if op == "gemm" else None
        self.info = torch.zeros(max(1, batch), dtype=torch.int32, device="cuda")
        self.ipiv = torch.zeros(max(1, batch * n), dtype=torch.int32, device="cuda")
        from paper_2609_28179_gb300.cells import bytes_flops
        self.bytes = 2 * bytes_flops(op, n)[0] * batch  # FP64: twice the FP32 bytes

    def restore(self):
        if self.op != "gemm":
            for w in self.work:
                for key, v in w.items():
                    v.copy_(self.pristine[key])

    def launch(self, i=0, scope=-1, pack=0):
        import paper_2609_28179_gb300 as g
        w, n, B = self.work[i % len(self.work)], self.n, self.batch
        o = g.make_opts(dtype=g.GLASS_F64, scope=scope, pack=pack)
        if self.op == "gemm":
            return g.glass_batched_gemm(n, n, n, w["A"], n, n * n, w["B"], n, n * n, self.out, n, n * n, B, o)
        if self.op == "posv":
            return g.glass_batched_posv(n, 1, w["A"], n, n * n, w["B"], n, n, self.info, B, o)
        if self.op == "trsm":
            return g.glass_batched_trsm(n, n, w["A"], n, n * n, w["B"], n, n * n, B, o)
        return g.glass_batched_getrf_getrs(n, 1, w["A"], n, n * n, self.ipiv, w["B"], n, n, self.info, B, o)


def fp64_sweep(out_path: str = F64_FILE, iters: int = 5, seed: int = 23):
    """Thread and warp placements of the FP64 storage variants over the
    sweep grid (n <= 8 for thread scope)."""
    import torch
    import paper_2609_28179_gb300 as g
    from paper_2609_28179_gb300.cells import SWEEP_B, SWEEP_N
    g.lib()
    rng = random.Random(seed)
    stream = torch.cuda.Stream()
    with open(out_path, "w") as f:
        for op in F64_OPS:
            for n in SWEEP_N:
                for batch in SWEEP_B:
                    probe = F64Cell(op, n, 1)
                    R = int(min(32, max(8, math.ceil(2 * L2_BYTES / max(1, probe.bytes * batch)))))
                    cell = F64Cell(op, n, batch, sets=R)
                    order = [(s, p) for s in (0, 1) for p in (1, 2, 4, 8) if not (s == 0 and n > 8)]
                    rng.shuffle(order)
                    meas = {}
                    for scope, pack in order:
                        st = cell.launch(0, scope, pack)
                        if st != g.GLASS_OK:
                            continue
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
                        meas[(scope, pack)] = {"us": statistics.median(samples)}
                        f.write(json.dumps({"op": op, "n": n, "batch": batch, "scope": scope, "pack": pack,
                                            "us": meas[(scope, pack)]["us"], "samples": samples, "reps": R}) + "\n")
                    f.flush()
                    best = choose(meas)
                    print(f"fp64 {op:12s} n={n:3d} B={batch:6d} best={g.SCOPE_NAMES[best[0]]}x{best[1]} "
                          f"{meas[best]['us']:.2f}us", flush=True)
                    del cell
                    torch.cuda.empty_cache()


def fp64_codegen(inp: str = F64_FILE, out: str = F64_H):
    from paper_2609_28179_gb300.cells import SWEEP_B, SWEEP_N
    cells = {}
    with open(inp) as f:
        for line in f:
            r = json.loads(line)
            cells.setdefault((r["op"], r["n"], r["batch"]), {})[(r["scope"], r["pack"])] = r
    rows = []
    for op in F64_OPS:
        per_n = []
        for n in SWEEP_N:
            codes = []
            for b in SWEEP_B:
                s, p = choose(cells[(op, n, b)])
                codes.append(str(s * 4 + int(math.log2(p))))
            per_n.append("{" + ", ".join(codes) + "}")
        rows.append(f"    /* {op} */ {{" + ", ".join(per_n) + "},")
    text = f"""// fp64_table.h -- GENERATED by paper_2609_28179_gb300/tune.py; do not edit.
// Placement of the FP64 storage variants per (op row, n, batch) cell: rows
// gemm, posv (potrf/potrs), trsm, getrf_getrs; code = scope * 4 + log2(pack)
// (Sec. IV-A: the fp64 half of the sweep).
// source: {os.path.relpath(inp, os.path.dirname(HERE))} (GB300 measurements, 5 % dispatch margin)
#pragma once
namespace glass {{
static const int kF64NumN = {len(SWEEP_N)};
static const int kF64N[{len(SWEEP_N)}] = {{{", ".join(map(str, SWEEP_N))}}};
static const int kF64NumB = {len(SWEEP_B)};
static const int kF64B[{len(SWEEP_B)}] = {{{", ".join(map(str, SWEEP_B))}}};
static const unsigned char kF64Table[{len(F64_OPS)}][{len(SWEEP_N)}][{len(SWEEP_B)}] = {{
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
    ap.add_argument("cmd", choices=["sweep", "random", "codegen", "launch", "riccati", "riccati-codegen", "robo",
                                    "robo-codegen", "fp64", "fp64-codegen"])
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
    elif args.cmd == "riccati":
        riccati_sweep(args.out or RICCATI_FILE)
    elif args.cmd == "fp64":
        fp64_sweep(args.out or F64_FILE)
    elif args.cmd == "fp64-codegen":
        print(fp64_codegen(args.inp if args.inp != GRID_FILE else F64_FILE))
    elif args.cmd == "robo":
        robo_sweep(args.out or ROBO_FILE)
    elif args.cmd == "robo-codegen":
        print(robo_codegen(args.inp if args.inp != GRID_FILE else ROBO_FILE))
    elif args.cmd == "riccati-codegen":
        print(riccati_codegen(args.inp if args.inp != GRID_FILE else RICCATI_FILE))
    else:
        print(codegen(args.inp))


if __name__ == "__main__":
    sys.exit(main())
