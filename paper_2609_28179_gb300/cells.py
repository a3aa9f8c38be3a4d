"""Cells of the placement sweep: one (operation, order n, batch) workload
with its synthetic inputs resident in device memory, a launcher through the
C ABI, and the algorithmic bytes / flops one launch must move / perform.

Workloads follow the paper's placement sweep (Sec. IV-A: synthetic batches
of independent problems swept over problem size and batch size): SPD systems
A = M M^T + n I, general systems N(0,1) + n I, lower-triangular factors
tril(N(0,1)) + n I with n right-hand sides, rotation chains from normalised
Gaussian quaternions, SE(3) chains applied to 1024 N(0,1) points.  For the
geometry operations n is the chain length.

Destructive operations (posv, trsm, getrf_getrs overwrite their inputs) get
`sets` device copies of the same pristine input so that every launch of a
timed sequence sees fresh valid data; `restore()` refreshes them untimed.
"""
from __future__ import annotations

import numpy as np

import paper_2609_28179_gb300 as g
from paper_2609_28179_gb300 import workloads as W

OPS = ["gemm", "posv", "trsm", "getrf_getrs", "rot3", "se3"]
OP_ID = {"gemm": g.GLASS_OP_GEMM, "posv": g.GLASS_OP_POSV, "trsm": g.GLASS_OP_TRSM,
         "getrf_getrs": g.GLASS_OP_GETRF_GETRS, "rot3": g.GLASS_OP_ROT3, "se3": g.GLASS_OP_SE3}
SWEEP_N = [3, 6, 7, 12, 14, 24, 32, 64]
# Orders of the placement table: the sweep's, plus 16 (the smallest order of
# the tensor-core GEMM kernels, which the FP32 block placement uses there).
TABLE_N = [3, 6, 7, 12, 14, 16, 24, 32, 64]
SWEEP_B = [1, 64, 1024, 16384]
NPTS = 1024
DESTRUCTIVE = {"posv", "trsm", "getrf_getrs"}


def rhs_of(op: str, n: int) -> int:
    """Right-hand sides (solves), inner size (gemm) or chain length (geometry)."""
    return {"gemm": n, "posv": 1, "trsm": n, "getrf_getrs": 1, "rot3": n, "se3": n}[op]


def bytes_flops(op: str, n: int, k: int | None = None):
    """Algorithmic bytes and flops of ONE problem (FP32 storage, s = 4 B)."""
    k = rhs_of(op, n) if k is None else k
    s = 4
    if op == "gemm":
        return s * 3 * n * n, 2 * n ** 3
    if op == "posv":  # L written back (lower triangle read + written) + B read + X written
        return s * (n * (n + 1) + 2 * n * k), n ** 3 / 3 + n * n / 2 + n / 6 + 2 * n * n * k
    if op == "potrf":
        return s * n * (n + 1), n ** 3 / 3 + n * n / 2 + n / 6
    if op in ("potrs", "trsm"):
        fl = (2 if op == "potrs" else 1) * n * n * k
        return s * (n * (n + 1) // 2 + 2 * n * k), fl
    if op == "getrf_getrs":
        return s * (2 * n * n + n + 2 * n * k), 2 * n ** 3 / 3 + 2 * n * n * k
    if op == "rot3":  # chain of k rotations in, one out
        return 36 * (k + 1), 45 * (k - 1)
    if op == "se3":   # chain of k transforms + npts points in, npts points out
        return 64 * k + 24 * NPTS, 18 * NPTS + 63 * (k - 1)
    raise ValueError(op)


class Cell:
    """Device-resident inputs of one cell and launchers through the C ABI."""

    def __init__(self, op: str, n: int, batch: int, seed: int = 1002, sets: int = 1, host=None,
                 device_inputs: bool = False):
        import torch
        self.op, self.n, self.batch = op, n, batch
        self.k = rhs_of(op, n)
        self.sets = sets if op in DESTRUCTIVE else 1
        self.dev = torch.device("cuda")
        if device_inputs:
            self.host = None
            self.pristine = make_inputs_device(op, n, batch, seed)
        else:
            h = host if host is not None else make_inputs(op, n, batch, seed)
            self.host = h
            t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(self.dev)
            self.pristine = {key: t(v) for key, v in h.items()}
        self.work = [{key: v.clone() for key, v in self.pristine.items()} for _ in range(self.sets)] \
            if op in DESTRUCTIVE else [self.pristine]
        nn, k = n, self.k
        if op == "gemm":
            self.out = torch.empty(batch * nn * nn, dtype=torch.float32, device=self.dev)
        elif op == "rot3":
            self.out = torch.empty(batch * 9, dtype=torch.float32, device=self.dev)
        elif op == "se3":
            self.out = torch.empty(batch * 3 * NPTS, dtype=torch.float32, device=self.dev)
        else:
            self.out = None
        self.info = torch.zeros(max(1, batch), dtype=torch.int32, device=self.dev)
        self.ipiv = torch.zeros(max(1, batch * nn), dtype=torch.int32, device=self.dev)
        self.bytes, self.flops = bytes_flops(op, n)
        self.bytes *= batch
        self.flops *= batch

    def restore(self):
        for w in self.work:
            for key, v in w.items():
                v.copy_(self.pristine[key])

    def launch(self, i: int = 0, scope: int = g.GLASS_SCOPE_AUTO, pack: int = 0, stream=None) -> int:
        w = self.work[i % len(self.work)]
        o = g.make_opts(scope=scope, pack=pack)
        n, k, B = self.n, self.k, self.batch
        if self.op == "gemm":
            return g.glass_batched_gemm(n, n, n, w["A"], n, n * n, w["B"], n, n * n, self.out, n, n * n, B, o, stream)
        if self.op == "posv":
            return g.glass_batched_posv(n, 1, w["A"], n, n * n, w["B"], n, n, self.info, B, o, stream)
        if self.op == "trsm":
            return g.glass_batched_trsm(n, n, w["A"], n, n * n, w["B"], n, n * n, B, o, stream)
        if self.op == "getrf_getrs":
            return g.glass_batched_getrf_getrs(n, 1, w["A"], n, n * n, self.ipiv, w["B"], n, n, self.info, B, o,
                                               stream)
        if self.op == "rot3":
            return g.glass_batched_rot3_compose(k, w["A"], 9 * k, self.out, 9, B, o, stream)
        if self.op == "se3":
            return g.glass_batched_se3_apply(k, w["A"], 16 * k, NPTS, w["B"], 3 * NPTS, self.out, 3 * NPTS, B, o,
                                             stream)
        raise ValueError(self.op)

    def feasible(self, scope: int, pack: int) -> bool:
        return g.glass_placement_feasible(OP_ID[self.op], self.n if self.op not in ("rot3", "se3") else
                                          (3 if self.op == "rot3" else 4), self.k, scope, pack)

    def nbytes_device(self) -> int:
        per = sum(v.numel() * v.element_size() for v in self.pristine.values())
        return per * (1 + (self.sets if self.op in DESTRUCTIVE else 0))


def make_inputs(op: str, n: int, batch: int, seed: int):
    """Host inputs (flat float32, column-major per problem) of a cell."""
    k = rhs_of(op, n)
    if op == "gemm":
        return {"A": W.gaussian(batch * n * n, seed), "B": W.gaussian(batch * n * n, seed + 1)}
    if op == "posv":
        return {"A": W.spd(n, batch, seed), "B": W.gaussian(batch * n, seed + 1)}
    if op == "trsm":
        Lm = np.tril(W.rng(seed).standard_normal((batch, n, n))) + n * np.eye(n)
        return {"A": W.colmajor(Lm), "B": W.gaussian(batch * n * k, seed + 1)}
    if op == "getrf_getrs":
        return {"A": W.general(n, batch, seed), "B": W.gaussian(batch * n, seed + 1)}
    if op == "rot3":
        return {"A": W.rotations(batch * k, seed)}
    if op == "se3":
        return {"A": W.se3_transforms(batch * k, seed), "B": W.gaussian(batch * 3 * NPTS, seed + 1)}
    raise ValueError(op)


def make_inputs_device(op: str, n: int, batch: int, seed: int):
    """The same distributions as make_inputs, drawn on the device with a
    seeded torch generator (used by the autotuner, where host generation of
    thousands of large cells would dominate).  Returns flat float32 device
    tensors, column-major per problem."""
    import torch
    dev = torch.device("cuda")
    gen = torch.Generator(device=dev)
    gen.manual_seed(seed)
    k = rhs_of(op, n)
    rn = lambda *shape: torch.randn(*shape, generator=gen, device=dev, dtype=torch.float32)
    eye = torch.eye(n, device=dev, dtype=torch.float32)
    if op == "gemm":
        return {"A": rn(batch * n * n), "B": rn(batch * n * n)}
    if op == "posv":
        M = rn(batch, n, n)
        A = torch.bmm(M, M.transpose(1, 2)) + n * eye
        return {"A": A.transpose(1, 2).contiguous().reshape(-1), "B": rn(batch * n)}
    if op == "trsm":
        L = torch.tril(rn(batch, n, n)) + n * eye
        return {"A": L.transpose(1, 2).contiguous().reshape(-1), "B": rn(batch * n * k)}
    if op == "getrf_getrs":
        A = rn(batch, n, n) + n * eye
        return {"A": A.transpose(1, 2).contiguous().reshape(-1), "B": rn(batch * n)}
    if op in ("rot3", "se3"):
        q = rn(batch * k, 4)
        q = q / q.norm(dim=1, keepdim=True)
        w, x, y, z = q.unbind(1)
        R = torch.stack([1 - 2 * (y * y + z * z), 2 * (x * y + w * z), 2 * (x * z - w * y),
                         2 * (x * y - w * z), 1 - 2 * (x * x + z * z), 2 * (y * z + w * x),
                         2 * (x * z + w * y), 2 * (y * z - w * x), 1 - 2 * (x * x + y * y)], dim=1)
        if op == "rot3":
            return {"A": R.reshape(-1).contiguous()}
        T = torch.zeros(batch * k, 16, device=dev, dtype=torch.float32)
        T[:, [0, 1, 2, 4, 5, 6, 8, 9, 10]] = R
        T[:, 12:15] = rn(batch * k, 3)
        T[:, 15] = 1.0
        return {"A": T.reshape(-1).contiguous(), "B": rn(batch * 3 * NPTS)}
    raise ValueError(op)
