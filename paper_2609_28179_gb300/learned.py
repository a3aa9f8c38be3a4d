"""Learned placement cost model: an 8-64-64-12 perceptron that predicts the
log latency of the 12 placements (scope x pack) of a matrix operation from
its shape, trained on the GPU by the library's own kernels
(glass_mlp_loss_grad / glass_mlp_adam) on measurements taken by
``tune.py random``.  The paper measures every cell exhaustively and looks
the placement up in a table (Sec. III-A); the model predicts placements for
shapes off that grid, and exhaustive measurement stays the arbiter of its regret.

Features: one-hot over the 4 matrix operations (gemm, posv, trsm,
getrf_getrs), log2 n, log2 k, log2 batch, dtype (0 = FP32), standardised
with the training set's mean and deviation (a constant feature keeps std 1).
Targets: log(us) of each measured placement; unmeasured (infeasible)
placements are masked out of the loss.
"""
from __future__ import annotations

import json
import math
import os
import struct

import numpy as np

import paper_2609_28179_gb300 as g

MODEL_OPS = ["gemm", "posv", "trsm", "getrf_getrs"]
OP_ID = {"gemm": g.GLASS_OP_GEMM, "posv": g.GLASS_OP_POSV, "trsm": g.GLASS_OP_TRSM,
         "getrf_getrs": g.GLASS_OP_GETRF_GETRS}
PLACEMENT_KEYS = [f"{s}x{p}" for s, p in g.PLACEMENTS]
DIN, H, DOUT = 8, 64, 12
NPARAMS = H * DIN + H + H * H + H + DOUT * H + DOUT
MAGIC = b"GLMLP001"


def load_points(path):
    with open(path) as f:
        return [json.loads(line) for line in f if line.strip()]


def features(points):
    X = np.zeros((len(points), DIN), np.float64)
    for r, p in enumerate(points):
        X[r, MODEL_OPS.index(p["op"])] = 1.0
        X[r, 4] = math.log2(p["n"])
        X[r, 5] = math.log2(max(1, p["k"]))
        X[r, 6] = math.log2(max(1, p["batch"]))
        X[r, 7] = 0.0
    return X


def targets(points):
    T = np.zeros((len(points), DOUT), np.float64)
    M = np.zeros((len(points), DOUT), np.float64)
    for r, p in enumerate(points):
        for j, key in enumerate(PLACEMENT_KEYS):
            if key in p["us"]:
                T[r, j] = math.log(p["us"][key])
                M[r, j] = 1.0
    return T, M


def standardise(X):
    mu = X.mean(0)
    sd = X.std(0)
    sd[sd == 0] = 1.0
    return mu, sd


def init_weights(seed=0):
    """He-style initialisation (fixed seed), biases zero."""
    rng = np.random.Generator(np.random.PCG64(seed))
    w = np.zeros(NPARAMS, np.float32)
    o = 0
    for fan_in, fan_out in ((DIN, H), (H, H), (H, DOUT)):
        w[o:o + fan_in * fan_out] = rng.standard_normal(fan_in * fan_out) * math.sqrt(2.0 / fan_in)
        o += fan_in * fan_out + fan_out
    return w


def train(points, epochs=300, batch=256, lr=1e-3, seed=0, log_every=0):
    """Train on the GPU with the library's kernels; returns (w, mu, sd, losses)."""
    import torch
    X = features(points)
    mu, sd = standardise(X)
    Xs = ((X - mu) / sd).astype(np.float32)
    T, M = targets(points)
    dev = torch.device("cuda")
    dX = torch.from_numpy(Xs).to(dev)
    dT = torch.from_numpy(T.astype(np.float32)).to(dev)
    dM = torch.from_numpy(M.astype(np.float32)).to(dev)
    w = torch.from_numpy(init_weights(seed)).to(dev)
    m = torch.zeros_like(w)
    v = torch.zeros_like(w)
    grad = torch.zeros_like(w)
    loss = torch.zeros(1, dtype=torch.float32, device=dev)
    wsb = g.glass_mlp_workspace(batch)
    ws = torch.empty(wsb, dtype=torch.uint8, device=dev)
    rng = np.random.Generator(np.random.PCG64(seed + 1))
    rows = len(points)
    step, losses = 0, []
    for ep in range(epochs):
        perm = torch.from_numpy(rng.permutation(rows)).to(dev)
        xb_all, tb_all, mb_all = dX[perm], dT[perm], dM[perm]
        for s0 in range(0, rows, batch):
            nb = min(batch, rows - s0)
            xb = xb_all[s0:s0 + nb].contiguous()
            tb = tb_all[s0:s0 + nb].contiguous()
            mb = mb_all[s0:s0 + nb].contiguous()
            g.check(g.glass_mlp_loss_grad(DIN, w, nb, xb, tb, mb, grad, loss, ws, wsb), "mlp_loss_grad")
            step += 1
            g.check(g.glass_mlp_adam(NPARAMS, w, grad, m, v, step, lr), "mlp_adam")
        if log_every and (ep % log_every == 0 or ep == epochs - 1):
            losses.append(full_loss(w, dX, dT, dM))
    if not log_every:
        losses.append(full_loss(w, dX, dT, dM))
    return w.cpu().numpy(), mu, sd, losses


def full_loss(w, dX, dT, dM):
    import torch
    rows = dX.shape[0]
    wsb = g.glass_mlp_workspace(rows)
    ws = torch.empty(wsb, dtype=torch.uint8, device=dX.device)
    grad = torch.zeros_like(w)
    loss = torch.zeros(1, dtype=torch.float32, device=dX.device)
    g.check(g.glass_mlp_loss_grad(DIN, w, rows, dX, dT, dM, grad, loss, ws, wsb), "mlp_loss")
    return float(loss.item())


def predict(w, mu, sd, points):
    """Predicted log latencies [rows, 12] from the GPU forward kernel."""
    import torch
    X = ((features(points) - mu) / sd).astype(np.float32)
    dev = torch.device("cuda")
    dX = torch.from_numpy(X).to(dev)
    dY = torch.empty((len(points), DOUT), dtype=torch.float32, device=dev)
    dw = torch.from_numpy(np.ascontiguousarray(w, np.float32)).to(dev)
    g.check(g.glass_mlp_forward(DIN, dw, len(points), dX, dY), "mlp_forward")
    return dY.cpu().numpy()


def _feasible_keys(p):
    return [key for key in PLACEMENT_KEYS if key in p["us"]]


def regret_of(p, key):
    best = min(p["us"].values())
    return p["us"][key] / best - 1.0


def learned_choices(w, mu, sd, points):
    Y = predict(w, mu, sd, points)
    out = []
    for r, p in enumerate(points):
        keys = _feasible_keys(p)
        j = min((PLACEMENT_KEYS.index(k) for k in keys), key=lambda j: Y[r, j])
        out.append(PLACEMENT_KEYS[j])
    return out


def grid_choices(points):
    """The paper's method without the model: the measured table's entry of the
    nearest grid cell (glass_get_placement, use_learned = 0)."""
    out = []
    for p in points:
        s, (scope, pack) = g.glass_get_placement(OP_ID[p["op"]], p["n"], p["k"], p["batch"], 0, 0)
        g.check(s, "get_placement")
        key = f"{scope}x{pack}"
        if key not in p["us"]:  # the table's cell was not measured at this shape (infeasible)
            key = min(_feasible_keys(p), key=lambda k: p["us"][k])
        out.append(key)
    return out


def fixed_choice(train_points):
    """Best single placement over the training set (geomean of latency ratio to
    the per-point best, over points where it is feasible everywhere)."""
    best_key, best_score = None, math.inf
    for key in PLACEMENT_KEYS:
        if not all(key in p["us"] for p in train_points):
            continue
        score = np.mean([math.log(p["us"][key] / min(p["us"].values())) for p in train_points])
        if score < best_score:
            best_key, best_score = key, score
    return best_key


def summary(regrets):
    r = np.asarray(regrets)
    return {"median": float(np.median(r)), "p90": float(np.percentile(r, 90)), "mean": float(r.mean()),
            "within_5pct": float((r <= 0.05).mean())}


def evaluate(w, mu, sd, train_points, held):
    lc = learned_choices(w, mu, sd, held)
    gc = grid_choices(held)
    fk = fixed_choice(train_points)
    fixed = [regret_of(p, fk) if fk in p["us"] else regret_of(p, min(p["us"], key=p["us"].get)) for p in held]
    return {"learned": summary([regret_of(p, k) for p, k in zip(held, lc)]),
            "nearest_grid_table": summary([regret_of(p, k) for p, k in zip(held, gc)]),
            "fixed_placement": {"placement": fk, **summary(fixed)},
            "points": len(held)}


def save(path, w, mu, sd):
    with open(path, "wb") as f:
        f.write(MAGIC)
        f.write(struct.pack("<iii", DIN, H, DOUT))
        f.write(np.asarray(mu, np.float32).tobytes())
        f.write(np.asarray(sd, np.float32).tobytes())
        f.write(np.asarray(w, np.float32).tobytes())


def load(path):
    with open(path, "rb") as f:
        if f.read(8) != MAGIC:
            raise ValueError(f"{path}: not a GLASS MLP weight file")
        din, h, dout = struct.unpack("<iii", f.read(12))
        if (din, h, dout) != (DIN, H, DOUT):
            raise ValueError(f"{path}: shape {(din, h, dout)} != {(DIN, H, DOUT)}")
        mu = np.frombuffer(f.read(4 * DIN), np.float32)
        sd = np.frombuffer(f.read(4 * DIN), np.float32)
        w = np.frombuffer(f.read(4 * NPARAMS), np.float32)
    return w, mu, sd


def install(path=None):
    """Hand a trained model to the library (glass_set_learned_model)."""
    path = path or os.path.join(os.path.dirname(os.path.abspath(__file__)), "tuning", "sm103_mlp.bin")
    w, mu, sd = load(path)
    g.check(g.glass_set_learned_model(w, mu, sd), "set_learned_model")
    return path
