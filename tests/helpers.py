"""Shared helpers of the GPU parity tests (marshalling only)."""
import numpy as np

import paper_2609_28179_gb300 as g

U32 = 2.0 ** -24  # unit roundoff of FP32


def dev():
    import torch
    return torch.device("cuda:0")


def to_dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).to(dev())


def host(t):
    return t.detach().cpu().numpy()


def zeros_i32(n):
    import torch
    return torch.zeros(max(1, n), dtype=torch.int32, device=dev())


def placements(op, n, k):
    """Every feasible (scope, pack) of (op, n, k)."""
    return [(s, p) for (s, p) in g.PLACEMENTS if g.glass_placement_feasible(op, n, k, s, p)]


def opts_for(scope, pack, **kw):
    return g.make_opts(scope=scope, pack=pack, **kw)


def sync():
    import torch
    torch.cuda.synchronize()


def backward_error(A, X, B):
    """Normwise backward error ||B - A X||_inf / (||A||_inf ||X||_inf + ||B||_inf)
    per problem, FP64; A (batch,n,n), X and B (batch,n,k)."""
    R = B - A @ X
    num = np.abs(R).sum(-1).max(-1) if R.ndim == 3 else np.abs(R).max(-1)
    nA = np.abs(A).sum(-1).max(-1)
    nX = np.abs(X).sum(-1).max(-1)
    nB = np.abs(B).sum(-1).max(-1)
    return num / (nA * nX + nB)


def per_problem_rel(got, want, batch, mask=None):
    """Largest over the batch of the per-problem error max|got - want| /
    max|want| (flat column-major arrays with equal per-problem sizes; mask
    selects entries within a problem)."""
    g_ = np.asarray(got, np.float64).reshape(batch, -1)
    w_ = np.asarray(want, np.float64).reshape(batch, -1)
    if mask is not None:
        g_, w_ = g_[:, mask], w_[:, mask]
    return float((np.abs(g_ - w_).max(1) / np.maximum(np.abs(w_).max(1), 1e-300)).max())


def lower_mask(n):
    """Entries of a column-major n x n matrix on or below the diagonal."""
    return np.tril(np.ones((n, n), dtype=bool)).T.reshape(-1)
