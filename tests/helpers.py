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
