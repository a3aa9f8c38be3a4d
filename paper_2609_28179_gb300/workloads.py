"""Seeded synthetic inputs for the batched small-matrix operations.

This module serves both the device library's tests/benchmark and the oracle's
tests.  It builds inputs only: it computes none of the operations under test
(no factorization, solve or composition).  Exact-arithmetic constructions
(integer Cholesky factors, dyadic LU factors) multiply small integer or dyadic
matrices with numpy, which is exact at these magnitudes, so the intended
factor is known without running any factorization.

Layout: every batch is returned as one flat float32 (or float64) array in
which problem b's element (i, j) sits at ``b*stride + j*ld + i`` (column-major
per problem, packed: ld = rows, stride = rows*cols), unless stated otherwise.

Distributions follow the workloads of the paper's placement sweep
(Sec. IV-A: synthetic batches of independent problems, N from 4 to 128,
B from 1 to 8192): SPD systems A = M M^T + s I with M i.i.d. N(0,1), general
systems N(0,1) + n I, rotations from normalised Gaussian quaternions,
translations and points N(0,1).
"""
from __future__ import annotations

import numpy as np

__all__ = [
    "rng", "colmajor", "from_colmajor", "gaussian", "spd", "general", "kappa_spd",
    "rotations", "se3_transforms", "int_cholesky_factor", "int_lower_pow2_diag",
    "dyadic_lu", "int_matrix", "varsize_sizes", "varsize_pack",
]


def rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def colmajor(mats: np.ndarray, dtype=np.float32) -> np.ndarray:
    """(batch, rows, cols) mathematical matrices -> flat column-major buffer."""
    return np.ascontiguousarray(np.transpose(mats, (0, 2, 1)), dtype=dtype).reshape(-1)


def from_colmajor(flat: np.ndarray, batch: int, rows: int, cols: int) -> np.ndarray:
    """Inverse of :func:`colmajor` for a packed buffer."""
    return np.transpose(np.asarray(flat)[: batch * rows * cols].reshape(batch, cols, rows),
                        (0, 2, 1))


def gaussian(count: int, seed: int, dtype=np.float32) -> np.ndarray:
    return rng(seed).standard_normal(count).astype(dtype)


def spd(n: int, batch: int, seed: int, shift: float | None = None) -> np.ndarray:
    """A = M M^T + shift*I with M_ij ~ N(0,1) (default shift n), rounded to FP32."""
    g = rng(seed)
    shift = float(n) if shift is None else float(shift)
    M = g.standard_normal((batch, n, n))
    A = M @ np.transpose(M, (0, 2, 1)) + shift * np.eye(n)
    return colmajor(A)


def general(n: int, batch: int, seed: int, shift: float | None = None) -> np.ndarray:
    """A_ij ~ N(0,1) + shift*delta_ij (default shift n), rounded to FP32."""
    g = rng(seed)
    shift = float(n) if shift is None else float(shift)
    A = g.standard_normal((batch, n, n)) + shift * np.eye(n)
    return colmajor(A)


def kappa_spd(n: int, batch: int, kappa: float, seed: int) -> np.ndarray:
    """SPD matrices Q diag(lambda) Q^T with lambda = logspace(0, -log10 kappa, n)
    and Q Haar-distributed (QR of a Gaussian with R's diagonal made positive);
    symmetrised, then rounded to FP32."""
    g = rng(seed)
    lam = np.logspace(0.0, -np.log10(kappa), n)
    out = np.empty((batch, n, n))
    for b in range(batch):
        Z = g.standard_normal((n, n))
        Q, R = np.linalg.qr(Z)
        Q = Q * np.sign(np.diag(R))[None, :]
        A = (Q * lam[None, :]) @ Q.T
        out[b] = 0.5 * (A + A.T)
    return colmajor(out)


def _quat_to_rot(q: np.ndarray) -> np.ndarray:
    w, x, y, z = q[..., 0], q[..., 1], q[..., 2], q[..., 3]
    R = np.empty(q.shape[:-1] + (3, 3))
    R[..., 0, 0] = 1 - 2 * (y * y + z * z)
    R[..., 0, 1] = 2 * (x * y - w * z)
    R[..., 0, 2] = 2 * (x * z + w * y)
    R[..., 1, 0] = 2 * (x * y + w * z)
    R[..., 1, 1] = 1 - 2 * (x * x + z * z)
    R[..., 1, 2] = 2 * (y * z - w * x)
    R[..., 2, 0] = 2 * (x * z - w * y)
    R[..., 2, 1] = 2 * (y * z + w * x)
    R[..., 2, 2] = 1 - 2 * (x * x + y * y)
    return R


def rotations(count: int, seed: int) -> np.ndarray:
    """`count` rotation matrices (3x3, column-major, 9 floats each) from
    normalised N(0,1)^4 quaternions."""
    q = rng(seed).standard_normal((count, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    return colmajor(_quat_to_rot(q))


def se3_transforms(count: int, seed: int) -> np.ndarray:
    """`count` homogeneous transforms (4x4 column-major, 16 floats each):
    rotation from a normalised Gaussian quaternion, translation N(0,1)."""
    g = rng(seed)
    q = g.standard_normal((count, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    T = np.zeros((count, 4, 4))
    T[:, :3, :3] = _quat_to_rot(q)
    T[:, :3, 3] = g.standard_normal((count, 3))
    T[:, 3, 3] = 1.0
    return colmajor(T)


# ------------------------------------------------------------- exact inputs
def int_matrix(rows: int, cols: int, batch: int, seed: int, lo: int = -4, hi: int = 4):
    """Integer entries uniform in [lo, hi], as (batch, rows, cols) float64."""
    return rng(seed).integers(lo, hi + 1, size=(batch, rows, cols)).astype(np.float64)


def int_lower_pow2_diag(n: int, batch: int, seed: int, off: int = 2, positive: bool = False):
    """Lower-triangular L with diagonal in {+-1, +-2, +-4} (only positive if
    `positive`) and integer off-diagonals in [-off, off]; (batch, n, n) float64."""
    g = rng(seed)
    L = np.tril(g.integers(-off, off + 1, size=(batch, n, n)), -1).astype(np.float64)
    d = g.choice(np.array([1.0, 2.0, 4.0]), size=(batch, n))
    if not positive:
        d = d * g.choice(np.array([-1.0, 1.0]), size=(batch, n))
    idx = np.arange(n)
    L[:, idx, idx] = d
    return L


def int_cholesky_factor(n: int, batch: int, seed: int, off: int = 2):
    """(A, L0): L0 integer lower with positive power-of-two diagonal and
    A = L0 L0^T (exact in float64 and float32 at these magnitudes)."""
    L0 = int_lower_pow2_diag(n, batch, seed, off=off, positive=True)
    A = L0 @ np.transpose(L0, (0, 2, 1))
    assert np.abs(A).max() < 2 ** 24
    return A, L0


def dyadic_lu(n: int, batch: int, seed: int):
    """(A, perm, L, U) with A[perm[i], :] = (L U)[i, :]: L unit lower with
    off-diagonals in {0, +-1/4, +-1/2}, U upper with integer entries in
    [-4, 4] and diagonal in {+-1, +-2, +-4}.  Because every sub-diagonal
    |l_ij| < 1, partial pivoting is forced to pick the row carrying L's unit
    diagonal, so (perm, L, U) is the unique partial-pivot factorization, and
    all of its arithmetic is exact in FP32."""
    g = rng(seed)
    L = np.tril(g.choice(np.array([0.0, 0.25, -0.25, 0.5, -0.5]), size=(batch, n, n)), -1)
    idx = np.arange(n)
    L[:, idx, idx] = 1.0
    U = np.triu(g.integers(-4, 5, size=(batch, n, n)), 1).astype(np.float64)
    U[:, idx, idx] = g.choice(np.array([1.0, 2.0, 4.0]), size=(batch, n)) * \
        g.choice(np.array([-1.0, 1.0]), size=(batch, n))
    LU = L @ U
    perm = np.stack([g.permutation(n) for _ in range(batch)])
    A = np.empty_like(LU)
    for b in range(batch):
        A[b, perm[b], :] = LU[b]
    return A, perm, L, U


# ------------------------------------------------------------ mixed sizes
def varsize_sizes(batch: int, seed: int, lo: int = 6, hi: int = 64) -> np.ndarray:
    """Problem orders n_i ~ U{lo..hi} (int32)."""
    return rng(seed).integers(lo, hi + 1, size=batch).astype(np.int32)


def varsize_pack(sizes: np.ndarray, nrhs: int, seed: int):
    """Packed SPD systems of mixed order: A_i = M M^T + n_i I (lda = n_i) and
    B_i ~ N(0,1) (n_i x nrhs), concatenated.  Returns (A, B, offA, offB) with
    int64 element offsets of every instance."""
    g = rng(seed)
    sizes = np.asarray(sizes, dtype=np.int64)
    offA = np.zeros(len(sizes), dtype=np.int64)
    offB = np.zeros(len(sizes), dtype=np.int64)
    offA[1:] = np.cumsum(sizes * sizes)[:-1]
    offB[1:] = np.cumsum(sizes * nrhs)[:-1]
    A = np.empty(int((sizes * sizes).sum()), dtype=np.float32)
    B = np.empty(int((sizes * nrhs).sum()), dtype=np.float32)
    for i, n in enumerate(sizes):
        n = int(n)
        M = g.standard_normal((n, n))
        a = M @ M.T + n * np.eye(n)
        A[offA[i]:offA[i] + n * n] = a.T.reshape(-1).astype(np.float32)
        B[offB[i]:offB[i] + n * nrhs] = g.standard_normal(n * nrhs).astype(np.float32)
    return A, B, offA, offB


# ------------------------------------------------------------ LQR gain inputs
# (nx, nu) pairs of the LQR-gain workload: cart-pole, quadrotor, 7-DoF arm
# (joint positions and velocities), a legged base with 12 actuated joints,
# and the largest state the library serves.
RICCATI_SIZES = [(4, 1), (12, 4), (14, 7), (36, 12), (64, 16)]


def riccati_inputs(nx: int, nu: int, batch: int, seed: int):
    """Packed column-major FP32 (A, B, P, R) for K = (R + B^T P B)^{-1} B^T P A:
    A = I + 0.1 N(0,1) (a discretised stable-ish system), B ~ N(0,1),
    P = M M^T + nx I (a cost-to-go, symmetric positive definite, exactly
    symmetric after rounding), R = M M^T + nu I."""
    g = rng(seed)
    A = np.eye(nx) + 0.1 * g.standard_normal((batch, nx, nx))
    B = g.standard_normal((batch, nx, nu))
    Mp = g.standard_normal((batch, nx, nx))
    P = Mp @ np.transpose(Mp, (0, 2, 1)) + nx * np.eye(nx)
    Mr = g.standard_normal((batch, nu, nu))
    R = Mr @ np.transpose(Mr, (0, 2, 1)) + nu * np.eye(nu)
    P = 0.5 * (P + np.transpose(P, (0, 2, 1)))
    R = 0.5 * (R + np.transpose(R, (0, 2, 1)))
    return colmajor(A), colmajor(B), colmajor(P), colmajor(R)


# ------------------------------------------------------- robotics operations
def unit_quaternions(batch: int, seed: int) -> np.ndarray:
    """(w, x, y, z) unit quaternions from normalised N(0,1)^4, [batch][4] FP32."""
    q = rng(seed).standard_normal((batch, 4))
    return (q / np.linalg.norm(q, axis=1, keepdims=True)).astype(np.float32).reshape(-1)


def rotation_vectors(batch: int, seed: int) -> np.ndarray:
    """Rotation vectors with angle ~ U(0, pi) about uniform axes, [batch][3] FP32."""
    g = rng(seed)
    ax = g.standard_normal((batch, 3))
    ax /= np.linalg.norm(ax, axis=1, keepdims=True)
    return (ax * g.uniform(0.0, np.pi, (batch, 1))).astype(np.float32).reshape(-1)


def twists(batch: int, seed: int) -> np.ndarray:
    """(rho, phi): rho ~ N(0,1)^3, phi a rotation vector, [batch][6] FP32."""
    g = rng(seed)
    rho = g.standard_normal((batch, 3))
    phi = rotation_vectors(batch, seed + 1).reshape(batch, 3)
    return np.concatenate([rho, phi], axis=1).astype(np.float32).reshape(-1)


def sym3(batch: int, seed: int) -> np.ndarray:
    """Symmetric 3x3 matrices (M + M^T with M ~ N(0,1)), column-major FP32."""
    M = rng(seed).standard_normal((batch, 3, 3))
    return colmajor(M + np.transpose(M, (0, 2, 1)))
