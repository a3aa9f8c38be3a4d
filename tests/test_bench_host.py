"""Host-side logic of the benchmark that needs no GPU: how the step graph
spreads its independent cells over streams."""
import random

import bench


def test_stream_assignment_is_longest_first_and_balanced():
    """The step graph's cells go to streams longest first, each to the least
    loaded stream: every cell once, loads within the largest cell of each
    other, and one stream keeps the original single-stream order."""
    rng = random.Random(7)
    per = [rng.uniform(0.004, 0.34) for _ in range(48)]
    for k in (1, 2, 3, 4, 8):
        owner = bench.stream_assignment(per, k)
        assert len(owner) == len(per) and all(0 <= o < k for o in owner)
        loads = [sum(t for t, o in zip(per, owner) if o == j) for j in range(k)]
        assert max(loads) - min(loads) <= max(per) + 1e-12
    assert bench.stream_assignment(per, 1) == [0] * len(per)
    # the two longest cells never share a stream when there are two or more
    i1, i2 = sorted(range(len(per)), key=lambda i: -per[i])[:2]
    assert bench.stream_assignment(per, 2)[i1] != bench.stream_assignment(per, 2)[i2]


def test_cell_errors_per_problem_relative_and_lower_triangle_only():
    """The bench's accuracy figure: the largest per-problem max|y - y*| /
    max|y*| over the compared prefix; for posv only L's lower triangle
    counts; pivot mismatches are counted."""
    import numpy as np
    n, s_ref, s = 3, 10, 4
    ref = {"X": np.arange(s_ref * n, dtype=float) + 1.0,
           "L": np.tile(np.eye(n).T.reshape(-1) * 2.0, s_ref), "ipiv": np.zeros(s_ref * n, np.int32)}
    got = {"X": ref["X"][: s * n].copy(), "L": ref["L"][: s * n * n].copy(), "ipiv": np.zeros(s * n, np.int32),
           "count": s}
    got["X"][n + 1] *= 1.01                 # problem 1, |x*| max 6
    got["L"][2 * n * n + n * 1 + 0] = 99.0  # problem 2, (0, 1): upper triangle, ignored
    got["ipiv"][5] = 2
    e, piv = bench.cell_errors("posv", n, got, ref, s_ref, s)
    assert abs(e - 0.05 / 6.0) < 1e-12 and piv == 1
    got["L"][2 * n * n + 1] = 2.5           # problem 2, (1, 0): lower triangle
    e, _ = bench.cell_errors("posv", n, got, ref, s_ref, s)
    assert abs(e - 2.5 / 2.0) < 1e-12
