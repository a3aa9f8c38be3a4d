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


def test_summarize_extras_reads_every_record_it_reports():
    """The result line's summaries of the other configurations come from
    the records extra_* produce; a key renamed on one side would turn into an
    error entry on the line.  A record of the same shape (values arbitrary)
    must summarise without errors, with the compensated-residual ratios."""
    import bench
    t = {"us": 10.0}
    refine = {f"time_n{n}_{k}": t for n in (32, 64)
              for k in ("refine0", "refine1", "refine1_fp64diag0", "refine0_fp64diag1", "refine1_dot2")}
    row = {"fwd_err_median": 1e-7, "fwd_err_max": 1e-6, "bwd_err_max": 1e-9, "failed": 0, "within_1e-4_fwd": 128}
    for n in (32, 64):
        for kappa in (1e1, 1e6):
            refine[f"n{n}_kappa{kappa:.0e}"] = {"x0": row, "x1": row, "x1d": row}
    ex = {"plain_posv_n6": {"us": 5.0, "matrices_per_s": 1e8},
          "mixed_size": {"best": {"schedule": "warps_per_cta=8", "us": 140.0, "matrices_per_s": 5e7,
                                  "frac_hbm": 0.06}},
          "tensor_core_gemm": {"bf16_n64": {"us": 317.0, "frac_hbm": 1.0}, "bf16_n16": {"us": 26.0, "frac_hbm": 0.75}},
          "refined_posv": refine,
          "learned_placement": {k: {"median": 0.0, "p90": 0.03} for k in
                                ("learned", "nearest_grid_table", "fixed_placement")}}
    out = bench.summarize_extras(ex)
    assert not any(isinstance(v, dict) and "error" in v for v in out.values()), out
    assert out["refined_posv"]["n64_refined_dot2_over_plain"] == 1.0
    assert out["refined_posv"]["n64_kappa1e+06"]["x1d_fwd_med"] == 1e-7
    assert list(out["tensor_core_gemm"]) == ["bf16_n64"]
