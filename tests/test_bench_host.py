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
