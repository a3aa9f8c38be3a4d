"""glass_posv_varsize_noalloc: the mixed-size solve for callers that cannot
allocate device memory (a real-time loop that forbids allocation once it
runs, or a program whose device memory belongs to another allocator).  Its
scratch is a fixed array inside the library, so the test checks that two
calls in a row -- the second one running over whatever the first left in
that array -- give the same results as glass_posv_varsize with caller
scratch, and that a batch beyond the array's limit is refused.

This file is collected last on purpose: a failure here leaves every other
test already run."""
import numpy as np
import pytest

import paper_2609_28179_gb300 as g
from paper_2609_28179_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def test_noalloc_matches_caller_scratch_on_two_calls():
    import torch
    g.lib()
    batch, nrhs = 1000, 4
    sizes = W.varsize_sizes(batch, 3100, lo=1, hi=64)
    A, B, offA, offB = W.varsize_pack(sizes, nrhs, 3101)
    dn = torch.from_numpy(sizes).cuda()
    doA, doB = torch.from_numpy(offA).cuda(), torch.from_numpy(offB).cuda()
    # reference: the existing entry point with caller-supplied scratch
    rA, rB = torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda()
    rinfo = torch.zeros(batch, dtype=torch.int32, device="cuda")
    wsb = g.glass_posv_varsize_workspace(batch)
    ws = torch.empty(wsb, dtype=torch.uint8, device="cuda")
    g.check(g.glass_posv_varsize(batch, dn, doA, doB, nrhs, rA, rB, rinfo, ws, wsb, None))
    torch.cuda.synchronize()
    refA, refB, refI = rA.cpu().numpy(), rB.cpu().numpy(), rinfo.cpu().numpy()
    assert (refI == 0).all()
    for call in range(2):
        dA, dB = torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda()
        info = torch.full((batch,), 77, dtype=torch.int32, device="cuda")
        st = g.glass_posv_varsize_noalloc(batch, dn, doA, doB, nrhs, dA, dB, info, None)
        assert st == g.GLASS_OK, (call, g.status_string(st))
        torch.cuda.synchronize()
        assert np.array_equal(info.cpu().numpy(), refI), call
        xb, xa = dB.cpu().numpy(), dA.cpu().numpy()
        assert np.abs(xb - refB).max() <= 1e-4 * np.abs(refB).max(), call
        assert np.abs(xa - refA).max() <= 1e-4 * np.abs(refA).max(), call


def test_noalloc_rejects_a_batch_beyond_its_array():
    g.lib()
    BAD = 0x10  # never dereferenced: the size check comes first
    assert g.glass_posv_varsize_noalloc(65537, BAD, BAD, BAD, 1, BAD, BAD, BAD, None, 0) == g.GLASS_ERR_UNSUPPORTED
    assert g.glass_posv_varsize_noalloc(0, BAD, BAD, BAD, 1, BAD, BAD, BAD, None, 0) == g.GLASS_OK
