"""The bounded-wait path of the tensor-core kernels (failure detection):
every mbarrier wait in the tcgen05 GEMM gives up after a cycle limit and
records GLASS_ERR_TIMEOUT in the device status word instead of hanging.

The test makes a wait run out without any fault: the self-test entry point
runs the order-64 GEMM with its bulk copies withheld (nothing is ever in
flight) and a short limit, so the first waits expire.  The call must return,
the status word must report the timeout, C must stay untouched, and the next
ordinary call on the same context must be correct with a clear status."""
import numpy as np
import pytest

import oracle
import paper_2609_28179_gb300 as g
from paper_2609_28179_gb300 import workloads as W
from tests.helpers import U32, host, to_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2609_28179_gb300 import _build
    _build.build()
    g.lib()


@pytest.mark.parametrize("batch", [1, 300])
def test_withheld_copies_time_out_and_the_context_stays_usable(batch):
    n = 64
    A = W.gaussian(batch * n * n, 3300 + batch)
    B = W.gaussian(batch * n * n, 3400 + batch)
    dA, dB = to_dev(A), to_dev(B)
    assert g.glass_last_device_status() == g.GLASS_OK  # clear before
    dC = to_dev(np.full(batch * n * n, 7.0, np.float32))
    st = g.glass_selftest_wait_timeout(dA, dB, dC, batch, 200000)  # ~0.1 ms at 2 GHz
    assert st == g.GLASS_OK, g.status_string(st)
    assert g.glass_last_device_status() == g.GLASS_ERR_TIMEOUT
    assert (host(dC) == 7.0).all()  # nothing written after the failure
    assert g.glass_last_device_status() == g.GLASS_OK  # the read cleared it
    # an ordinary call on the same context
    ref = oracle.gemm(n, n, n, A.astype(np.float64), B.astype(np.float64), batch)
    g.check(g.glass_batched_gemm(n, n, n, dA, n, n * n, dB, n, n * n, dC, n, n * n, batch,
                                 g.make_opts(scope=2, pack=1)))
    assert g.glass_last_device_status() == g.GLASS_OK
    M = lambda x: W.from_colmajor(x, batch, n, n)
    bound = n * 2 * U32 * (np.abs(M(A)) @ np.abs(M(B))) + 1e-30
    assert (np.abs(M(host(dC).astype(np.float64) - ref)) <= bound).all()
