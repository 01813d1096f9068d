"""Bounded device waits (failure detection without a GPU fault).

Every wait of the library's kernels on other CTAs gives up after a time
limit, sets an error word and lets the kernel end.  cbfm_wait_selftest runs
the two barrier forms with an arrival that never comes (a grid barrier
awaited for one CTA more than were launched; a cluster mbarrier initialised
for one arrival more than the cluster has): the call must return
CBFM_ETIMEOUT within its limit and leave the device usable (a completed
barrier and a real computation afterwards).
"""
import time

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.init()
    from paper_2111_11058_gb300 import build as B
    B.build()
    import paper_2111_11058_gb300 as pkg
    return pkg


@pytest.mark.parametrize("kind,limit", [(0, 0.05), (1, 0.05)])   # WAIT_GRID_EXPIRES, WAIT_CLUSTER_EXPIRES
def test_wait_expires_with_status(P, kind, limit):
    t0 = time.perf_counter()
    with pytest.raises(P.CbfmError) as e:
        P.wait_selftest(kind, limit)
    dt = time.perf_counter() - t0
    assert e.value.status == 6   # CBFM_ETIMEOUT
    assert dt < 5.0               # the grid barrier's fixed limit is one second
    # the device stays usable: a completed barrier, then a real computation
    P.wait_selftest(P.WAIT_CLUSTER_COMPLETES, 0.5)
    rng = np.random.default_rng(1)
    A = rng.standard_normal((40, 40)) + 1j * rng.standard_normal((40, 40)) + 8 * np.eye(40)
    X = P.gram_inverse(A)[0]
    assert np.abs(X @ A - np.eye(40)).max() < 1e-12


def test_wait_selftest_arguments(P):
    with pytest.raises(P.CbfmError) as e:
        P.wait_selftest(3, 0.05)
    assert e.value.status == 1   # CBFM_EINVAL
    with pytest.raises(P.CbfmError):
        P.wait_selftest(1, 2.0)
