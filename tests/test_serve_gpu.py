"""The continuous-batching service on the GPU: requests for two scatterers
at two frequencies arrive together, are batched and run on three streams;
each request's monostatic RCS equals the one computed for that request alone
(fresh build, its own block GMRES solve) within the stated 1e-4 peak-normalised
tolerance of the mixed-precision path, and batches overlap on the device."""
import time

import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def S():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.init()
    from paper_2111_11058_gb300 import build as B
    B.build()
    from paper_2111_11058_gb300 import serve
    return serve


def _requests(S, count=16, seed=7):
    sph = W.icosphere(2, 0.3)
    cub = W.cube(6, 0.6)
    scs = [S.Scatterer("sphere", sph.verts, sph.tris, 4.0, 8, "octant"),
           S.Scatterer("cube", cub.verts, cub.tris, 2.5, 8, "rcb")]
    rng = np.random.default_rng(seed)
    pool = W.plane_wave_set(W.fibonacci_dirs(32))
    reqs = []
    for i in range(count):
        nrhs = int(rng.integers(1, 25))
        exc = pool[rng.choice(pool.shape[0], nrhs, replace=False)]
        reqs.append(S.Request(scs[i % 2], (1.0, 1.15)[(i // 2) % 2], exc))
    return reqs


def test_served_results_equal_alone_and_overlap(S):
    import torch
    be = S.GpuBackend(gen_dirs=12)
    free, _ = torch.cuda.mem_get_info()
    srv = S.Server(be, hbm_budget=free // 2, n_streams=3)
    reqs = _requests(S)
    res, wall = S.replay(srv, reqs, np.zeros(len(reqs)))
    stats = S.summarize(res, srv.log, wall, srv)
    misses = srv.misses
    srv.close()
    print(stats)
    st = be.make_stream()
    worst = 0.0
    for key in sorted({r.key for r in reqs}):
        group = [(r, o) for r, o in zip(reqs, res) if r.key == key]
        handle, _n = be.build(group[0][0].scatterer, group[0][0].freq, st)
        for r, o in group:
            alone, _it = be.solve(handle, r.exc, st)
            err = np.abs(o.rcs.sum(-1) - alone.sum(-1)).max() / np.abs(alone.sum(-1)).max()
            worst = max(worst, err)
        be.free(handle)
    print(f"served vs alone: worst peak-normalised RCS difference {worst:.2e}")
    assert worst <= 1e-4
    assert stats["max_batch_requests"] >= 2          # waiting requests shared a batch
    assert stats["device_overlap_ms"] > 0.0          # batches on different streams overlapped
    assert misses == len({r.key for r in reqs})      # every (scatterer, frequency) built once


def test_served_join_and_cross_key_batch(S):
    """One stream: a request joins the running group of its key, and the cache
    misses of three other keys that waited meanwhile are built in one batch
    (one batched assembly); every result equals its request solved alone."""
    be = S.GpuBackend(gen_dirs=12)
    import torch
    free, _ = torch.cuda.mem_get_info()
    srv = S.Server(be, hbm_budget=free // 2, n_streams=1)
    sph = W.icosphere(2, 0.3)
    cub = W.cube(6, 0.6)
    scs = [S.Scatterer("sphere", sph.verts, sph.tris, 4.0, 8, "octant"),
           S.Scatterer("cube", cub.verts, cub.tris, 2.5, 8, "rcb")]
    pool = W.plane_wave_set(W.fibonacci_dirs(32))
    reqs = [S.Request(scs[0], 1.0, pool[:12]), S.Request(scs[0], 1.0, pool[12:20]),
            S.Request(scs[1], 1.0, pool[20:28]), S.Request(scs[0], 1.15, pool[28:36]),
            S.Request(scs[1], 1.15, pool[36:40])]
    futs = [srv.submit(reqs[0])]
    time.sleep(0.02)                                  # the first batch has started
    futs += [srv.submit(r) for r in reqs[1:]]
    res = [f.result(timeout=300) for f in futs]
    srv.close()                                       # the workers have logged every batch
    log = list(srv.log)
    print(log)
    assert res[0].batch_id == res[1].batch_id         # joined the open group of its key
    assert any(len(b["keys"]) >= 2 for b in log)      # cross-key build
    assert sum(b["joined"] for b in log) >= 1
    st = be.make_stream()
    worst = 0.0
    for key in sorted({r.key for r in reqs}):
        group = [(r, o) for r, o in zip(reqs, res) if r.key == key]
        handle, _n = be.build(group[0][0].scatterer, group[0][0].freq, st)
        for r, o in group:
            alone, _it = be.solve(handle, r.exc, st)
            worst = max(worst, np.abs(o.rcs.sum(-1) - alone.sum(-1)).max() / np.abs(alone.sum(-1)).max())
        be.free(handle)
    print(f"served (joined / cross-key) vs alone: worst peak-normalised RCS difference {worst:.2e}")
    assert worst <= 1e-4
