"""Block GMRES solve sessions (cbfm_session_*): right-hand sides joining a
running solve of the reduced system (paper Eqs. (CBFM_outer)/(CBFM_inner)).

* A session nobody joins is the block solve of cbfm_solve: same RCS (to
  rounding) and iteration counts.
* Right-hand sides that join while the solve runs are taken at a block-iteration
  boundary (the cycle restarts with them, the others warm-started): every slot
  converges to tol, and the joined excitations' monostatic RCS equal those of
  a solve of them alone within the mixed path's 1e-4 peak-normalised bound
  (both are converged solutions of the same system; they differ by the
  solver tolerance, not by the joining).
* A session refuses joins once it has finished (CBFM_EFULL)."""
import threading
import time

import numpy as np
import pytest

import workloads as W

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


@pytest.fixture(scope="module")
def sphere(P):
    d = W.sphere_c1()
    g = d["mesh"]
    m = P.mesh(g.verts, g.tris, d["ncell"], complex(*d["eps"]), partition=d["partition"])
    c = P.build_cbfs(m, d["gen"], 1e-3)
    r = P.assemble_reduced(m, c, P.MIXED)
    P.cmp_setup(r)
    return dict(m=m, c=c, r=r)


@pytest.fixture(scope="module")
def cube(P):
    d = W.cube_c2(128)
    g = d["mesh"]
    m = P.mesh(g.verts, g.tris, d["ncell"], complex(*d["eps"]), partition=d["partition"])
    c = P.build_cbfs(m, d["gen"], 1e-3)
    r = P.assemble_reduced(m, c, P.MIXED)
    P.cmp_setup(r)
    return dict(d=d, m=m, c=c, r=r)


def test_session_without_joins_is_the_block_solve(P, sphere):
    exc = W.plane_wave_set(W.fibonacci_dirs(16))
    ref = P.solve(sphere["r"], exc, tol=1e-6, monostatic=True, want_j=False, solver=P.BLOCK)
    s = P.session(sphere["r"], exc, tol=1e-6)
    s.run()
    rcs, iters, resid = s.results()
    s.free()
    assert rcs.shape == (exc.shape[0], 2)
    a, b = ref.rcs[:, 0, :].sum(-1), rcs.sum(-1)
    assert np.abs(a - b).max() <= 1e-10 * np.abs(a).max()
    assert np.array_equal(iters, ref.iters)
    assert (resid <= 1e-6).all()


def test_joined_rhs_equal_alone(P, cube):
    r = cube["r"]
    pool = cube["d"]["exc"]
    first, late = pool[:64], pool[64:80]
    s = P.session(r, first, tol=1e-6, maxit=2000, restart=1000)
    out = {}
    n0 = P.launch_count()

    def run():
        out["status"] = s.run(allow_noconv=False)

    th = threading.Thread(target=run)
    th.start()
    # join once the solve is iterating: the library's launch counter has moved
    # by one block iteration's worth of kernels (about 80)
    t0 = time.perf_counter()
    while P.launch_count() - n0 < 150 and time.perf_counter() - t0 < 10.0:
        time.sleep(0.0002)
    slot = s.join(late)
    th.join()
    rcs, iters, resid = s.results()
    with pytest.raises(P.CbfmError) as ei:          # finished: no more joins
        s.join(late[:1])
    assert ei.value.status == 7
    s.free()
    assert slot == 64 and rcs.shape == (80, 2)
    assert (resid <= 1e-6).all()
    print(f"session: block iterations of the first 64 {iters[:64].max()}, of the 16 joined {iters[64:].max()}")
    alone = P.solve(r, late, tol=1e-6, maxit=2000, restart=1000, monostatic=True, want_j=False, solver=P.BLOCK)
    a = alone.rcs[:, 0, :].sum(-1)
    err = np.abs(rcs[64:].sum(-1) - a).max() / np.abs(a).max()
    print(f"joined vs alone: peak-normalised RCS difference {err:.2e}")
    assert err <= 1e-4
    ref = P.solve(r, first, tol=1e-6, maxit=2000, restart=1000, monostatic=True, want_j=False, solver=P.BLOCK)
    b = ref.rcs[:, 0, :].sum(-1)
    assert np.abs(rcs[:64].sum(-1) - b).max() / np.abs(b).max() <= 1e-4
