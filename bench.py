"""Benchmark: solved right-hand sides per second of the CBFM + CMP hot path.

One step = one pass of the whole hot path on the 9216-unknown dielectric cube
(side 1 lambda0, eps_r 2.5, 16 x 16 squares per face, 32 cells, CBFs from 64
Fibonacci directions x 2 polarisations): reduced-matrix assembly (far-pair
quadrature, singular near pairs, projection onto the CBFs), CBF Gram matrix
and its inverse (CMP), then 128 right-hand sides (64 Fibonacci directions x
{theta, phi} polarisation) solved by right-preconditioned GMRES to 1e-6 with
currents recovered and the monostatic RCS evaluated.  The CBFs are built once
before timing (set-up, excitation independent) and stay resident.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gb300|reference]

N > 1 runs independent replicas, one per GPU (torchrun, NCCL only for the
barrier and the max over ranks).  --impl reference times the CPU oracle on a
bounded sample of the same workload.

Besides the headline, the JSON line carries comparisons on the same cube and
right-hand sides (each can be switched off): the plain FP64 path, the other GMRES
variant, the paper's conventional MoM (T-diagonal arrangement with its diagonal
preconditioner) with the times in the paper's relative format and the RCS RMSE of
the CBFM against it, IPCBFs generated from that MoM, the inexact (G^CBF)^{-1} of
the paper, batched assembly of mixed scatterers and the serving loop.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import workloads as W  # noqa: E402

METRIC = "solved RHS/sec and p99 solve latency vs plain FP64 GPU path at <=1e-4 RCS err"
UNIT = "RHS/s"
N_RHS = 128
GMRES_TOL = 1e-6
MOM_RESTART = 200      # GMRES restart of the MoM comparison (the paper does not state one)
IPCBF_DELTA_R = 1e-2   # residual allowance of the IPCBF generation (the paper uses 1e-1 to 1e-3)
CMP_INNER_TOL = 1e-5   # inner GMRES tolerance of the inexact (G^CBF)^{-1} (the paper's value)
PEAKS_FALLBACK = {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}
FP32_LANES_PER_SM = 128


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        try:
            return json.load(open(p)), "measured"
        except Exception:
            pass
    return dict(PEAKS_FALLBACK), "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu: int):
        self.gpu = gpu
        self.rows = []
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([x.strip() for x in line.split(",")])

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        if not self.rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(r[1]) for r in self.rows if len(r) > 2 and r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in self.rows if len(r) > 2 and r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        for r in self.rows:
            for i, n in enumerate(names):
                if len(r) > 5 + i and r[5 + i].lower().startswith("active"):
                    reasons.add(n)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(self.rows)}


FP64_PEAK_TFLOPS = 1.25      # nominal GB300 FP64 (CUDA cores)
# FP32 peak derived from the device's SM count and the maximum SM clock (set in main)
DEV = {"n_sm": 152, "sm_max_mhz": 2070.0}


def fp32_peak_tflops() -> float:
    return DEV["n_sm"] * FP32_LANES_PER_SM * 2 * DEV["sm_max_mhz"] * 1e6 / 1e12
FP64_KERNELS = {"k_dots", "k_orth_update", "k_near_blocks", "k_finish", "k_lu_solve", "k_jacobi_svd",
                "k_gemm_z64", "k_pchol", "k_trinv", "k_gj_sweep", "k_gjb_inv", "k_gjb_persistent"}
FP32_KERNELS = {"k_far", "k_fused", "k_matvec", "k_gemm_c32"}


def roofline(name, rec, peaks, peak_src):
    """Roofline entry for one kernel from the library's CUDA-event profile:
    achieved = algorithmic work / measured time (both summed over the launches)."""
    secs = rec["ms"] / 1e3
    out = {"kernel": name, "launches": rec["launches"], "per_launch_ms": rec["ms"] / max(1, rec["launches"]),
           "traffic": None}
    if name in FP64_KERNELS or name in FP32_KERNELS:
        fp64 = name in FP64_KERNELS
        peak = FP64_PEAK_TFLOPS if fp64 else fp32_peak_tflops()
        ach = rec.get("flop", 0.0) / secs / 1e12 if secs > 0 and rec.get("flop") else None
        out.update({"bound": "alu", "unit": "TFLOP/s", "peak": peak, "achieved": ach,
                    "frac": (ach / peak) if ach else None,
                    "peak_source": ("nominal FP64 1.25 TFLOP/s (FP64 units, 2070 MHz)" if fp64 else
                                    f"derived: {DEV['n_sm']} SM x 128 FP32 lanes x 2 flop x "
                                    f"{DEV['sm_max_mhz']:.0f} MHz")})
    else:
        peak = peaks.get("hbm_gbs")
        ach = rec.get("bytes", 0.0) / secs / 1e9 if secs > 0 and rec.get("bytes") else None
        out.update({"bound": "hbm", "unit": "GB/s", "peak": peak, "achieved": ach,
                    "frac": (ach / peak) if ach else None, "peak_source": peak_src})
    return out


def max_over_ranks(x: float, device: str = "cuda") -> float:
    """The largest x over all ranks: the slowest replica sets the whole job's step time."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_value(ws: int, n_rhs: int, t_max_ms: float) -> float:
    """Whole-job throughput: every one of the ws replicas solves n_rhs right-hand sides per step."""
    return ws * n_rhs / (t_max_ms / 1000.0)


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


WORKLOAD = "cube9216"
WORKLOAD_TEXT = {
    "cube9216": "dielectric cube side 1 lambda0, eps_r 2.5, T=3072, N=9216, 32 cells, s=128 generating waves",
    "cube2304": "dielectric cube side 1 lambda0, eps_r 2.5, T=768, N=2304, 16 cells, s=128 generating waves",
    "sphere960": "dielectric sphere radius 0.3 lambda0, eps_r 4, T=320, N=960, 8 cells, s=24 generating waves (12 directions x 2)",
}
PREC_TEXT = {"mixed": "mixed precision", "fused": "mixed precision, fused assembly-projection",
             "unfused": "mixed precision, unfused assembly-projection"}


def workload():
    """The benchmark workload (cube9216); smaller cases exist for profiler captures."""
    if WORKLOAD == "cube9216":
        return W.cube_c2(N_RHS)
    if WORKLOAD == "cube2304":      # same construction, 8 x 8 squares per face, 16 cells
        d = W.cube_c2(N_RHS)
        d.update(mesh=W.cube(8, 1.0), ncell=16)
        return d
    if WORKLOAD == "sphere960":
        d = W.sphere_c1()
        d["exc"] = W.plane_wave_set(W.fibonacci_dirs(N_RHS // 2))[:N_RHS]
        return d
    raise ValueError(WORKLOAD)


# ---- oracle baseline on the host cores (spawned worker processes, one thread each)
_CPU = {}
GMRES_ITERS_ORACLE = 374   # iterations the oracle needs on the bench cube at tol 1e-6


def _cpu_init():
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[k] = "1"
    from oracle import cbfm as OC, mesh as OM
    d = W.cube_c2(N_RHS)
    g = d["mesh"]
    m = OM.build_rwg(g.verts, g.tris)
    cell = OM.cells_rcb(m, 32)
    Ns = np.bincount(cell)
    Ls = [14] * 32
    CM, CJ = W.random_cbfs(Ns, Ls, seed=1)
    _CPU.update(OC=OC, m=m, cbfs=[OC.CellCBF(np.nonzero(cell == c)[0], CM[c], CJ[c], np.ones(1), 14)
                                  for c in range(32)], n=2 * sum(Ls))


def _cpu_noop(_):
    return os.getpid()


def _cpu_blocks(pairs):
    for (a, b) in pairs:
        _CPU["OC"].reduced_block(_CPU["m"], _CPU["cbfs"], 2.5, a, b)
    return len(pairs)


def _cpu_gmres(seed):
    import scipy.linalg as sla
    n = _CPU["n"]
    rng = np.random.default_rng(seed)
    A = np.eye(n) * 4 + (rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))) / np.sqrt(n)
    G = np.eye(n) * 2 + (rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))) / np.sqrt(4 * n)
    lu = sla.lu_factor(G)
    b = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    _x, it, _h = _CPU["OC"].gmres(lambda v: A @ v, b, 0.0, 1000, GMRES_ITERS_ORACLE,
                                  precond=lambda z: sla.lu_solve(lu, z))
    return it


def cpu_step(pool, cores: int) -> dict:
    """One bounded oracle sample of the bench step on the host cores
    (4 x cores cell-pair blocks of the reduced matrix by the oracle's dense
    definition, both media, seeded stand-in CBFs of the workload's sizes; and
    the oracle's GMRES -- MGS, CMP applied as an LU solve, 374 iterations --
    for `cores` right-hand sides on a stand-in system of the same order),
    extrapolated to the whole step: 1024 blocks and 128 right-hand sides."""
    pairs = [(a, b) for a in range(32) for b in range(32)]
    rng = np.random.default_rng(0)
    pick = [pairs[i] for i in rng.choice(len(pairs), 4 * cores, replace=False)]
    t0 = time.perf_counter()
    assert sum(pool.map(_cpu_blocks, [[p] for p in pick])) == len(pick)
    t_asm = time.perf_counter() - t0
    t1 = time.perf_counter()
    its = list(pool.map(_cpu_gmres, range(cores)))
    t_gm = time.perf_counter() - t1
    assert min(its) == GMRES_ITERS_ORACLE
    t_step = t_asm * len(pairs) / len(pick) + t_gm * N_RHS / cores
    return {"value": N_RHS / t_step, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{len(pick)} of 1024 cell-pair blocks of the reduced matrix (oracle dense definition, both "
                      f"media, seeded stand-in CBFs) + oracle GMRES ({GMRES_ITERS_ORACLE} MGS iterations, CMP as LU "
                      f"solve) for {cores} of {N_RHS} RHS on a same-order stand-in system; extrapolated to 1024 "
                      f"blocks and {N_RHS} RHS; {cores} worker processes, one thread each",
            "measured_s": t_asm + t_gm}


def cpu_pool():
    import concurrent.futures as cf
    import multiprocessing as mp
    import oracle
    oracle.build()                      # compile once before the workers load it
    cores = os.cpu_count() or 1
    # one thread per worker: the variables must be in the environment the
    # spawned processes inherit, before they import numpy or load the oracle
    keys = ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")
    saved = {k: os.environ.get(k) for k in keys}
    for k in keys:
        os.environ[k] = "1"
    try:
        pool = cf.ProcessPoolExecutor(max_workers=cores, mp_context=mp.get_context("spawn"), initializer=_cpu_init)
        assert len(set(pool.map(_cpu_noop, range(4 * cores)))) >= 1   # start and initialise the workers
        for f in [pool.submit(_cpu_noop, i) for i in range(cores)]:
            f.result()
    finally:
        for k, v in saved.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v
    return pool, cores


def cpu_sample() -> dict:
    pool, cores = cpu_pool()
    try:
        return cpu_step(pool, cores)
    finally:
        pool.shutdown()


def run_serving(budget_bytes: int) -> dict:
    """Serving workload: Poisson arrivals of requests for scatterers of the
    cube class (cube, sphere, finite cylinder of about one wavelength),
    frequencies from a 16-point sweep 0.8-1.2 f0 (each frequency its own CBFs
    and reduced system) and 1-128 monostatic excitations each, through the
    continuous-batching service on three streams.  The closed-loop capacity is
    measured first; then the same request class is offered at 0.5, 0.8 and
    1.2 times that rate."""
    from paper_2111_11058_gb300 import serve as S
    cub, sph, cyl = W.cube(8, 1.0), W.icosphere(3, 0.5), W.cylinder(0.4, 1.0, 28, 10, 3)
    scs = [S.Scatterer("cube", cub.verts, cub.tris, 2.5, 16, "rcb"),
           S.Scatterer("sphere", sph.verts, sph.tris, 4.0, 16, "rcb"),
           S.Scatterer("cylinder", cyl.verts, cyl.tris, 3.0, 16, "rcb")]
    freqs = np.linspace(0.8, 1.2, 16)
    pool = W.plane_wave_set(W.fibonacci_dirs(128))

    def draw(count, seed):
        rng = np.random.default_rng(seed)
        out = []
        for _ in range(count):
            nrhs = int(rng.integers(1, 129))
            exc = pool[rng.choice(pool.shape[0], nrhs, replace=False)]
            out.append(S.Request(scs[int(rng.integers(0, 3))], float(freqs[int(rng.integers(0, 16))]), exc))
        return out

    be = S.GpuBackend(gen_dirs=64)
    srv = S.Server(be, hbm_budget=budget_bytes, n_streams=3)
    S.replay(srv, draw(12, 100), np.zeros(12))          # warm-up (library, pools)
    srv.drain()
    reqs = draw(48, 101)
    nlog = len(srv.log)
    res, wall = S.replay(srv, reqs, np.zeros(len(reqs)))
    srv.drain()
    closed = S.summarize(res, srv.log[nlog:], wall, srv)
    cap_req_per_s = len(reqs) / wall
    loads = []
    for k, f in enumerate((0.5, 0.8, 1.2)):
        reqs = draw(48, 200 + k)
        nlog = len(srv.log)
        res, wall = S.replay(srv, reqs, S.poisson_arrivals(f * cap_req_per_s, len(reqs), seed=300 + k))
        srv.drain()
        st = S.summarize(res, srv.log[nlog:], wall, srv)
        st["offered_x_capacity"] = f
        loads.append(st)
    srv.close()
    return {"recipe": "cube 2304 / sphere 3840 / cylinder unknowns, 16 cells, s=128, 16 frequencies 0.8-1.2, "
                      "1-128 RHS per request, 48 requests per load, 3 streams, MIXED, block GMRES tol 1e-6 "
                      "(solve sessions that requests of the same key join; cache misses of several keys built "
                      "in one batched assembly when no other stream is free)",
            "budget_bytes": int(budget_bytes), "closed_loop": closed, "capacity_req_per_s": cap_req_per_s,
            "loads": loads}


def run_batch(count: int = 200) -> dict:
    """Batched-scatterer workload: a seeded mix of `count` spheres, cubes and
    finite cylinders (0.2-1.2 wavelengths, eps_r in [1.5, 6], 500-6000
    unknowns, cells of about 200 RWGs) with seeded stand-in CBFs (L_m =
    min(N_m, 16)); all reduced matrices assembled by the batched call (one
    launch per stage) and, for comparison, one scatterer at a time.  Both
    timed with CUDA events; the batched matrices must equal the single ones."""
    import torch
    import paper_2111_11058_gb300 as P
    meshes, cbfs, unknowns = [], [], 0
    for k, d in enumerate(W.scatterer_mix(count, seed=0)):
        g = d["mesh"]
        ne = 3 * g.tris.shape[0] // 2
        unknowns += 2 * ne
        ncell = max(2, ne // 200)
        gm = P.mesh(g.verts, g.tris, ncell, complex(*d["eps"]), partition="rcb")
        Ns = np.bincount(gm.cells(), minlength=ncell)
        CM, CJ = W.random_cbfs(Ns, [int(min(16, n)) for n in Ns], seed=k)
        meshes.append(gm)
        cbfs.append(P.cbf_import(gm, CM, CJ))
    stream = torch.cuda.current_stream()

    def timed(fn):
        torch.cuda.synchronize()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        out = fn()
        b.record(stream)
        torch.cuda.synchronize()
        return a.elapsed_time(b), out

    for r in P.assemble_reduced_batch(meshes[:4], cbfs[:4], P.MIXED):   # warm-up and tuning
        r.free()
    t_batch, reds = timed(lambda: P.assemble_reduced_batch(meshes, cbfs, P.MIXED))
    for r in reds:
        r.free()
    P.profile(True)
    P.profile_read(reset=True)
    _t, reds = timed(lambda: P.assemble_reduced_batch(meshes, cbfs, P.MIXED))
    prof = P.profile_read(reset=True)
    prof = {k: v for k, v in prof.items() if not k.startswith("site:")}
    P.profile(False)
    t_single, singles = timed(lambda: [P.assemble_reduced(m, c, P.MIXED) for m, c in zip(meshes, cbfs)])
    worst = 0.0
    for k in range(0, count, max(1, count // 20)):
        a, b = singles[k].export(), reds[k].export()
        worst = max(worst, float(np.abs(a - b).max()))
    for r in reds + singles:
        r.free()
    return {"recipe": f"{count} scatterers (seeded sphere/cube/cylinder mix, {unknowns} unknowns in total), "
                      "cells of ~200 RWGs, stand-in CBFs L_m = min(N_m, 16), MIXED",
            "batched_ms": t_batch, "one_at_a_time_ms": t_single, "speedup": t_single / t_batch,
            "scatterers_per_s": count / (t_batch / 1e3), "max_abs_diff_batched_vs_single": worst,
            "batched_kernels_ms": {k: round(v["ms"], 3) for k, v in sorted(prof.items(), key=lambda kv: -kv[1]["ms"])[:8]},
            "tuning": P.tuning()}


def run_mom(P, mesh, d, exc_d, cbfm_rcs, t_cbfm_ms: float, timed) -> dict:
    """The paper's comparison method on the same scatterer and right-hand sides:
    the RWG matrix of Eq. (Z) in the T-diagonal arrangement with the diagonal
    preconditioner (Eq. (MoM_T)), mixed precision, per-RHS GMRES to the same
    tolerance, monostatic RCS.  Times are reported as in Sec. IV: CBF generation
    and the CBFM step (reduced assembly, CMP, solve), each relative to the MoM
    total; the RCS difference as the RMSE of Eq. (RMSE), MoM as reference."""
    import torch
    rcs_m = torch.zeros((N_RHS, 1, 2), dtype=torch.float64, device="cuda")
    out = {}

    def step():
        mo = P.assemble_mom(mesh, P.MIXED)
        P.tdiag_setup(mo, jacobi=True)
        res = P.solve(mo, exc_d, tol=GMRES_TOL, maxit=5000, restart=MOM_RESTART, monostatic=True, want_j=False,
                      out_rcs=rcs_m, allow_noconv=True, solver=P.PER_RHS, precond=P.PC_TDIAG)
        out["iters"], out["status"] = res.iters.copy(), res.status
        mo.free()

    step()
    t_mom = float(np.mean(timed(2, step)))
    t_cbf = float(np.mean(timed(2, lambda: P.build_cbfs(mesh, d["gen"], 1e-3).free())))
    sm = rcs_m.sum(-1).cpu().numpy().ravel()

    def rmse_db(sc):
        sc = np.asarray(sc).ravel()
        return 10.0 * math.log10(math.sqrt(float(np.mean((sc - sm) ** 2))) / float(sm.max() - sm.min()))

    # IPCBFs (Sec. III-A): the same generating waves solved on the whole MoM system to delta_r,
    # then the same CBFM step with them
    rcs_i = torch.zeros_like(rcs_m)
    ip = {}

    def gen_ipcbf():
        mo = P.assemble_mom(mesh, P.MIXED)
        ip["cb"] = P.build_ipcbfs(mo, d["gen"], delta_r=IPCBF_DELTA_R, delta_svd=1e-3, restart=MOM_RESTART)
        mo.free()

    def step_ipcbf(prec=P.MIXED, out=rcs_i):
        red = P.assemble_reduced(mesh, ip["cb"], prec)
        ip["n"] = red.n
        P.cmp_setup(red)
        # basis allowed to reach N^CBF + 128 (the block Krylov space saturates instead of restarting)
        res = P.solve(red, exc_d, tol=GMRES_TOL, maxit=2000, restart=1 << 16, monostatic=True, want_j=False,
                      out_rcs=out, allow_noconv=True, solver=P.BLOCK)
        ip["iters"] = res.iters.copy()
        red.free()

    t_ipgen = float(np.mean(timed(1, gen_ipcbf)))
    step_ipcbf()
    t_ipstep = float(np.mean(timed(2, step_ipcbf)))
    rcs_i64 = torch.zeros_like(rcs_m)
    step_ipcbf(P.FP64, rcs_i64)          # the same CBFs on the plain FP64 path, for the precision effect
    it = out["iters"]
    return {"arrangement": "T-diagonal, diagonal preconditioner", "precision": "mixed", "solver": "per_rhs",
            "restart": MOM_RESTART, "n": 2 * mesh.n_edges, "ms_per_step": t_mom,
            "value": N_RHS / (t_mom / 1000.0), "converged": out["status"] == 0,
            "gmres_iters": {"min": int(it.min()), "max": int(it.max()), "mean": float(it.mean())},
            "relative_time": {"cbf_generation": t_cbf / t_mom, "cbfm_step": t_cbfm_ms / t_mom},
            "rcs_rmse_db_cbfm_vs_mom": rmse_db(cbfm_rcs),
            "ipcbf": {"delta_r": IPCBF_DELTA_R, "n_cbf": ip["n"], "generation_iters_max": int(ip["cb"].iters.max()),
                      "relative_time": {"cbf_generation": t_ipgen / t_mom, "cbfm_step": t_ipstep / t_mom},
                      "gmres_iters_max": int(ip["iters"].max()),
                      "rcs_rmse_db_cbfm_vs_mom": rmse_db(rcs_i.sum(-1).cpu().numpy()),
                      "rcs_rmse_db_cbfm_fp64_vs_mom": rmse_db(rcs_i64.sum(-1).cpu().numpy())}}


def run_fused(P, mesh, cbf, exc_d, headline_rcs, t_headline_ms: float, timed, peaks, peak_src) -> dict:
    """The headline step with the assembly fused with the tensor-core projection
    (CBFM_MIXED_FUSED: no local-block or RWG matrix in memory) instead of the form
    CBFM_MIXED picks when memory allows (RWG matrices in memory, then the GEMMs)."""
    import torch
    rcs = torch.zeros((N_RHS, 1, 2), dtype=torch.float64, device="cuda")

    def step():
        red = P.assemble_reduced(mesh, cbf, P.MIXED_FUSED)
        P.cmp_setup(red)
        P.solve(red, exc_d, tol=GMRES_TOL, maxit=2000, restart=1000, monostatic=True, want_j=False, out_rcs=rcs,
                allow_noconv=True, solver=P.BLOCK)
        red.free()
    step()
    t = float(np.mean(timed(2, step)))
    P.profile(True)
    P.profile_read(reset=True)
    red = P.assemble_reduced(mesh, cbf, P.MIXED_FUSED)
    pr = P.profile_read(reset=True)
    pr = {k: v for k, v in pr.items() if not k.startswith("site:")}
    red.free()
    P.profile(False)
    a = rcs.sum(-1).cpu().numpy()
    return {"ms_per_step": t, "value": N_RHS / (t / 1000.0), "time_vs_headline": t / t_headline_ms,
            "rcs_err_vs_headline": float(np.abs(a - headline_rcs).max() / np.abs(headline_rcs).max()),
            "k_fused": roofline("k_fused", pr["k_fused"], peaks, peak_src),
            "assembly_kernels_ms": {k: v["ms"] for k, v in sorted(pr.items(), key=lambda kv: -kv[1]["ms"])}}


C5_CPU_BLOCKS = 2   # oracle cell-pair blocks per host core in the c5 CPU sample


def _cpu_c5_block(pair):
    from oracle import cbfm as OC
    return OC.reduced_block(_CPU["m5"], _CPU["cbfs5"], _CPU["eps5"], pair[0], pair[1]) is not None


def _cpu_c5_init(L):
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[k] = "1"
    from oracle import cbfm as OC, mesh as OM
    d = W.spheroid_c5()
    g = d["mesh"]
    m = OM.build_rwg(g.verts, g.tris)
    cell = OM.cells_rcb(m, d["ncell"])
    Ns = np.bincount(cell, minlength=d["ncell"])
    CM, CJ = W.random_cbfs(Ns, L, seed=2)
    _CPU.update(m5=m, eps5=complex(*d["eps"]),
                cbfs5=[OC.CellCBF(np.nonzero(cell == c)[0], CM[c], CJ[c], np.ones(1), L[c]) for c in range(len(L))])


def run_c5(P, timed, peaks, peak_src, cpu: bool) -> dict:
    """The 90 000-unknown lossy prolate spheroid (256 cells, 256 directions x 2
    polarisations as generating waves and as 512 monostatic excitations): set-up
    (mesh, primary CBFs), then the step -- reduced matrix (CBFM_MIXED takes the
    fused form: the unfused scratch would not fit), CMP, block GMRES to 1e-6 over
    the whole basis -- timed with CUDA events.  The plain FP64 path is not run: its
    assembly needs ~390 GB of scratch."""
    import time as _t
    import torch
    d = W.spheroid_c5()
    g = d["mesh"]
    t0 = _t.perf_counter()
    mesh = P.mesh(g.verts, g.tris, d["ncell"], complex(*d["eps"]), partition=d["partition"])
    cbf = P.build_cbfs(mesh, d["gen"], 1e-3)
    torch.cuda.synchronize()
    t_setup = _t.perf_counter() - t0
    exc = torch.tensor(d["exc"], dtype=torch.float64, device="cuda")
    nrhs = exc.shape[0]
    rcs = torch.zeros((nrhs, 1, 2), dtype=torch.float64, device="cuda")
    st = {}

    def step():
        red = P.assemble_reduced(mesh, cbf, P.MIXED)
        st["n"] = red.n
        P.cmp_setup(red)
        res = P.solve(red, exc, tol=GMRES_TOL, maxit=200, restart=red.n + 256, monostatic=True, want_j=False,
                      out_rcs=rcs, allow_noconv=True, solver=P.BLOCK)
        st["iters"], st["status"] = res.iters.copy(), res.status
        red.free()
    step()
    ts = timed(2, step)
    t = float(np.mean(ts))
    P.profile(True)
    P.profile_read(reset=True)
    step()
    pr = P.profile_read(reset=True)
    pr = {k: v for k, v in pr.items() if not k.startswith("site:")}
    P.profile(False)
    out = {"workload": "lossy prolate spheroid, semi-axes 2 and 0.5 lambda0, eps_r 3-0.1j, T=30000, N=90000, "
                       "256 cells, s=512 generating waves, 512 monostatic RHS, GMRES tol 1e-6, mixed precision",
           "n_cbf": st["n"], "L_range": [int(cbf.L.min()), int(cbf.L.max())], "setup_s": t_setup,
           "ms_per_step": t, "value": nrhs / (t / 1000.0), "unit": UNIT,
           "latency_ms": {"p50": float(np.percentile(ts, 50)), "p99": float(np.percentile(ts, 99))},
           "block_iters": int(st["iters"].max()), "converged": st["status"] == 0,
           "k_fused": roofline("k_fused", pr["k_fused"], peaks, peak_src),
           "kernels_ms": {k: v["ms"] for k, v in sorted(pr.items(), key=lambda kv: -kv[1]["ms"])[:8]},
           "fp64_path": "not run: the plain FP64 assembly needs ~390 GB of scratch"}
    if cpu:
        import concurrent.futures as cf
        import multiprocessing as mp
        import oracle
        oracle.build()
        cores = os.cpu_count() or 1
        Ls = [int(x) for x in cbf.L]
        keys = ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")
        saved = {k: os.environ.get(k) for k in keys}
        for k in keys:
            os.environ[k] = "1"
        try:
            pool = cf.ProcessPoolExecutor(max_workers=cores, mp_context=mp.get_context("spawn"), initializer=_cpu_c5_init,
                                          initargs=(Ls,))
            list(pool.map(_cpu_noop, range(cores)))
        finally:
            for k, v in saved.items():
                if v is None:
                    os.environ.pop(k, None)
                else:
                    os.environ[k] = v
        try:
            rng = np.random.default_rng(0)
            nc = len(Ls)
            pick = [(int(a), int(b)) for a, b in rng.integers(0, nc, size=(C5_CPU_BLOCKS * cores, 2))]
            t1 = _t.perf_counter()
            assert all(pool.map(_cpu_c5_block, pick))
            dt = _t.perf_counter() - t1
        finally:
            pool.shutdown()
        t_asm = dt * nc * nc / len(pick)
        out["cpu_baseline"] = {"kind": "oracle", "cores": cores, "assembly_s_extrapolated": t_asm,
                               "sample": f"{len(pick)} of {nc * nc} cell-pair blocks of the reduced matrix (oracle dense "
                                         f"definition, both media, seeded stand-in CBFs of the GPU's L_m), extrapolated "
                                         f"to all blocks; the oracle's solve is not included",
                               "measured_s": dt,
                               "value": nrhs / t_asm, "unit": UNIT + " (upper bound: assembly only)"}
    return out


def run_cmp_inexact(P, mesh, cbf, exc_d, exact_rcs, t_exact_ms: float, timed) -> dict:
    """The headline step with the paper's inexact (G^CBF)^{-1} (an inner GMRES with
    the diagonal preconditioner D^CBF to 1e-5, Sec. III-C and IV) in place of the
    exact FP64 inverse; everything else unchanged."""
    import torch
    rcs = torch.zeros((N_RHS, 1, 2), dtype=torch.float64, device="cuda")
    out = {}

    def step():
        red = P.assemble_reduced(mesh, cbf, P.MIXED)
        P.cmp_setup(red, inexact=True, inner_tol=CMP_INNER_TOL)
        res = P.solve(red, exc_d, tol=GMRES_TOL, maxit=2000, restart=1000, monostatic=True, want_j=False,
                      out_rcs=rcs, allow_noconv=True, solver=P.BLOCK, precond=P.PC_CMP_INEXACT)
        out["iters"], out["status"] = res.iters.copy(), res.status
        red.free()

    step()
    t = float(np.mean(timed(2, step)))
    a, b = rcs.sum(-1).cpu().numpy(), np.asarray(exact_rcs)
    return {"inner_tol": CMP_INNER_TOL, "ms_per_step": t, "value": N_RHS / (t / 1000.0),
            "time_vs_exact_inverse": t / t_exact_ms, "converged": out["status"] == 0,
            "gmres_iters_max": int(out["iters"].max()),
            "rcs_err_vs_exact_inverse": float(np.abs(a - b).max() / np.abs(b).max())}


def run_reference(args):
    ws, rank, _ = _dist()
    if rank != 0:
        return
    pool, cores = cpu_pool()
    try:
        for _ in range(args.warmup):
            cpu_step(pool, cores)
        vals = []
        t0 = time.perf_counter()
        for _ in range(args.steps):
            vals.append(cpu_step(pool, cores))
        wall = time.perf_counter() - t0
    finally:
        pool.shutdown()
    v = float(np.median([x["value"] for x in vals]))
    cb = dict(vals[0])
    cb["value"] = v
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1000.0 * N_RHS / v, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "dielectric cube 9216 unknowns, 32 cells, 128 RHS (CPU oracle sample)"},
            "cpu_baseline": cb, "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "ms_per_step_kind": "extrapolated: the measured sample (a fraction of the step's cell-pair blocks and "
                                "right-hand sides) scaled to the whole step",
            "sample_ms_per_step": 1000.0 * float(np.median([x["measured_s"] for x in vals])),
            "wall_s": wall}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--no-fp64", action="store_true", help="skip the FP64-path comparison step")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU-oracle baseline")
    ap.add_argument("--no-alt", action="store_true", help="skip the comparison with the other GMRES variant")
    ap.add_argument("--no-serve", action="store_true", help="skip the serving (continuous batching) run")
    ap.add_argument("--no-batch", action="store_true", help="skip the batched-scatterer assembly run")
    ap.add_argument("--no-mom", action="store_true", help="skip the conventional-MoM comparison")
    ap.add_argument("--no-inexact", action="store_true", help="skip the inexact-CMP comparison")
    ap.add_argument("--no-fused", action="store_true", help="skip the fused assembly-projection step on the headline cube")
    ap.add_argument("--no-c5", action="store_true", help="skip the 90 000-unknown spheroid section")
    ap.add_argument("--solver", default="block", choices=["block", "per_rhs"],
                    help="GMRES variant of the timed step: block GMRES over all right-hand sides, or one per RHS")
    ap.add_argument("--prec", default="mixed", choices=["mixed", "fused", "unfused"],
                    help="form of the timed step's mixed-precision assembly: CBFM_MIXED (the faster form that fits), "
                         "CBFM_MIXED_FUSED or CBFM_MIXED_UNFUSED")
    ap.add_argument("--workload", default="cube9216", choices=["cube9216", "cube2304", "sphere960"],
                    help="cube9216 is the benchmark; the others are small cases for profiler captures")
    args = ap.parse_args()
    global WORKLOAD
    WORKLOAD = args.workload
    if args.impl == "reference":
        return run_reference(args)

    import torch
    ws, rank, local = _dist()
    torch.cuda.set_device(local)
    torch.cuda.init()
    DEV["n_sm"] = torch.cuda.get_device_properties(local).multi_processor_count
    DEV["sm_max_mhz"] = float(_peaks()[0].get("sm_max_mhz", DEV["sm_max_mhz"]))
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    from paper_2111_11058_gb300 import build as B
    B.build()
    import paper_2111_11058_gb300 as P

    d = workload()
    g = d["mesh"]
    stream = torch.cuda.current_stream()
    mesh = P.mesh(g.verts, g.tris, d["ncell"], complex(*d["eps"]), partition=d["partition"])
    cbf = P.build_cbfs(mesh, d["gen"], 1e-3)
    exc_d = torch.tensor(d["exc"], dtype=torch.float64, device="cuda")
    rcs_d = torch.zeros((N_RHS, 1, 2), dtype=torch.float64, device="cuda")
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")

    state = {}
    solver = P.BLOCK if args.solver == "block" else P.PER_RHS
    other = P.PER_RHS if solver == P.BLOCK else P.BLOCK

    def make_step(prec, out, slv, exc=exc_d):
        def fn():
            red = P.assemble_reduced(mesh, cbf, prec)
            state["n"] = red.n
            P.cmp_setup(red)
            res = P.solve(red, exc, tol=GMRES_TOL, maxit=2000, restart=1000, monostatic=True, want_j=False,
                          out_rcs=out, allow_noconv=True, solver=slv)
            state["iters"] = res.iters.copy()
            red.free()
        return fn

    prec = {"mixed": P.MIXED, "fused": P.MIXED_FUSED, "unfused": P.MIXED_UNFUSED}[args.prec]
    step = make_step(prec, rcs_d, solver)
    for _ in range(args.warmup):
        step()
    iters = state["iters"].copy()

    def timed(nsteps, fn):
        ts = []
        for _ in range(nsteps):
            flush.fill_(1.0)             # L2 flush between steps (outside the timed span)
            if ws > 1:
                torch.distributed.barrier()
            torch.cuda.synchronize()
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            fn()
            b.record(stream)
            torch.cuda.synchronize()
            ts.append(a.elapsed_time(b))
        return ts

    l0 = P.launch_count()
    with ClockSampler(local) as clk:
        ts = timed(args.steps, step)
    launches = (P.launch_count() - l0) // max(1, args.steps)
    t_step = float(np.mean(ts))
    t_max = max_over_ranks(t_step, "cuda")
    value = job_value(ws, N_RHS, t_max)

    # end to end through the public API with pinned host buffers
    exc_h = torch.tensor(d["exc"], dtype=torch.float64).pin_memory()
    rcs_h = torch.zeros((N_RHS, 1, 2), dtype=torch.float64).pin_memory()
    step_host = make_step(prec, rcs_h.numpy(), solver, exc=exc_h.numpy())
    ts_e2e = timed(max(1, min(args.steps, 3)), step_host)
    e2e = job_value(ws, N_RHS, max_over_ranks(float(np.mean(ts_e2e)), "cuda"))

    # per-kernel profile of the same steps (CUDA events on the launching stream)
    P.profile(True)
    P.profile_read(reset=True)
    n_prof = max(1, min(args.steps, 3))
    timed(n_prof, step)
    prof = P.profile_read(reset=True)
    P.profile(False)
    # "site:*" records split the FP64 products by the solver step that launched them
    sites = {k[5:]: round(v["ms"] / n_prof, 3) for k, v in prof.items() if k.startswith("site:")}
    site_tflops = {k[5:]: round(v["flop"] / (v["ms"] / 1e3) / 1e12, 3) for k, v in prof.items()
                   if k.startswith("site:") and v.get("flop") and v["ms"] > 0}
    prof = {k: v for k, v in prof.items() if not k.startswith("site:")}
    tot = sum(v["ms"] for v in prof.values())
    dom_name, dom = max(prof.items(), key=lambda kv: kv[1]["ms"])
    peaks, peak_src = _peaks()
    clocks = clk.summary()
    roof = roofline(dom_name, dom, peaks, peak_src)
    roof["share"] = dom["ms"] / tot if tot else None
    mixed_rcs = rcs_d.sum(-1).cpu().numpy()

    # the other GMRES variant on the same step, for comparison
    alt = None
    if not args.no_alt:
        rcs_alt = torch.zeros_like(rcs_d)
        step_alt = make_step(prec, rcs_alt, other)
        step_alt()
        alt_iters = state["iters"].copy()
        ts_alt = timed(max(1, min(args.steps, 3)), step_alt)
        alt_rcs = rcs_alt.sum(-1).cpu().numpy()
        alt = {"solver": "per_rhs" if other == P.PER_RHS else "block",
               "value": ws * N_RHS / (float(np.mean(ts_alt)) / 1000.0), "ms_per_step": float(np.mean(ts_alt)),
               "iters_max": int(alt_iters.max()),
               "rcs_err_vs_headline": float(np.abs(alt_rcs - mixed_rcs).max() / np.abs(mixed_rcs).max())}

    # plain FP64 GPU path (the metric's denominator, same solver) and the mixed-vs-FP64 RCS difference
    fp64 = None
    if not args.no_fp64:
        rcs64 = torch.zeros_like(rcs_d)
        t64 = timed(1, make_step(P.FP64, rcs64, solver))
        ref_rcs = rcs64.sum(-1).cpu().numpy()
        err = float(np.abs(mixed_rcs - ref_rcs).max() / np.abs(ref_rcs).max())
        fp64 = {"value": ws * N_RHS / (t64[0] / 1000.0), "ms_per_step": t64[0], "rcs_err_mixed_vs_fp64": err,
                "speedup_mixed_over_fp64": (t64[0] / t_step)}

    mom = None
    if not args.no_mom and ws == 1:
        mom = run_mom(P, mesh, d, exc_d, mixed_rcs, t_step, timed)

    fused = None
    if not args.no_fused and ws == 1:
        fused = run_fused(P, mesh, cbf, exc_d, mixed_rcs, t_step, timed, peaks, peak_src)

    c5 = None
    if not args.no_c5 and ws == 1 and WORKLOAD == "cube9216":
        c5 = run_c5(P, timed, peaks, peak_src, cpu=not args.no_cpu)

    inexact = None
    if not args.no_inexact and ws == 1:
        try:
            inexact = run_cmp_inexact(P, mesh, cbf, exc_d, mixed_rcs, t_step, timed)
        except Exception as e:  # pragma: no cover - reported, not fatal to the benchmark line
            inexact = {"error": str(e)}

    batch = None
    if not args.no_batch and ws == 1 and WORKLOAD == "cube9216":
        batch = run_batch()

    serving = None
    if not args.no_serve and ws == 1 and WORKLOAD == "cube9216":
        free, _tot = torch.cuda.mem_get_info()
        serving = run_serving(int(free * 0.6))

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": t_max, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
                "config": {"workload": WORKLOAD_TEXT[WORKLOAD] + f", {N_RHS} monostatic RHS, GMRES tol 1e-6, "
                                       + PREC_TEXT[args.prec],
                           "solver": args.solver,
                           "n_cbf": state.get("n"), "l2": "512 MB buffer written between timed steps",
                           "parallelism": "replicas" if ws > 1 else "single GPU"},
                "latency_ms": {"p50": float(np.percentile(ts, 50)), "p99": float(np.percentile(ts, 99))},
                "gmres_iters": {"min": int(iters.min()), "max": int(iters.max()), "mean": float(iters.mean())},
                "clocks": clocks, "e2e": {"value": e2e, "unit": UNIT, "h2d_bytes_per_step": int(exc_h.numel() * 8),
                                          "d2h_bytes_per_step": int(rcs_h.numel() * 8)},
                "gpu_launches": int(launches), "roofline": roof, "tuning": P.tuning(),
                "kernels": {k: roofline(k, v, peaks, peak_src) | {"ms_per_step": v["ms"] / n_prof}
                            for k, v in sorted(prof.items(), key=lambda kv: -kv[1]["ms"])[:8]},
                "fp64_products_ms_by_step": dict(sorted(sites.items(), key=lambda kv: -kv[1])),
                # the same products' rate per solver step (6 flop per complex MAC, the three-multiplication form)
                "fp64_products_tflops_by_step": dict(sorted(site_tflops.items(), key=lambda kv: -kv[1])),
                # all timed kernels of a step together (the rest of ms_per_step is launch and host gaps)
                "kernel_ms_per_step": round(tot / n_prof, 3),
                "fp64_path": fp64, "other_solver": alt, "mom": mom, "cmp_inexact": inexact, "batch": batch,
                "serving": serving, "fused": fused, "c5": c5}
        if not args.no_cpu and ws == 1 and WORKLOAD == "cube9216":
            try:
                line["cpu_baseline"] = cpu_sample()
            except Exception as e:  # pragma: no cover
                line["cpu_baseline"] = {"error": str(e)}
        print(json.dumps(line), flush=True)
    if ws > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
