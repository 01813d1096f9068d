"""Continuous-batching solve service on one GPU.

A request asks for the monostatic RCS of one scatterer at one frequency for a
set of plane-wave excitations (the serving workload: requests arriving over
time, drawn from a class of scatterers, frequencies and 1-128 excitations).
The service

* keeps meshes, CBFs and CMP-ready reduced systems resident on the device in a
  cache keyed by (scatterer, frequency); when the HBM budget would be
  exceeded it evicts the least recently used entry that no work holds;
* admits work by HBM footprint: a batch starts only when the bytes it will
  hold (the cache entry it must build, if any, the transient of that build
  and its solve scratch) fit beside everything resident and in flight;
* batches continuously: whenever a worker slot is free, the oldest waiting
  request that fits is taken together with every other waiting request for
  the same scatterer and frequency (up to 128 right-hand sides, one block
  GMRES solve), so requests that arrive while others run join the next batch
  instead of waiting for a queue to drain;
* runs batches on several CUDA streams at once (one worker thread per
  stream; the library releases the GIL during its calls and its scratch
  memory is stream-ordered), so the kernels of different batches overlap.

Frequencies.  The library works in free-space wavelengths.  A scatterer given
in wavelengths at f0, requested at f = s f0, is the same electrical problem as
the geometry scaled by s, so the service scales the vertices and reports the
RCS in units of the request's wavelength squared.

The scheduling logic talks to a small backend interface (`GpuBackend` drives
the library); tests run it on the CPU with a fake backend.
"""
from __future__ import annotations

import dataclasses
import itertools
import threading
import time
from concurrent.futures import Future
from typing import Any, Dict, List, Optional, Tuple

import numpy as np

MAX_BLOCK_RHS = 128   # block GMRES groups (the library's block width)


@dataclasses.dataclass(frozen=True)
class Scatterer:
    """A closed triangle surface with its medium and cell division."""
    name: str                   # cache identity
    verts: np.ndarray           # (nv, 3), wavelengths at f0
    tris: np.ndarray            # (nt, 3) int32
    eps: complex
    ncell: int
    partition: str = "rcb"

    @property
    def nt(self) -> int:
        return int(self.tris.shape[0])

    @property
    def ne(self) -> int:
        return 3 * self.nt // 2


@dataclasses.dataclass
class Request:
    scatterer: Scatterer
    freq: float                 # f / f0
    exc: np.ndarray             # (nrhs, 3): theta, phi, polarisation angle
    arrival: float = 0.0        # time.perf_counter() at submission (set by submit)
    rid: int = 0

    @property
    def key(self) -> Tuple[str, float]:
        return (self.scatterer.name, float(self.freq))

    @property
    def nrhs(self) -> int:
        return int(self.exc.shape[0])


@dataclasses.dataclass
class Result:
    rid: int
    rcs: np.ndarray             # (nrhs, 2): |E_theta|^2 and |E_phi|^2 parts of the monostatic RCS
    iters: np.ndarray
    latency_s: float
    batch_id: int
    batch_rhs: int              # right-hand sides in the batch this request rode in
    cache_hit: bool


# ------------------------------------------------------------- footprints
def entry_bytes(nt: int, ne: int, n: int, ncell: int) -> int:
    """Device bytes a resident entry holds: mesh records and near list, CBFs
    (FP64 and complex64), reduced matrix and CMP operators (A and B in
    complex64, G and G^-1 in complex128, G^-1 in complex64)."""
    mesh = nt * 48 * 12 + ne * 64 + 40 * nt * 8
    cbf = 2 * 24 * ne * max(1, n // 2 // max(1, ncell) + 1)
    red = n * n * (8 + 8 + 16 + 16 + 8)
    return int(mesh + cbf + red)


def build_transient_bytes(nt: int, ne: int, n: int) -> int:
    """Peak scratch of building an entry: the FP64 local blocks of the CBF
    generation, or the mixed-precision assembly (local blocks, RWG operators,
    their split-TF32 planes and the transposed products), whichever is larger."""
    ldz = (2 * ne + 31) // 32 * 32
    cbf_gen = 27 * nt * nt * 16 + 3 * ne * ne * 16
    assembly = 27 * nt * nt * 8 + 3 * ne * ne * 8 + 2 * 3 * ne * ldz * 4 + 2 * 4 * n * ldz * 4
    return int(max(cbf_gen, assembly))


def solve_bytes(n: int, nrhs: int, ne: int) -> int:
    """Block GMRES scratch for nrhs right-hand sides of a reduced system of order n."""
    p = min(nrhs, MAX_BLOCK_RHS)
    dcap = max(2 * p, min(1000, n + p))
    return int((dcap + 6 * p) * n * 16 + 4 * dcap * dcap * 16 + 3 * dcap * p * 16 + 2 * ne * nrhs * 16)


def estimate_n(sc: Scatterer, s: int) -> int:
    """Upper bound of the reduced order before the CBFs exist: 2 sum_m min(N_m, s)."""
    per = max(1, sc.ne // max(1, sc.ncell))
    return 2 * sc.ncell * min(per, s)


# ------------------------------------------------------------------ cache
class Entry:
    """A resident (scatterer, frequency): library handles, reduced order and bytes."""

    def __init__(self, key, n_est: int, est_bytes: int):
        self.key = key
        self.handle: Any = None
        self.n = n_est
        self.bytes = est_bytes
        self.ready = threading.Event()
        self.error: Optional[BaseException] = None
        self.users = 0
        self.last_used = 0.0


# ---------------------------------------------------------------- backends
class GpuBackend:
    """Drives the library: build = cbfm_mesh, cbfm_build_cbfs,
    cbfm_assemble_reduced (mixed precision), cbfm_cmp_setup; solve = block
    GMRES with monostatic RCS.  Every call is ordered on the worker's stream."""

    def __init__(self, gen_dirs: int = 64, delta_svd: float = 1e-3, tol: float = 1e-6, maxit: int = 2000,
                 restart: int = 1000, prec: Optional[int] = None):
        import torch
        from . import cbfm as C
        self.torch, self.C = torch, C
        self.gen = _plane_waves(gen_dirs)
        self.s = int(self.gen.shape[0])
        self.delta, self.tol, self.maxit, self.restart = delta_svd, tol, maxit, restart
        self.prec = C.MIXED if prec is None else prec

    def make_stream(self):
        return self.torch.cuda.Stream()

    def build(self, sc: Scatterer, freq: float, stream) -> Tuple[Any, int]:
        C, sp = self.C, stream.cuda_stream
        m = C.mesh(np.ascontiguousarray(sc.verts * freq), sc.tris, sc.ncell, sc.eps, partition=sc.partition,
                   stream=sp)
        c = C.build_cbfs(m, self.gen, self.delta, stream=sp)
        r = C.assemble_reduced(m, c, self.prec, stream=sp)
        C.cmp_setup(r, stream=sp)
        return (m, c, r), int(r.n)

    def solve(self, handle, exc: np.ndarray, stream) -> Tuple[np.ndarray, np.ndarray]:
        r = handle[2]
        res = self.C.solve(r, exc, tol=self.tol, maxit=self.maxit, restart=self.restart, monostatic=True,
                           want_j=False, solver=self.C.BLOCK, stream=stream.cuda_stream, allow_noconv=True)
        return res.rcs[:, 0, :].copy(), res.iters.copy()

    def free(self, handle) -> None:
        for h in reversed(handle):
            h.free()

    def event(self, stream):
        ev = self.torch.cuda.Event(enable_timing=True)
        ev.record(stream)
        return ev

    def elapsed_ms(self, e0, e1) -> float:
        e1.synchronize()
        return float(e0.elapsed_time(e1))


def _plane_waves(ndirs: int) -> np.ndarray:
    """ndirs Fibonacci arrival directions x {theta, phi} polarisation (the CBF generating waves)."""
    i = np.arange(ndirs) + 0.5
    theta = np.arccos(1.0 - 2.0 * i / ndirs)
    phi = np.mod(np.pi * (1.0 + 5.0 ** 0.5) * i, 2.0 * np.pi)
    out = np.zeros((2 * ndirs, 3))
    out[0::2, 0], out[0::2, 1], out[0::2, 2] = theta, phi, 0.0
    out[1::2, 0], out[1::2, 1], out[1::2, 2] = theta, phi, np.pi / 2
    return out


# ------------------------------------------------------------------ server
class Server:
    """Continuous-batching service.  `submit` returns a Future of `Result`."""

    def __init__(self, backend, hbm_budget: int, n_streams: int = 3, max_batch_rhs: int = MAX_BLOCK_RHS):
        self.be = backend
        self.budget = int(hbm_budget)
        self.max_rhs = int(min(max_batch_rhs, MAX_BLOCK_RHS))
        self.lock = threading.Condition()
        self.waiting: List[Tuple[Request, Future]] = []      # arrival order
        self.cache: Dict[Tuple[str, float], Entry] = {}
        self.inflight = 0                                      # scratch bytes of running batches
        self.peak_bytes = 0                                    # most bytes held at once (accounting)
        self.busy = [False] * n_streams
        self.work: List[Optional[tuple]] = [None] * n_streams
        self.rid = itertools.count()
        self.bid = itertools.count()
        self.running = True
        self.log: List[dict] = []                              # one record per finished batch
        self.hits = self.misses = self.evictions = 0
        self.streams = [backend.make_stream() for _ in range(n_streams)]
        self.t0_event = backend.event(self.streams[0]) if hasattr(backend, "event") else None
        self.threads = [threading.Thread(target=self._worker, args=(i,), daemon=True) for i in range(n_streams)]
        for t in self.threads:
            t.start()

    # ---- public
    def submit(self, req: Request) -> Future:
        fut: Future = Future()
        req.rid = next(self.rid)
        req.arrival = time.perf_counter()
        if req.nrhs > self.max_rhs:
            fut.set_exception(ValueError(f"request with {req.nrhs} right-hand sides exceeds {self.max_rhs}"))
            return fut
        with self.lock:
            self.waiting.append((req, fut))
            self._dispatch()
        return fut

    def close(self) -> None:
        with self.lock:
            self.running = False
            self.lock.notify_all()
        for t in self.threads:
            t.join()
        with self.lock:
            for e in list(self.cache.values()):
                if e.handle is not None:
                    self.be.free(e.handle)
            self.cache.clear()

    def resident_bytes(self) -> int:
        return sum(e.bytes for e in self.cache.values())

    # ---- scheduling (called with the lock held)
    def _footprint(self, req: Request, nrhs: int) -> Tuple[int, bool]:
        """(bytes the batch adds, whether its entry is already resident or being built)."""
        sc = req.scatterer
        e = self.cache.get(req.key)
        if e is not None:
            return solve_bytes(e.n, nrhs, sc.ne), True
        n = estimate_n(sc, getattr(self.be, "s", 128))
        new = entry_bytes(sc.nt, sc.ne, n, sc.ncell) + build_transient_bytes(sc.nt, sc.ne, n)
        return new + solve_bytes(n, nrhs, sc.ne), False

    def _evict_for(self, need: int) -> bool:
        """Evict idle entries, least recently used first, until `need` bytes fit."""
        while self.resident_bytes() + self.inflight + need > self.budget:
            idle = [e for e in self.cache.values() if e.users == 0 and e.ready.is_set()]
            if not idle:
                return False
            victim = min(idle, key=lambda e: e.last_used)
            del self.cache[victim.key]
            if victim.handle is not None:
                self.be.free(victim.handle)
            self.evictions += 1
        return True

    def _dispatch(self) -> None:
        while self.running and self.waiting and False in self.busy:
            started = False
            for i, (req, _f) in enumerate(self.waiting):
                # this request and every later one for the same key, up to max_rhs right-hand sides
                group, nrhs = [], 0
                for r2, f2 in self.waiting[i:]:
                    if r2.key == req.key and nrhs + r2.nrhs <= self.max_rhs:
                        group.append((r2, f2))
                        nrhs += r2.nrhs
                need, resident = self._footprint(req, nrhs)
                if need > self.budget:
                    for r2, f2 in group:
                        f2.set_exception(MemoryError(f"request needs {need} bytes, budget {self.budget}"))
                    self.waiting = [w for w in self.waiting if all(w[0] is not g[0] for g in group)]
                    started = True
                    break
                if self.resident_bytes() + self.inflight + need > self.budget and not self._evict_for(need):
                    continue          # does not fit now; a smaller or resident one may
                self.waiting = [w for w in self.waiting if all(w[0] is not g[0] for g in group)]
                entry = self.cache.get(req.key)
                hit = entry is not None
                transient = 0
                if hit:
                    self.hits += 1
                    scratch = need
                else:
                    self.misses += 1
                    sc = req.scatterer
                    n = estimate_n(sc, getattr(self.be, "s", 128))
                    entry = Entry(req.key, n, entry_bytes(sc.nt, sc.ne, n, sc.ncell))
                    self.cache[req.key] = entry
                    scratch = need - entry.bytes
                    transient = build_transient_bytes(sc.nt, sc.ne, n)
                entry.users += 1
                self.inflight += scratch
                self.peak_bytes = max(self.peak_bytes, self.resident_bytes() + self.inflight)
                w = self.busy.index(False)
                self.busy[w] = True
                self.work[w] = (group, entry, hit, scratch, transient, next(self.bid))
                self.lock.notify_all()
                started = True
                break
            if not started:
                return

    # ---- workers
    def _worker(self, w: int) -> None:
        st = self.streams[w]
        while True:
            with self.lock:
                while self.running and self.work[w] is None:
                    self.lock.wait()
                if self.work[w] is None:
                    return
                group, entry, hit, scratch, transient, bid = self.work[w]
            t_start = time.perf_counter()
            ev0 = self.be.event(st) if self.t0_event is not None else None
            err: Optional[BaseException] = None
            rcs = iters = None
            exc = np.concatenate([r.exc for r, _ in group], axis=0)
            try:
                if not hit:
                    sc = group[0][0].scatterer
                    try:
                        handle, n = self.be.build(sc, group[0][0].freq, st)
                    except BaseException as e:
                        entry.error = e
                        raise
                    finally:
                        if entry.error is not None:
                            entry.ready.set()
                    with self.lock:
                        entry.handle, entry.n = handle, n
                        entry.bytes = entry_bytes(sc.nt, sc.ne, n, sc.ncell)
                        self.inflight -= transient          # the build's scratch is gone
                        scratch -= transient
                    entry.ready.set()
                else:
                    entry.ready.wait()
                    if entry.error is not None:
                        raise entry.error
                rcs, iters = self.be.solve(entry.handle, exc, st)
            except BaseException as e:  # delivered to the requests of the batch
                err = e
            ev1 = self.be.event(st) if ev0 is not None else None
            t_end = time.perf_counter()
            ofs = 0
            for r, f in group:
                if err is not None:
                    f.set_exception(err)
                else:
                    f.set_result(Result(r.rid, rcs[ofs:ofs + r.nrhs], iters[ofs:ofs + r.nrhs], t_end - r.arrival, bid,
                                        int(exc.shape[0]), hit))
                ofs += r.nrhs
            rec = {"batch": bid, "worker": w, "key": group[0][0].key, "requests": len(group),
                   "rhs": int(exc.shape[0]), "hit": hit, "t_start": t_start, "t_end": t_end, "error": err is not None}
            if ev0 is not None:
                rec["dev_ms"] = (self.be.elapsed_ms(self.t0_event, ev0), self.be.elapsed_ms(self.t0_event, ev1))
            with self.lock:
                entry.users -= 1
                entry.last_used = t_end
                if entry.error is not None and self.cache.get(entry.key) is entry:
                    del self.cache[entry.key]                # a failed build is not cached
                self.inflight -= scratch
                self.busy[w] = False
                self.work[w] = None
                self.log.append(rec)
                self._dispatch()
                self.lock.notify_all()


# -------------------------------------------------------------- statistics
def overlap_ms(intervals: List[Tuple[float, float]]) -> float:
    """Total time during which at least two of the intervals are open."""
    ev = sorted([(a, 1) for a, b in intervals] + [(b, -1) for a, b in intervals])
    depth, last, tot = 0, None, 0.0
    for t, d in ev:
        if depth >= 2 and last is not None:
            tot += t - last
        depth += d
        last = t
    return tot


def summarize(results: List[Result], log: List[dict], wall_s: float, server: Optional[Server] = None) -> dict:
    lat = np.array([r.latency_s for r in results]) * 1e3
    rhs = int(sum(r.rcs.shape[0] for r in results))
    out = {"requests": len(results), "rhs": rhs, "wall_s": wall_s,
           "rhs_per_s": rhs / wall_s if wall_s > 0 else None,
           "latency_ms": {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99)),
                          "max": float(lat.max())} if len(lat) else None,
           "batches": len(log), "mean_batch_requests": float(np.mean([b["requests"] for b in log])) if log else 0.0,
           "max_batch_requests": max([b["requests"] for b in log], default=0)}
    dev = [b["dev_ms"] for b in log if "dev_ms" in b]
    if dev:
        out["device_overlap_ms"] = overlap_ms(dev)
        out["device_busy_ms"] = float(sum(b - a for a, b in dev))
    if server is not None:
        tot = server.hits + server.misses
        out.update(cache_hit_rate=server.hits / tot if tot else None, evictions=server.evictions,
                   peak_accounted_bytes=server.peak_bytes, budget_bytes=server.budget)
    return out


def poisson_arrivals(rate_per_s: float, count: int, seed: int) -> np.ndarray:
    """Arrival offsets (s) of a Poisson process with the given rate."""
    rng = np.random.default_rng(seed)
    return np.cumsum(rng.exponential(1.0 / rate_per_s, size=count))


def replay(server: Server, requests: List[Request], offsets: np.ndarray) -> Tuple[List[Result], float]:
    """Submit the requests at the given offsets from now; wait for all results."""
    t0 = time.perf_counter()
    futs = []
    for req, off in zip(requests, offsets):
        dt = t0 + float(off) - time.perf_counter()
        if dt > 0:
            time.sleep(dt)
        futs.append(server.submit(req))
    res = [f.result() for f in futs]
    return res, time.perf_counter() - t0
