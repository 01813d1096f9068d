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
  GMRES solve); when that is a cache miss and no other worker is free, the
  cache misses of other waiting keys are built in the same batch (one
  batched assembly launch for all of them, `cbfm_assemble_reduced_batch`);
* lets requests join running work: a request whose key has an open group
  (a batch building or solving it) joins that group -- appended while the
  entry is built, and handed to the running block GMRES session otherwise,
  which takes it at its next block-iteration boundary (`cbfm_session_join`);
  only when no group is open, or the group is full, does it wait;
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

    def build_many(self, items, stream) -> List[Tuple[Any, int]]:
        """Several entries at once: meshes and CBFs one by one, the reduced
        systems in one batched assembly, then the CMP of each."""
        C, sp = self.C, stream.cuda_stream
        ms = [C.mesh(np.ascontiguousarray(sc.verts * f), sc.tris, sc.ncell, sc.eps, partition=sc.partition, stream=sp)
              for sc, f in items]
        cs = [C.build_cbfs(m, self.gen, self.delta, stream=sp) for m in ms]
        rs = C.assemble_reduced_batch(ms, cs, self.prec, stream=sp)
        for r in rs:
            C.cmp_setup(r, stream=sp)
        return [((m, c, r), int(r.n)) for m, c, r in zip(ms, cs, rs)]

    def open_session(self, handle, exc: np.ndarray, stream):
        return _GpuSession(self, handle[2], exc, stream)

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


class _GpuSession:
    """A block GMRES solve (cbfm_session_*) that requests may join while it runs."""

    def __init__(self, be: GpuBackend, red, exc: np.ndarray, stream):
        self.C, self.stream = be.C, stream
        self.s = be.C.session(red, exc, tol=be.tol, maxit=be.maxit, restart=be.restart)

    def join(self, exc: np.ndarray) -> Optional[int]:
        try:
            return self.s.join(exc)
        except self.C.CbfmError as e:
            if e.status == 7:       # CBFM_EFULL: finished or full
                return None
            raise

    def run(self) -> Tuple[np.ndarray, np.ndarray]:
        self.s.run(stream=self.stream.cuda_stream, allow_noconv=True)
        rcs, iters, _resid = self.s.results()
        return rcs, iters

    def free(self) -> None:
        self.s.free()


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
class _Group:
    """The requests of one key in a batch: open to joins until its solve finishes."""

    def __init__(self, key, entry: Entry, hit: bool):
        self.key = key
        self.entry = entry
        self.hit = hit
        self.members: List[list] = []     # [request, future, first slot or None]
        self.nrhs = 0
        self.state = "pending"            # pending (joins append) -> running (joins go to the session) -> done
        self.session: Any = None
        self.scratch = 0                  # solve scratch accounted for this group
        self.joined = 0                   # requests that joined after the batch started


class Server:
    """Continuous-batching service.  `submit` returns a Future of `Result`."""

    def __init__(self, backend, hbm_budget: int, n_streams: int = 3, max_batch_rhs: int = MAX_BLOCK_RHS,
                 max_build_keys: int = 4, joins: bool = True):
        self.be = backend
        self.budget = int(hbm_budget)
        self.max_rhs = int(min(max_batch_rhs, MAX_BLOCK_RHS))
        self.max_build_keys = max(1, int(max_build_keys))
        self.joins = joins
        self.lock = threading.Condition()
        self.waiting: List[Tuple[Request, Future]] = []      # arrival order
        self.cache: Dict[Tuple[str, float], Entry] = {}
        self.open: Dict[Tuple[str, float], _Group] = {}      # groups of running batches that take joins
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
            if not self._try_join(req, fut):
                self.waiting.append((req, fut))
                self._dispatch()
        return fut

    def drain(self, timeout: float = 600.0) -> None:
        """Wait until nothing waits or runs (every finished batch is in the log)."""
        end = time.perf_counter() + timeout
        with self.lock:
            while (self.waiting or any(self.busy)) and time.perf_counter() < end:
                self.lock.wait(timeout=0.05)

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
    def _account(self, delta: int) -> None:
        self.inflight += delta
        self.peak_bytes = max(self.peak_bytes, self.resident_bytes() + self.inflight)

    def _try_join(self, req: Request, fut: Future) -> bool:
        """Add a request to the open group of its key: appended while the group
        waits for its build, handed to the running solve session otherwise."""
        g = self.open.get(req.key)
        if not self.joins or g is None or g.state == "done" or g.nrhs + req.nrhs > self.max_rhs:
            return False
        sc = req.scatterer
        delta = solve_bytes(g.entry.n, g.nrhs + req.nrhs, sc.ne) - solve_bytes(g.entry.n, g.nrhs, sc.ne)
        if self.resident_bytes() + self.inflight + delta > self.budget:
            return False
        if g.state == "running":
            slot = g.session.join(req.exc)
            if slot is None:          # the solve has finished or is full
                return False
        else:
            slot = None
        g.members.append([req, fut, slot])
        g.nrhs += req.nrhs
        g.scratch += delta
        g.joined += 1
        self._account(delta)
        return True

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

    def _same_key(self, i: int, key) -> Tuple[list, int]:
        """The waiting requests from index i on with this key, up to max_rhs right-hand sides."""
        group, nrhs = [], 0
        for r2, f2 in self.waiting[i:]:
            if r2.key == key and nrhs + r2.nrhs <= self.max_rhs:
                group.append((r2, f2))
                nrhs += r2.nrhs
        return group, nrhs

    def _take(self, reqs: list) -> None:
        ids = {id(r) for r, _ in reqs}
        self.waiting = [w for w in self.waiting if id(w[0]) not in ids]

    def _new_group(self, key, reqs: list, nrhs: int, hit: bool, entry: Entry, scratch: int) -> _Group:
        g = _Group(key, entry, hit)
        g.members = [[r, f, None] for r, f in reqs]
        g.nrhs = nrhs
        g.scratch = scratch
        self.open[key] = g
        entry.users += 1
        return g

    def _dispatch(self) -> None:
        while self.running and self.waiting and False in self.busy:
            started = False
            for i, (req, _f) in enumerate(self.waiting):
                if req.key in self.open and self._try_join(req, _f):   # an open group took it meanwhile
                    self._take([(req, _f)])
                    started = True
                    break
                group, nrhs = self._same_key(i, req.key)
                need, resident = self._footprint(req, nrhs)
                if need > self.budget:
                    for r2, f2 in group:
                        f2.set_exception(MemoryError(f"request needs {need} bytes, budget {self.budget}"))
                    self._take(group)
                    started = True
                    break
                if self.resident_bytes() + self.inflight + need > self.budget and not self._evict_for(need):
                    continue          # does not fit now; a smaller or resident one may
                self._take(group)
                groups, transient = [], 0
                entry = self.cache.get(req.key)
                if entry is not None:
                    self.hits += 1
                    groups.append(self._new_group(req.key, group, nrhs, True, entry, need))
                    self._account(need)
                else:
                    # a cache miss: when this is the last free worker, other waiting misses of other
                    # keys are built in the same batch (idle workers would rather take them in parallel)
                    todo = [(req.key, group, nrhs, need)]
                    gather = self.busy.count(False) == 1
                    for r3, _f3 in list(self.waiting):
                        if not gather or len(todo) >= self.max_build_keys:
                            break
                        if r3.key in self.cache or r3.key in self.open or any(r3.key == t[0] for t in todo):
                            continue
                        j = next((i for i, w in enumerate(self.waiting) if w[0] is r3), None)
                        if j is None:
                            continue
                        g3, n3 = self._same_key(j, r3.key)
                        if not g3:
                            continue
                        need3, _res3 = self._footprint(r3, n3)
                        if self.resident_bytes() + self.inflight + sum(t[3] for t in todo) + need3 > self.budget:
                            continue
                        todo.append((r3.key, g3, n3, need3))
                        self._take(g3)
                    for key, g3, n3, need3 in todo:
                        self.misses += 1
                        sc = g3[0][0].scatterer
                        n = estimate_n(sc, getattr(self.be, "s", 128))
                        e = Entry(key, n, entry_bytes(sc.nt, sc.ne, n, sc.ncell))
                        self.cache[key] = e
                        tr = build_transient_bytes(sc.nt, sc.ne, n)
                        transient += tr
                        groups.append(self._new_group(key, g3, n3, False, e, need3 - e.bytes - tr))
                        self._account(need3 - e.bytes)
                w = self.busy.index(False)
                self.busy[w] = True
                self.work[w] = (groups, transient, next(self.bid))
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
                groups, transient, bid = self.work[w]
            t_start = time.perf_counter()
            ev0 = self.be.event(st) if self.t0_event is not None else None
            # builds of the cache misses, together
            misses = [g for g in groups if not g.hit]
            build_err: Optional[BaseException] = None
            if misses:
                items = [(g.members[0][0].scatterer, g.members[0][0].freq) for g in misses]
                try:
                    if len(items) > 1 and hasattr(self.be, "build_many"):
                        built = self.be.build_many(items, st)
                    else:
                        built = [self.be.build(sc, f, st) for sc, f in items]
                except BaseException as e:
                    build_err = e
                    built = None
                with self.lock:
                    for k, g in enumerate(misses):
                        sc = items[k][0]
                        if build_err is None:
                            g.entry.handle, g.entry.n = built[k]
                            g.entry.bytes = entry_bytes(sc.nt, sc.ne, g.entry.n, sc.ncell)
                        else:
                            g.entry.error = build_err
                        g.entry.ready.set()
                    self.inflight -= transient          # the builds' scratch is gone
            for g in groups:
                if g.hit:
                    g.entry.ready.wait()
            # the solves, one session per key; joins reach a session while it runs
            for g in groups:
                err: Optional[BaseException] = g.entry.error
                rcs = iters = None
                if err is None:
                    try:
                        with self.lock:
                            exc = np.concatenate([m[0].exc for m in g.members], axis=0)
                            ofs = 0
                            for m in g.members:
                                m[2] = ofs
                                ofs += m[0].nrhs
                            if hasattr(self.be, "open_session"):
                                g.session = self.be.open_session(g.entry.handle, exc, st)
                                g.state = "running"
                            else:
                                g.state = "done"
                                del self.open[g.key]
                        if g.session is not None:
                            rcs, iters = g.session.run()
                        else:
                            rcs, iters = self.be.solve(g.entry.handle, exc, st)
                    except BaseException as e:  # delivered to the requests of the group
                        err = e
                t_end = time.perf_counter()
                with self.lock:
                    if g.state != "done":
                        g.state = "done"
                        if self.open.get(g.key) is g:
                            del self.open[g.key]
                    requeue = []
                    nsolved = 0 if rcs is None else int(rcs.shape[0])
                    for req, fut, slot in g.members:
                        if err is not None:
                            fut.set_exception(err)
                        elif slot is not None and slot + req.nrhs <= nsolved:
                            fut.set_result(Result(req.rid, rcs[slot:slot + req.nrhs], iters[slot:slot + req.nrhs],
                                                  t_end - req.arrival, bid, nsolved, g.hit))
                        else:
                            requeue.append((req, fut))   # joined too late for the solve: wait again
                    if g.session is not None and hasattr(g.session, "free"):
                        g.session.free()
                    self.waiting[0:0] = requeue
            ev1 = self.be.event(st) if ev0 is not None else None
            t_end = time.perf_counter()
            rec = {"batch": bid, "worker": w, "keys": [g.key for g in groups],
                   "requests": sum(len(g.members) for g in groups), "joined": sum(g.joined for g in groups),
                   "rhs": sum(g.nrhs for g in groups), "hit": all(g.hit for g in groups), "t_start": t_start,
                   "t_end": t_end, "error": any(g.entry.error is not None for g in groups)}
            if ev0 is not None:
                rec["dev_ms"] = (self.be.elapsed_ms(self.t0_event, ev0), self.be.elapsed_ms(self.t0_event, ev1))
            with self.lock:
                for g in groups:
                    g.entry.users -= 1
                    g.entry.last_used = t_end
                    if g.entry.error is not None and self.cache.get(g.entry.key) is g.entry:
                        del self.cache[g.entry.key]               # a failed build is not cached
                    self.inflight -= g.scratch
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
           "max_batch_requests": max([b["requests"] for b in log], default=0),
           "mean_batch_keys": float(np.mean([len(b.get("keys", [0])) for b in log])) if log else 0.0,
           "joined_requests": int(sum(b.get("joined", 0) for b in log))}
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
