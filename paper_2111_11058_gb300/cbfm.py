"""Thin ctypes binding of libcbfm.so (include/cbfm.h).

Argument marshalling only: every step of the method runs in the library's
CUDA kernels.  Arrays may be numpy arrays (host) or CUDA torch tensors
(device); outputs come back as numpy arrays unless device tensors are passed
in `out_*` arguments.  Streams are the caller's current torch stream when
torch is present, else the legacy default stream.

Loading fails loudly (CbfmError) when the shared library is missing or was
built for another machine; there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import json
import os
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_HERE, "libcbfm.so")

FP64 = 0
MIXED = 1
MIXED_SIMT = 2   # mixed precision with the projections on the CUDA cores instead of the tensor cores
MIXED_UNFUSED = 3   # mixed precision, RWG matrices assembled in memory, then projected on the tensor cores
MIXED_FUSED = 4     # mixed precision, assembly fused with the tensor-core projection (no RWG matrix in memory)

STATUS = {0: "CBFM_OK", 1: "CBFM_EINVAL", 2: "CBFM_ENOMEM", 3: "CBFM_ECUDA", 4: "CBFM_ESINGULAR",
          5: "CBFM_ENOCONV", 6: "CBFM_ETIMEOUT", 7: "CBFM_EFULL"}

ETA0 = 376.730313668


class CbfmError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


_lib = None
_vp = ctypes.c_void_p
_i64 = ctypes.c_int64
_i32 = ctypes.c_int32
_f64 = ctypes.c_double


def lib():
    """The loaded library (raises CbfmError if it cannot be loaded)."""
    global _lib
    if _lib is None:
        if not os.path.exists(_LIB_PATH):
            raise CbfmError(3, f"{_LIB_PATH} is missing: run paper_2111_11058_gb300.build.build() first")
        try:
            L = ctypes.CDLL(_LIB_PATH)
        except OSError as e:  # pragma: no cover - platform specific
            raise CbfmError(3, f"cannot load {_LIB_PATH}: {e}") from e
        sig = {
            "cbfm_mesh": [_vp, _i64, _vp, _i64, _vp, _i32, _i32, _f64, _f64, _f64, _f64, _vp, _vp],
            "cbfm_mesh_info": [_vp, _vp, _vp, _vp],
            "cbfm_mesh_edges": [_vp, _i64, _vp, _i64, _i32, _i32, _vp, _vp, _vp],
            "cbfm_mesh_cells": [_vp, _vp, _vp],
            "cbfm_build_cbfs": [_vp, _vp, _i32, _f64, _i32, _vp, _vp, _vp, _vp],
            "cbfm_cbf_import": [_vp, _vp, _vp, _vp, _vp, _vp],
            "cbfm_cbf_export": [_vp, _vp, _vp, _vp],
            "cbfm_assemble_reduced": [_vp, _vp, _i32, _vp, _vp, _vp],
            "cbfm_assemble_reduced_batch": [_vp, _vp, _i32, _i32, _vp, _vp, _vp],
            "cbfm_assemble_mom": [_vp, _i32, _vp, _vp, _vp],
            "cbfm_tdiag_setup": [_vp, _i32, _vp],
            "cbfm_build_ipcbfs": [_vp, _vp, _i32, _f64, _i32, _i32, _f64, _i32, _vp, _vp, _vp, _vp, _vp],
            "cbfm_red_export": [_vp, _vp, _vp],
            "cbfm_red_export_noalloc": [_vp, _vp, _vp],
            "cbfm_cmp_setup": [_vp, _vp],
            "cbfm_cmp_setup_inexact": [_vp, _f64, _i32, _i32, _vp],
            "cbfm_gram_export": [_vp, _vp, _vp],
            "cbfm_gram_inverse": [_vp, _i64, _i32, _vp, _vp],
            "cbfm_wait_selftest": [_i32, _f64, _vp],
            "cbfm_solve": [_vp, _vp, _i32, _f64, _i32, _i32, _i32, _i32, _vp, _vp, _i32, _vp, _vp, _vp, _vp],
            "cbfm_session_create": [_vp, _vp, _i32, _f64, _i32, _i32, _i32, _vp],
            "cbfm_session_join": [_vp, _vp, _i32, _vp],
            "cbfm_session_run": [_vp, _vp],
            "cbfm_session_results": [_vp, _i32, _vp, _vp, _vp, _vp],
        }
        for name, args in sig.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = ctypes.c_int
        L.cbfm_free.argtypes = [_vp]
        L.cbfm_free.restype = None
        L.cbfm_last_error.argtypes = []
        L.cbfm_last_error.restype = ctypes.c_char_p
        L.cbfm_launch_count.argtypes = []
        L.cbfm_launch_count.restype = ctypes.c_int64
        L.cbfm_profile.argtypes = [_i32]
        L.cbfm_profile.restype = None
        L.cbfm_profile_read.argtypes = [ctypes.c_char_p, _i64, _i32]
        L.cbfm_profile_read.restype = ctypes.c_int64
        L.cbfm_tuning.argtypes = [ctypes.c_char_p, _i64]
        L.cbfm_tuning.restype = ctypes.c_int64
        _lib = L
    return _lib


def exported_symbols():
    """Names of the C entry points declared in include/cbfm.h."""
    return ["cbfm_mesh", "cbfm_mesh_edges", "cbfm_mesh_info", "cbfm_mesh_cells", "cbfm_build_cbfs", "cbfm_cbf_import",
            "cbfm_cbf_export", "cbfm_assemble_reduced", "cbfm_assemble_reduced_batch", "cbfm_assemble_mom", "cbfm_tdiag_setup", "cbfm_build_ipcbfs", "cbfm_tuning", "cbfm_red_export", "cbfm_red_export_noalloc", "cbfm_cmp_setup", "cbfm_cmp_setup_inexact", "cbfm_gram_export",
            "cbfm_gram_inverse", "cbfm_wait_selftest", "cbfm_solve", "cbfm_session_create", "cbfm_session_join",
            "cbfm_session_run", "cbfm_session_results", "cbfm_free", "cbfm_last_error", "cbfm_launch_count",
            "cbfm_profile", "cbfm_profile_read"]


def _check(st: int):
    if st != 0:
        raise CbfmError(st, lib().cbfm_last_error().decode())


def _stream(stream):
    if stream is not None:
        return ctypes.c_void_p(int(stream))
    try:
        import torch
        if torch.cuda.is_available() and torch.cuda.is_initialized():
            return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    except Exception:  # pragma: no cover
        pass
    return ctypes.c_void_p(0)


def _ptr(a, dtype):
    """(pointer, keepalive) for a numpy array or a torch tensor of `dtype`."""
    if a is None:
        return None, None
    if hasattr(a, "data_ptr") and hasattr(a, "is_cuda"):
        if not a.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return ctypes.c_void_p(a.data_ptr()), a
    arr = np.ascontiguousarray(a, dtype=dtype)
    return ctypes.c_void_p(arr.ctypes.data), arr


def gram_inverse(A, stream=None) -> np.ndarray:
    """cbfm_gram_inverse: inverses of a (nbatch, n, n) complex128 batch by the
    routine cbfm_cmp_setup uses (testing hook)."""
    A = np.ascontiguousarray(A, dtype=np.complex128)
    if A.ndim == 2:
        A = A[None]
    nb, n, n2 = A.shape
    if n != n2:
        raise ValueError("square matrices expected")
    out = np.zeros_like(A)
    _check(lib().cbfm_gram_inverse(ctypes.c_void_p(A.ctypes.data), n, nb, ctypes.c_void_p(out.ctypes.data),
                                   _stream(stream)))
    return out


WAIT_GRID_EXPIRES, WAIT_CLUSTER_EXPIRES, WAIT_CLUSTER_COMPLETES = 0, 1, 2


def wait_selftest(kind: int, limit_s: float = 0.05, stream=None) -> None:
    """cbfm_wait_selftest: a bounded device wait that runs out (kinds 0, 1:
    raises CbfmError with CBFM_ETIMEOUT) or completes (kind 2); testing hook."""
    _check(lib().cbfm_wait_selftest(int(kind), float(limit_s), _stream(stream)))


def launch_count() -> int:
    return int(lib().cbfm_launch_count())


def profile(enable: bool) -> None:
    """Per-kernel CUDA-event timing inside the library on/off."""
    lib().cbfm_profile(1 if enable else 0)


def profile_read(reset: bool = True) -> dict:
    """{kernel: {"launches": n, "ms": total}} accumulated since the last reset."""
    import json
    need = lib().cbfm_profile_read(None, 0, 0)
    buf = ctypes.create_string_buffer(int(need) + 64)
    lib().cbfm_profile_read(buf, len(buf), 1 if reset else 0)
    return json.loads(buf.value.decode())


class _Handle:
    def __init__(self, h):
        self._h = h

    @property
    def handle(self):
        return self._h

    def free(self):
        if getattr(self, "_h", None):
            lib().cbfm_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


class Mesh(_Handle):
    def __init__(self, h, verts):
        super().__init__(h)
        ne = ctypes.c_int64()
        nc = ctypes.c_int32()
        nn = ctypes.c_int64()
        _check(lib().cbfm_mesh_info(h, ctypes.byref(ne), ctypes.byref(nc), ctypes.byref(nn)))
        self.n_edges = int(ne.value)
        self.n_cells = int(nc.value)
        self.n_near = int(nn.value)
        self.n_tris = 2 * self.n_edges // 3

    def cells(self, stream=None) -> np.ndarray:
        out = np.zeros(self.n_edges, np.int32)
        _check(lib().cbfm_mesh_cells(self._h, ctypes.c_void_p(out.ctypes.data), _stream(stream)))
        return out


class CBFs(_Handle):
    def __init__(self, h, mesh: Mesh, L, sigma=None):
        super().__init__(h)
        self.mesh = mesh          # keeps the mesh alive
        self.L = np.asarray(L, np.int32)
        self.sigma = sigma

    def export(self, stream=None):
        """(C^M, C^J) as lists of per-cell (N_m, L_m) complex128 arrays."""
        cells = self.mesh.cells()
        Ns = np.bincount(cells, minlength=self.mesh.n_cells)
        tot = int(np.sum(Ns * self.L))
        CM = np.zeros(tot, np.complex128)
        CJ = np.zeros(tot, np.complex128)
        _check(lib().cbfm_cbf_export(self._h, ctypes.c_void_p(CM.ctypes.data), ctypes.c_void_p(CJ.ctypes.data),
                                     _stream(stream)))
        outM, outJ, off = [], [], 0
        for N, L in zip(Ns, self.L):
            outM.append(CM[off:off + N * L].reshape(N, L))
            outJ.append(CJ[off:off + N * L].reshape(N, L))
            off += N * L
        return outM, outJ


class Reduced(_Handle):
    """A reduced system (cbf set) or the conventional MoM system (cbf None)."""

    def __init__(self, h, cbf: CBFs | None, n: int, prec: int, mesh: Mesh | None = None):
        super().__init__(h)
        self.cbf = cbf
        self.mesh = mesh if mesh is not None else cbf.mesh
        self.n = n
        self.prec = prec

    def export(self, stream=None) -> np.ndarray:
        A = np.zeros((self.n, self.n), np.complex128)
        _check(lib().cbfm_red_export(self._h, ctypes.c_void_p(A.ctypes.data), _stream(stream)))
        return A

    def export_noalloc(self, stream=None) -> np.ndarray:
        """cbfm_red_export_noalloc: as export(), without any device allocation
        (fixed library scratch; n <= 512)."""
        A = np.zeros((self.n, self.n), np.complex128)
        _check(lib().cbfm_red_export_noalloc(self._h, ctypes.c_void_p(A.ctypes.data), _stream(stream)))
        return A

    def gram(self, stream=None) -> np.ndarray:
        G = np.zeros((self.n, self.n), np.complex128)
        _check(lib().cbfm_gram_export(self._h, ctypes.c_void_p(G.ctypes.data), _stream(stream)))
        return G


def mesh(verts, tris, ncell: int, eps_r: complex, partition: str = "rcb", edge_cell=None, mu_r: float = 1.0,
         alpha: float = 2.0, stream=None) -> Mesh:
    """cbfm_mesh: geometry staging and cell division."""
    v, kv = _ptr(verts, np.float64)
    t, kt = _ptr(tris, np.int32)
    c, kc = _ptr(edge_cell, np.int32)
    nv = int(kv.shape[0])
    nt = int(kt.shape[0])
    h = ctypes.c_void_p()
    eps = complex(eps_r)
    _check(lib().cbfm_mesh(v, nv, t, nt, c, int(ncell), 0 if partition == "octant" else 1, eps.real, eps.imag,
                           float(mu_r), float(alpha), _stream(stream), ctypes.byref(h)))
    return Mesh(h, verts)


def mesh_edges(verts, tris, ncell: int, partition: str = "rcb"):
    """cbfm_mesh_edges (host only, no GPU): canonical edges (ne, 2) and the
    built-in cell of each edge (ne,)."""
    v = np.ascontiguousarray(verts, np.float64)
    t = np.ascontiguousarray(tris, np.int32)
    ne = ctypes.c_int64()
    cap = 3 * t.shape[0] // 2
    edges = np.zeros((cap, 2), np.int32)
    cells = np.zeros(cap, np.int32)
    _check(lib().cbfm_mesh_edges(ctypes.c_void_p(v.ctypes.data), v.shape[0], ctypes.c_void_p(t.ctypes.data),
                                 t.shape[0], int(ncell), 0 if partition == "octant" else 1, ctypes.byref(ne),
                                 ctypes.c_void_p(edges.ctypes.data), ctypes.c_void_p(cells.ctypes.data)))
    n = int(ne.value)
    return edges[:n], cells[:n]


def build_cbfs(m: Mesh, waves, delta_svd: float = 1e-3, lmax: int = 0, stream=None) -> CBFs:
    """cbfm_build_cbfs: primary CBFs with the dual SVD orthogonalisation."""
    w, kw = _ptr(waves, np.float64)
    s = int(kw.shape[0])
    L = np.zeros(m.n_cells, np.int32)
    sig = np.zeros((m.n_cells, s), np.float64)
    h = ctypes.c_void_p()
    _check(lib().cbfm_build_cbfs(m.handle, w, s, float(delta_svd), int(lmax), _stream(stream), ctypes.byref(h),
                                 ctypes.c_void_p(L.ctypes.data), ctypes.c_void_p(sig.ctypes.data)))
    return CBFs(h, m, L, sig)


def cbf_import(m: Mesh, CM_blocks, CJ_blocks, stream=None) -> CBFs:
    """cbfm_cbf_import: inject per-cell (N_m, L_m) C^M and C^J blocks."""
    L = np.array([b.shape[1] for b in CM_blocks], np.int32)
    CM = np.ascontiguousarray(np.concatenate([np.asarray(b, np.complex128).ravel() for b in CM_blocks]))
    CJ = np.ascontiguousarray(np.concatenate([np.asarray(b, np.complex128).ravel() for b in CJ_blocks]))
    h = ctypes.c_void_p()
    _check(lib().cbfm_cbf_import(m.handle, ctypes.c_void_p(L.ctypes.data), ctypes.c_void_p(CM.ctypes.data),
                                 ctypes.c_void_p(CJ.ctypes.data), _stream(stream), ctypes.byref(h)))
    return CBFs(h, m, L)


def assemble_reduced(m: Mesh, c: CBFs, prec: int = FP64, stream=None) -> Reduced:
    """cbfm_assemble_reduced: A = (C^JM)^H Z C^MJ."""
    h = ctypes.c_void_p()
    n = ctypes.c_int64()
    _check(lib().cbfm_assemble_reduced(m.handle, c.handle, int(prec), _stream(stream), ctypes.byref(h),
                                       ctypes.byref(n)))
    return Reduced(h, c, int(n.value), prec)


def assemble_reduced_batch(meshes, cbfs, prec: int = MIXED, stream=None) -> list:
    """cbfm_assemble_reduced_batch: reduced systems of several scatterers, one launch per stage."""
    cnt = len(meshes)
    if len(cbfs) != cnt:
        raise ValueError("meshes and cbfs differ in length")
    hm = (ctypes.c_void_p * max(1, cnt))(*[m.handle for m in meshes])
    hc = (ctypes.c_void_p * max(1, cnt))(*[c.handle for c in cbfs])
    out = (ctypes.c_void_p * max(1, cnt))()
    n = np.zeros(max(1, cnt), np.int64)
    _check(lib().cbfm_assemble_reduced_batch(ctypes.cast(hm, ctypes.c_void_p), ctypes.cast(hc, ctypes.c_void_p), cnt,
                                             int(prec), _stream(stream), ctypes.cast(out, ctypes.c_void_p),
                                             ctypes.c_void_p(n.ctypes.data)))
    return [Reduced(ctypes.c_void_p(out[k]), cbfs[k], int(n[k]), prec) for k in range(cnt)]


def assemble_mom(m: Mesh, prec: int = FP64, stream=None) -> Reduced:
    """cbfm_assemble_mom: the conventional MoM matrix Z over all RWG functions (N = 2 ne)."""
    h = ctypes.c_void_p()
    n = ctypes.c_int64()
    _check(lib().cbfm_assemble_mom(m.handle, int(prec), _stream(stream), ctypes.byref(h), ctypes.byref(n)))
    return Reduced(h, None, int(n.value), prec, mesh=m)


def tdiag_setup(r: Reduced, jacobi: bool = True, stream=None) -> None:
    """cbfm_tdiag_setup: T-diagonal arrangement Z_t D^{-1} (D = diag(Z_t) when jacobi, else I)."""
    _check(lib().cbfm_tdiag_setup(r.handle, 1 if jacobi else 0, _stream(stream)))


def build_ipcbfs(mom: Reduced, waves, delta_r: float = 1e-2, delta_svd: float = 1e-3, lmax: int = 0,
                 maxit: int = 5000, restart: int = 200, stream=None) -> CBFs:
    """cbfm_build_ipcbfs: IPCBFs from loose-tolerance GMRES solutions of the whole MoM
    system (a handle from assemble_mom), dual SVD orthogonalised.  The GMRES
    iteration count of every wave is kept in the result's `iters`."""
    if mom.cbf is not None:
        raise ValueError("build_ipcbfs needs a handle from assemble_mom")
    m = mom.mesh
    w, kw = _ptr(waves, np.float64)
    s = int(kw.shape[0])
    L = np.zeros(m.n_cells, np.int32)
    sig = np.zeros((m.n_cells, s), np.float64)
    its = np.zeros(s, np.int32)
    h = ctypes.c_void_p()
    _check(lib().cbfm_build_ipcbfs(mom.handle, w, s, float(delta_r), int(maxit), int(restart), float(delta_svd),
                                   int(lmax), _stream(stream), ctypes.byref(h), ctypes.c_void_p(L.ctypes.data),
                                   ctypes.c_void_p(sig.ctypes.data), ctypes.c_void_p(its.ctypes.data)))
    cb = CBFs(h, m, L, sig)
    cb.iters = its
    return cb


def tuning() -> dict:
    """cbfm_tuning: launch parameters tuned so far in this process."""
    n = lib().cbfm_tuning(None, 0)
    buf = ctypes.create_string_buffer(int(n) + 1)
    lib().cbfm_tuning(buf, len(buf))
    return json.loads(buf.value.decode())


def cmp_setup(r: Reduced, stream=None, inexact: bool = False, inner_tol: float = 1e-5, inner_maxit: int = 1000,
              inner_restart: int = 200) -> None:
    """cbfm_cmp_setup: G^CBF and its inverse; inexact=True: cbfm_cmp_setup_inexact, G^CBF
    applied later by an inner GMRES with D^CBF (solve with precond=PC_CMP_INEXACT)."""
    if inexact:
        _check(lib().cbfm_cmp_setup_inexact(r.handle, float(inner_tol), int(inner_maxit), int(inner_restart),
                                            _stream(stream)))
    else:
        _check(lib().cbfm_cmp_setup(r.handle, _stream(stream)))


@dataclass
class SolveResult:
    j: np.ndarray | None          # (2 ne, nrhs) complex128, canonical edges, [alpha^M; alpha^J]
    rcs: np.ndarray | None        # (nrhs, ndir, 2) partial RCS
    iters: np.ndarray
    resid: np.ndarray
    status: int


PER_RHS = 0
BLOCK = 1

PC_NONE = 0     # K-diagonal system, no preconditioner
PC_CMP = 1      # Calderon multiplicative preconditioner (cmp_setup)
PC_TDIAG = 2    # T-diagonal arrangement (tdiag_setup)
PC_CMP_INEXACT = 3   # CMP with (G^CBF)^{-1} by an inner GMRES (cmp_setup(inexact=True))


def solve(r: Reduced, exc, tol: float = 1e-6, maxit: int = 2000, restart: int = 1000, use_cmp: bool = True,
          obs=None, monostatic: bool = False, want_j: bool = True, out_j=None, out_rcs=None, stream=None,
          allow_noconv: bool = False, solver: int = PER_RHS, precond: int | None = None) -> SolveResult:
    """cbfm_solve: GMRES on the reduced system (solver PER_RHS or BLOCK), currents and RCS.
    precond (PC_NONE, PC_CMP, PC_TDIAG) overrides use_cmp when given."""
    e, ke = _ptr(exc, np.float64)
    nrhs = int(ke.shape[0])
    ne = r.mesh.n_edges
    pc = int(precond) if precond is not None else (PC_CMP if use_cmp else PC_NONE)
    iters = np.zeros(nrhs, np.int32)
    resid = np.zeros(nrhs, np.float64)
    j = None
    if out_j is not None:
        jp, _kj = _ptr(out_j, np.complex128)
    elif want_j:
        j = np.zeros((2 * ne, nrhs), np.complex128)
        jp = ctypes.c_void_p(j.ctypes.data)
    else:
        jp = None
    if monostatic:
        op, ko, nd = None, None, -1
        ndir_out = 1
    elif obs is not None:
        op, ko = _ptr(obs, np.float64)
        nd = int(ko.shape[0])
        ndir_out = nd
    else:
        op, ko, nd, ndir_out = None, None, 0, 0
    rcs = None
    if out_rcs is not None:
        rp, _kr = _ptr(out_rcs, np.float64)
    elif ndir_out > 0:
        rcs = np.zeros((nrhs, ndir_out, 2), np.float64)
        rp = ctypes.c_void_p(rcs.ctypes.data)
    else:
        rp = None
    st = lib().cbfm_solve(r.handle, e, nrhs, float(tol), int(maxit), int(restart), pc, int(solver), jp, op,
                          int(nd), rp, ctypes.c_void_p(iters.ctypes.data), ctypes.c_void_p(resid.ctypes.data),
                          _stream(stream))
    if st != 0 and not (st == 5 and allow_noconv):
        _check(st)
    return SolveResult(j, rcs, iters, resid, st)


class Session(_Handle):
    """cbfm_session_*: a block solve that right-hand sides may join while it runs."""

    def __init__(self, h, red: Reduced):
        super().__init__(h)
        self.red = red

    def join(self, exc) -> int:
        """Queue excitations (n x 3); returns the slot of the first.  CbfmError with
        status 7 (CBFM_EFULL) once the session has finished or is full."""
        e, ke = _ptr(exc, np.float64)
        first = ctypes.c_int32(0)
        _check(lib().cbfm_session_join(self.handle, e, int(ke.shape[0]), ctypes.byref(first)))
        return int(first.value)

    def run(self, stream=None, allow_noconv: bool = False) -> int:
        st = lib().cbfm_session_run(self.handle, _stream(stream))
        if st != 0 and not (st == 5 and allow_noconv):
            _check(st)
        return st

    def results(self):
        """(rcs (nslots, 2), iters (nslots,), resid (nslots,)) in slot order."""
        ns = ctypes.c_int32(0)
        _check(lib().cbfm_session_results(self.handle, 0, None, None, None, ctypes.byref(ns)))
        k = int(ns.value)
        rcs = np.zeros((k, 2), np.float64)
        iters = np.zeros(k, np.int32)
        resid = np.zeros(k, np.float64)
        _check(lib().cbfm_session_results(self.handle, k, ctypes.c_void_p(rcs.ctypes.data),
                                          ctypes.c_void_p(iters.ctypes.data), ctypes.c_void_p(resid.ctypes.data),
                                          ctypes.byref(ns)))
        return rcs, iters, resid


def session(r: Reduced, exc, tol: float = 1e-6, maxit: int = 2000, restart: int = 1000,
            precond: int = PC_CMP) -> Session:
    """cbfm_session_create on reduced system r with the first excitations exc (n x 3)."""
    e, ke = _ptr(exc, np.float64)
    h = ctypes.c_void_p()
    _check(lib().cbfm_session_create(r.handle, e, int(ke.shape[0]), float(tol), int(maxit), int(restart),
                                     int(precond), ctypes.byref(h)))
    return Session(h, r)
