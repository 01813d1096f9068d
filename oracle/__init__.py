"""Plain FP64 CPU oracle for the CBFM + CMP PMCHWT hot path.

TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and bench.py's
cpu_baseline / reference legs may import or execute anything in this package.
It shares no code with the CUDA library (paper_2111_11058_gb300), and the
library never imports it.  Inputs come from the `workloads` generators.

Modules
  zmat.c   dense RWG K_i, T_i, plane-wave RHS and far field (plain C, FP64)
  mesh.py  RWG edge table, octant / RCB cell division
  mom.py   PMCHWT matrix Z, RHS v, currents, RCS; conventional MoM solve
  cbfm.py  primary CBFs, dual SVD orthogonalisation, reduced system, CMP,
           GMRES, current recovery
  mie.py   Mie series for a homogeneous dielectric sphere (pin)

Pins (tests/test_oracle_*.py) tie each part to something other than itself;
see the module docstrings for which passage of the paper each follows.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "_zmat.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile zmat.c with the host gcc (no fast-math: IEEE FP64)."""
    src = os.path.join(_HERE, "zmat.c")
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(src):
        tmp = _SO + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-shared", "-fPIC", "-std=c11",
                               "-o", tmp, src, "-lm"])
        os.replace(tmp, _SO)
    return _SO


def lib():
    global _lib
    if _lib is None:
        build()
        _lib = ctypes.CDLL(_SO)
    return _lib
