"""GB300 (sm_103a) CBFM + Calderon-preconditioned PMCHWT solver.

The compute path lives in libcbfm.so (hand-written CUDA, C ABI in
include/cbfm.h); `cbfm` is its thin Python binding, `build` compiles it and
`serve` is the continuous-batching solve service built on the binding.
"""
from .cbfm import (BLOCK, FP64, MIXED, MIXED_SIMT, MIXED_UNFUSED, MIXED_FUSED, PC_CMP, PC_CMP_INEXACT, PC_NONE, PC_TDIAG, PER_RHS, CbfmError,
                   assemble_mom, assemble_reduced, assemble_reduced_batch, build_cbfs, build_ipcbfs, cbf_import,
                   cmp_setup, gram_inverse, launch_count, mesh, mesh_edges, profile, profile_read, session, solve,
                   tdiag_setup, tuning, wait_selftest, WAIT_GRID_EXPIRES, WAIT_CLUSTER_EXPIRES,
                   WAIT_CLUSTER_COMPLETES)

__all__ = ["BLOCK", "PER_RHS", "FP64", "MIXED", "MIXED_SIMT", "MIXED_UNFUSED", "MIXED_FUSED", "PC_NONE", "PC_CMP", "PC_TDIAG", "PC_CMP_INEXACT",
           "CbfmError", "assemble_mom", "assemble_reduced", "assemble_reduced_batch", "build_cbfs", "build_ipcbfs",
           "cbf_import", "cmp_setup", "gram_inverse", "launch_count", "mesh", "mesh_edges", "profile", "profile_read",
           "session", "solve", "tdiag_setup", "tuning", "wait_selftest", "WAIT_GRID_EXPIRES", "WAIT_CLUSTER_EXPIRES",
           "WAIT_CLUSTER_COMPLETES"]
