/*
 * cbfm.h -- C ABI of the GB300 (sm_103a) CBFM + Calderon-preconditioned
 * PMCHWT solver for homogeneous dielectric scatterers.
 *
 * Method: K. Tanaka, K. Niino, N. Nishimura, "Characteristic basis function
 * method ... with the Calderon multiplicative preconditioner" (arXiv 2111.11058).
 *
 * Units and conventions
 *   - lengths in free-space wavelengths (k0 = 2 pi); time factor exp(+j w t);
 *   - exterior medium 1 = free space (eta0 = 376.730313668 ohm); interior
 *     medium 2 with k2 = k0 sqrt(eps_r mu_r) (Re > 0, Im <= 0),
 *     eta2 = eta0 sqrt(mu_r / eps_r); eps_r = eps_re + j eps_im, eps_im <= 0;
 *   - a plane wave is a triple (theta, phi, psi): it arrives from direction
 *     r_hat(theta, phi) (travels along -r_hat) with polarisation
 *     cos(psi) theta_hat + sin(psi) phi_hat and unit amplitude;
 *   - RWG edges are numbered canonically: unique vertex pairs (u < v) in
 *     lexicographic order; the plus triangle is the one whose counter-
 *     clockwise vertex order runs u -> v;
 *   - RWG unknowns are ordered j = [alpha^M ; alpha^J] (paper Eq. (coef_vector)).
 *
 * Memory and streams
 *   - every call is stream-ordered on `stream` (a cudaStream_t, NULL = the
 *     legacy default stream) except the host-side mesh preparation inside
 *     cbfm_mesh;
 *   - input arrays may be host or device memory (detected per pointer) and
 *     are copied; output arrays may be host or device memory of the stated
 *     size and are owned by the caller;
 *   - handles own their device memory until cbfm_free; the GPU current when a
 *     handle is created must be current for every later call on it.
 *
 * Errors: every call returns a cbfm_status and never aborts the process; the
 * message of the last failure on the calling thread is cbfm_last_error().
 * Device-side waits are bounded and report CBFM_ETIMEOUT.
 *
 * Call sequence
 *   CBFM with the CMP:   cbfm_mesh -> cbfm_build_cbfs (or cbfm_build_ipcbfs) ->
 *                        cbfm_assemble_reduced -> cbfm_cmp_setup -> cbfm_solve (CBFM_PC_CMP)
 *                        (cbfm_cmp_setup_inexact -> cbfm_solve (CBFM_PC_CMP_INEXACT): the paper's
 *                        inner-GMRES inverse of G^CBF)
 *   conventional MoM:    cbfm_mesh -> cbfm_assemble_mom -> cbfm_tdiag_setup(jacobi = 1) ->
 *                        cbfm_solve (CBFM_PC_TDIAG)
 *   T-diagonal CBFM:     ... cbfm_assemble_reduced -> cbfm_tdiag_setup(jacobi = 0) ->
 *                        cbfm_solve (CBFM_PC_TDIAG)
 *   every handle ends with cbfm_free.
 */
#ifndef CBFM_H
#define CBFM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct cbfm_mesh_s *cbfm_mesh_t;
typedef struct cbfm_cbf_s *cbfm_cbf_t;
typedef struct cbfm_red_s *cbfm_red_t;
typedef struct cbfm_session_s *cbfm_session_t;

typedef enum {
    CBFM_OK = 0,
    CBFM_EINVAL = 1,      /* bad argument, size or mesh */
    CBFM_ENOMEM = 2,      /* device or host allocation failed */
    CBFM_ECUDA = 3,       /* CUDA runtime error */
    CBFM_ESINGULAR = 4,   /* zero pivot in an LU / Gauss-Jordan factorisation */
    CBFM_ENOCONV = 5,     /* GMRES reached maxit without meeting tol (results are the last iterate) */
    CBFM_ETIMEOUT = 6,    /* a bounded device wait expired */
    CBFM_EFULL = 7        /* a solve session has finished or holds 128 right-hand sides */
} cbfm_status;

typedef enum {
    CBFM_FP64 = 0,        /* every step in FP64 (reference GPU path) */
    CBFM_MIXED = 1,       /* FP32 far-pair quadrature; projections on the tensor cores
                             (split-TF32 products, FP32 accumulation); complex64 reduced
                             matrix; FP64 singular near pairs, SVD, CMP Gram inverse,
                             GMRES Arnoldi / residual.  Chooses the faster form that fits:
                             CBFM_MIXED_UNFUSED when its RWG matrices fit in a quarter of
                             the free device memory and 16 GiB, else CBFM_MIXED_FUSED
                             (when the cells fit its tiles) */
    CBFM_MIXED_SIMT = 2,  /* as CBFM_MIXED, but the projections run as FP32 products on
                             the CUDA cores (for comparison with the tensor-core path) */
    CBFM_MIXED_UNFUSED = 3,  /* RWG matrices Z assembled in device memory (27 T^2 + 7 N^2 / 4
                             complex64 entries of scratch), then projected by a separate
                             tensor-core GEMM */
    CBFM_MIXED_FUSED = 4  /* assembly fused with the tensor-core projection, per cell pair:
                             no local-block or RWG matrix in device memory.  Its tiles take
                             cells with L_m <= 32 CBFs and N_m <= 256 RWG functions; a
                             scatterer with a larger cell is assembled as CBFM_MIXED_UNFUSED */
} cbfm_precision;

/* Right preconditioner / unknown arrangement of cbfm_solve (its `precond` argument). */
typedef enum {
    CBFM_PC_NONE = 0,     /* the K-diagonal system as assembled (Eq. (Z) order), no preconditioner */
    CBFM_PC_CMP = 1,      /* Calderon multiplicative preconditioner (G^CBF)^{-1} (cbfm_cmp_setup) */
    CBFM_PC_TDIAG = 2,    /* T-diagonal arrangement with optional Jacobi scaling (cbfm_tdiag_setup) */
    CBFM_PC_CMP_INEXACT = 3   /* CMP with (G^CBF)^{-1} by an inner GMRES (cbfm_cmp_setup_inexact) */
} cbfm_precond;

/*
 * cbfm_mesh -- geometry staging of a closed triangle surface (paper Sec. II-B,
 * RWG functions; Sec. III-A, division into cells).
 *   verts     (nv, 3) float64, row-major
 *   tris      (nt, 3) int32, counter-clockwise seen from outside
 *   edge_cell (ne) int32 cell of each canonical edge, or NULL for the built-in
 *             partition: ncell == 8 with partition 0 -> octants of the edge
 *             midpoint (a coordinate counts negative below -1e-12 * max|vertex|);
 *             otherwise recursive coordinate bisection of edge midpoints into
 *             ncell parts (longest axis, lower part floor(M/2) cells and
 *             round(n floor(M/2)/M) edges, ties by edge index)
 *   partition 0 = octant (ncell must be 8), 1 = RCB; ignored when edge_cell given
 *   eps_re, eps_im, mu_r   interior medium; near-pair factor alpha (> 0): a
 *             triangle pair is near when it shares a vertex or its centroid
 *             distance is below alpha * max(longest edge)
 * Fails with CBFM_EINVAL for open, non-manifold or inconsistently oriented
 * meshes, an empty cell, or sizes beyond int32.
 */
cbfm_status cbfm_mesh(const double *verts, int64_t nv, const int32_t *tris, int64_t nt,
                      const int32_t *edge_cell, int32_t ncell, int32_t partition,
                      double eps_re, double eps_im, double mu_r, double alpha,
                      void *stream, cbfm_mesh_t *out);

/*
 * cbfm_mesh_edges -- host-only variant of the edge table and built-in cell
 * division of cbfm_mesh (no GPU needed; same rules).  verts/tris are host
 * arrays.  n_edges out; edges (ne, 2) int32 canonical (u < v) and cells (ne)
 * int32 may be NULL; when given they must hold 3 nt / 2 entries.
 */
cbfm_status cbfm_mesh_edges(const double *verts, int64_t nv, const int32_t *tris, int64_t nt, int32_t ncell,
                            int32_t partition, int64_t *n_edges, int32_t *edges, int32_t *cells);

/* Number of canonical RWG edges (N = 2 * edges unknowns), of cells and of
 * near triangle pairs (t <= s, self pairs included); NULL outputs are skipped. */
cbfm_status cbfm_mesh_info(cbfm_mesh_t mesh, int64_t *n_edges, int32_t *n_cells, int64_t *n_near);

/* Cell of each canonical edge (ne int32, host or device). */
cbfm_status cbfm_mesh_cells(cbfm_mesh_t mesh, int32_t *edge_cell, void *stream);

/*
 * cbfm_build_cbfs -- primary CBFs with the dual SVD orthogonalisation
 * (paper Sec. III-A Eq. (pcbf); Sec. III-B Eqs. (gram_CBF), (gram_CBF_SVD), (CBF)).
 *   waves      (s, 3) generating plane waves (theta, phi, psi)
 *   delta_svd  keep singular values with sigma_i / sigma_1 >= delta_svd
 *   lmax       cap on L_m (<= 0: none)
 *   L_per_cell out (ncell) int32, host
 *   sigma_out  out (ncell, s) float64 normalised singular values of G'_m, or NULL
 * Runs in FP64.  Requires s <= 1024 and 2 N_m <= 4096.
 */
cbfm_status cbfm_build_cbfs(cbfm_mesh_t mesh, const double *waves, int32_t s, double delta_svd,
                            int32_t lmax, void *stream, cbfm_cbf_t *out, int32_t *L_per_cell,
                            double *sigma_out);

/*
 * cbfm_cbf_import / export -- inject or read the dual CBFs.
 *   L_per_cell (ncell) int32 host;  CM, CJ: complex128 arrays holding, cell
 *   after cell, the N_m x L_m row-major blocks C_m^M and C_m^J with rows in
 *   increasing canonical edge order of the cell.  Total sum_m N_m L_m each.
 */
cbfm_status cbfm_cbf_import(cbfm_mesh_t mesh, const int32_t *L_per_cell, const double *CM,
                            const double *CJ, void *stream, cbfm_cbf_t *out);
cbfm_status cbfm_cbf_export(cbfm_cbf_t cbf, double *CM, double *CJ, void *stream);

/*
 * cbfm_assemble_reduced -- reduced matrix A = (C^JM)^H Z C^MJ (paper Eq.
 * (CBFM_outer)) with Z the PMCHWT Galerkin matrix (Eq. (Z)) assembled from
 * 7-point quadrature (far pairs) and singularity extraction (near pairs).
 *   n_cbf out: N^CBF = 2 sum_m L_m.
 * Row/column order of A: [J-tested / M-coefficient CBFs of cells 0..M-1,
 * M-tested / J-coefficient CBFs of cells 0..M-1].
 */
cbfm_status cbfm_assemble_reduced(cbfm_mesh_t mesh, cbfm_cbf_t cbf, cbfm_precision prec,
                                  void *stream, cbfm_red_t *out, int64_t *n_cbf);

/*
 * cbfm_assemble_reduced_batch -- cbfm_assemble_reduced for `count` scatterers
 * at once (mixed precision only: prec CBFM_MIXED or CBFM_MIXED_FUSED).  The
 * scatterers that take the fused form (all that fit its tiles under
 * CBFM_MIXED_FUSED; under CBFM_MIXED those whose unfused scratch would not
 * fit) are assembled by one launch of the near-pair stage and one launch of the
 * fused assembly-projection kernel over all their cell pairs: persistent CTAs take (scatterer, test cell,
 * trial cell) items from an atomic counter, largest first, so scatterers of
 * uneven size share the GPU.  The others go through the unfused stages (far
 * pairs with a strip width picked on the first call per device by timing the
 * candidates, see cbfm_tuning; near pairs; RWG gather; two tensor-core GEMMs),
 * in waves whose transient operators fit in half of the free device memory and
 * in 6 GiB.
 *   meshes, cbfs  count handles (cbfs[k] built on meshes[k])
 *   out           count new reduced-system handles (NULL on failure)
 *   n_cbf         out, count values of N^CBF (may be NULL)
 * Each out[k] equals what cbfm_assemble_reduced(meshes[k], cbfs[k], prec)
 * returns (up to the summation order of the fused kernel's FP32 atomic adds:
 * last-bit differences).  Returns after the work has completed.
 */
cbfm_status cbfm_assemble_reduced_batch(const cbfm_mesh_t *meshes, const cbfm_cbf_t *cbfs, int32_t count,
                                        cbfm_precision prec, void *stream, cbfm_red_t *out, int64_t *n_cbf);

/*
 * cbfm_tuning -- the launch parameters tuned so far in this process, as a
 * JSON object {"name": value, ...} written to buf (NUL-terminated, truncated
 * to cap bytes).  Returns the length of the full text.  Library service; the
 * paper has no counterpart.
 */
int64_t cbfm_tuning(char *buf, int64_t cap);

/*
 * cbfm_assemble_mom -- the conventional method of moments (paper Sec. IV,
 * the comparison method): the PMCHWT Galerkin matrix Z of Eq. (Z) over all N =
 * 2 ne RWG functions, from the same far-pair quadrature and near-pair
 * singularity extraction as cbfm_assemble_reduced, with no CBFs.  The result
 * is a reduced-system handle whose basis functions are the RWG functions
 * themselves (C^M = C^J = I):
 *   - cbfm_solve takes it with precond CBFM_PC_NONE or CBFM_PC_TDIAG; the
 *     right-hand side is v = [v^E; v^H] and the solution the RWG currents;
 *   - cbfm_red_export returns Z (N x N) in canonical edge order, columns
 *     [alpha^M; alpha^J], rows [E-tested; H-tested];
 *   - cbfm_cmp_setup and cbfm_red_export_noalloc refuse it (CBFM_EINVAL): a
 *     Calderon preconditioner on RWG functions alone has a singular Gram
 *     matrix (Sec. III-A).
 *   prec  CBFM_FP64 (complex128 Z) or a mixed mode (FP32 far pairs, complex64 Z)
 *   n     out, N = 2 ne (may be NULL)
 * Memory: 7 N^2/4 complex entries while assembling, N^2 kept.
 */
cbfm_status cbfm_assemble_mom(cbfm_mesh_t mesh, cbfm_precision prec, void *stream, cbfm_red_t *out, int64_t *n);

/*
 * cbfm_tdiag_setup -- the T-diagonal arrangement of Eq. (MoM_T) for a handle
 * from cbfm_assemble_mom or cbfm_assemble_reduced.  The operator's two column
 * halves are swapped (Z_t = Z P: unknowns [alpha^J; alpha^M], so that the
 * diagonal blocks hold the T operators), then right-scaled by D^{-1}:
 *   jacobi != 0: D = diag(Z_t), the diagonal preconditioner of the paper's
 *                conventional MoM;
 *   jacobi == 0: D = I; on a reduced system this is the T-diagonal CBFM of
 *                Eq. (cbfm_Tdiag), whose matrix (C^JM)^H Z_t C^JM is A with its
 *                column halves swapped and whose right-hand side is unchanged.
 * cbfm_solve with precond CBFM_PC_TDIAG then runs GMRES on Z_t D^{-1} y = b and
 * returns x = P D^{-1} y in the K-diagonal unknown order.  The scaled operator
 * (N^2 entries) is kept in the handle; a later call replaces it.  Returns
 * CBFM_ESINGULAR when jacobi != 0 and a diagonal entry of Z_t is zero.
 */
cbfm_status cbfm_tdiag_setup(cbfm_red_t red, int32_t jacobi, void *stream);

/*
 * cbfm_build_ipcbfs -- IPCBFs, GMRES version (paper Sec. III-A, the proposal
 * after Eq. (ipcbf)), with the dual SVD orthogonalisation of cbfm_build_cbfs.
 * Every generating wave's whole-system MoM problem, in the arrangement of Eq.
 * (MoM_T) with its diagonal preconditioner, is solved by per-RHS GMRES and
 * stopped at the relative residual delta_r; the coefficient sets J_m^M, J_m^J
 * of cell m are those solutions restricted to the cell's RWG functions.  Unlike
 * primary CBFs they carry the coupling between cells, so a connected
 * scatterer divided into cells has no fictitious open edges.
 *   mom        handle from cbfm_assemble_mom on the mesh the CBFs are for (its
 *              T-diagonal Jacobi operator is built here if cbfm_tdiag_setup
 *              was not called with jacobi != 0); its precision is the solve's
 *   waves      (s, 3) generating plane waves (theta, phi, psi), s <= 1024
 *   delta_r    GMRES residual allowance (the paper uses 1e-1 to 1e-3)
 *   maxit, restart  GMRES limits per wave
 *   delta_svd, lmax, L_per_cell, sigma_out   as for cbfm_build_cbfs
 *   iters_out  (s) int32 GMRES iterations per wave, or NULL
 *   out        new CBF handle for mom's mesh
 * Returns CBFM_ENOCONV (and no handle) when a wave does not reach delta_r.
 */
cbfm_status cbfm_build_ipcbfs(cbfm_red_t mom, const double *waves, int32_t s, double delta_r, int32_t maxit,
                              int32_t restart, double delta_svd, int32_t lmax, void *stream, cbfm_cbf_t *out,
                              int32_t *L_per_cell, double *sigma_out, int32_t *iters_out);

/* A as complex128 row-major (n_cbf, n_cbf), host or device. */
cbfm_status cbfm_red_export(cbfm_red_t red, double *A, void *stream);

/*
 * cbfm_red_export_noalloc -- the same output as cbfm_red_export for callers
 * that cannot allocate device memory at the time of the call (a serving
 * process whose HBM is full of cached matrices, an allocator that forbids
 * cudaMalloc, a thread that must not trigger the device-wide synchronisation
 * cudaMalloc/cudaFree may cause).  The paper has no counterpart: this is a
 * library service, not part of the method.
 *   Calls no cudaMalloc, cudaFree or allocating library routine.  A mixed-
 *   precision matrix is widened to complex128 in a fixed 4 MiB scratch array
 *   built into the library, so n_cbf must be <= 512; larger systems, and
 *   conventional-MoM handles, return CBFM_EINVAL.
 *   CUDA loads the scratch array on a device lazily; the library does so in
 *   its first call on each device (any entry point, e.g. cbfm_mesh), which is
 *   where those 4 MiB are taken and then held until the process exits, so the
 *   export itself never needs new device memory.  Each call looks the array's
 *   device address up again (cudaGetSymbolAddress with the handle's device
 *   current), so a re-created context is handled.  Like every entry point it
 *   synchronises `stream`: never call it on a stream that is being captured.
 *   All calls share the one scratch array, which keeps the last call's
 *   contents: calls that overlap on the GPU (different streams or threads)
 *   race and must be serialised by the caller.  Returns after the copy into A
 *   (host or device) has completed.
 */
cbfm_status cbfm_red_export_noalloc(cbfm_red_t red, double *A, void *stream);

/*
 * cbfm_cmp_setup -- CBF Gram matrix G^CBF = (C^JM)^H G_ffff C^MJ (paper Eq.
 * (CBF_Gram_matrix)) and the inverse of each of its two diagonal halves in
 * FP64 (the off-half blocks are zero): Gauss-Jordan elimination with 32 x 32
 * block pivots (no row exchanges between blocks), kept when every diagonal
 * block's pivots stay above 1e-13 of its largest entry and A^{-1}(A x)
 * reproduces a fixed probe x to 1e-8; otherwise Gauss-Jordan with partial
 * pivoting.  Returns CBFM_ESINGULAR on a zero pivot.
 */
cbfm_status cbfm_cmp_setup(cbfm_red_t red, void *stream);

/*
 * cbfm_cmp_setup_inexact -- the CMP as the paper applies it (Sec. III-C, after
 * Eq. (CBFM_inner); Sec. IV): G^CBF as in cbfm_cmp_setup, but no inverse.
 * Every application of (G^CBF)^{-1} inside cbfm_solve (precond
 * CBFM_PC_CMP_INEXACT: once per outer GMRES step and once for j^CBF) is an
 * inner per-RHS GMRES on G^CBF z = v, right-preconditioned by the diagonal
 * D^CBF = 1 / diag(G^CBF), FP64, x0 = 0, stopped at relative residual
 * inner_tol (the paper: 1e-5) or after inner_maxit steps (restart
 * inner_restart).  The outer preconditioner then varies slightly from step to
 * step, as in the paper.  Returns CBFM_ESINGULAR when a diagonal entry of
 * G^CBF is zero.
 */
cbfm_status cbfm_cmp_setup_inexact(cbfm_red_t red, double inner_tol, int32_t inner_maxit, int32_t inner_restart,
                                   void *stream);

/*
 * cbfm_wait_selftest -- a testing hook for the bounded device waits (the paper
 * has no counterpart).  Every wait of the library's kernels on other CTAs (the
 * grid barrier of the persistent Gauss-Jordan kernels, the cluster barriers of
 * the Cholesky and Jacobi kernels) gives up after a time limit, sets an error
 * word and lets the kernel end, so the call returns CBFM_ETIMEOUT and the
 * device stays usable.  kind 0: a grid barrier awaited by 4 CTAs for 5
 * arrivals (its fixed limit, one second, expires); kind 1: a cluster barrier
 * of 2 CTAs initialised for 3 arrivals (expires after limit_s); kind 2: the
 * same barrier for 2 arrivals (completes).  limit_s in (0, 1].  Returns
 * CBFM_ETIMEOUT when the wait expired, CBFM_OK when it completed, CBFM_EINVAL
 * on bad arguments.
 */
cbfm_status cbfm_wait_selftest(int32_t kind, double limit_s, void *stream);

/*
 * cbfm_gram_inverse -- the inverse routine of cbfm_cmp_setup applied to
 * caller matrices: a testing hook for both of its paths (the paper has no
 * counterpart).  A: nbatch complex128 row-major n x n matrices, consecutive,
 * host or device (read only); Ainv: the inverses in the same layout, host or
 * device, caller-owned.  Returns CBFM_ESINGULAR when a matrix is singular to
 * working precision, CBFM_EINVAL on bad arguments.
 */
cbfm_status cbfm_gram_inverse(const double *A, int64_t n, int32_t nbatch, double *Ainv, void *stream);

/* G^CBF as complex128 row-major (n_cbf, n_cbf), host or device; after cbfm_cmp_setup or cbfm_cmp_setup_inexact. */
cbfm_status cbfm_gram_export(cbfm_red_t red, double *G, void *stream);

/*
 * cbfm_solve -- right-preconditioned GMRES on A (G^CBF)^{-1} y = (C^JM)^H v
 * (Eqs. (CBFM_outer), (CBFM_inner)), j^CBF = (G^CBF)^{-1} y, j = C^MJ j^CBF
 * (Eq. (trans_current)), far field and RCS.  Each right-hand side runs its own
 * GMRES (x0 = 0, restart `restart`, stop at ||b - A P y|| / ||b|| <= tol).
 *   exc     (nrhs, 3) excitations (theta, phi, psi)
 *   precond CBFM_PC_CMP: P = (G^CBF)^{-1} (requires cbfm_cmp_setup);
 *           CBFM_PC_NONE: P = I; CBFM_PC_TDIAG: P = (column-half swap) D^{-1}
 *           as set by cbfm_tdiag_setup (required); CBFM_PC_CMP_INEXACT: P =
 *           the inner GMRES of cbfm_cmp_setup_inexact (required)
 *   j_out   (2 ne, nrhs) complex128 RWG coefficients in canonical edge order, or NULL
 *   obs     (ndir, 2) observation directions (theta, phi); obs == NULL with
 *           ndir == -1 selects monostatic: each RHS observed at its own arrival
 *           direction (ndir = 1 per RHS)
 *   rcs_out (nrhs, ndir, 2) float64 partial RCS (sigma_theta, sigma_phi) =
 *           4 pi |F_theta|^2, 4 pi |F_phi|^2, or NULL
 *   iters_out (nrhs) int32 GMRES iterations, or NULL
 *   resid_out (nrhs) float64 final relative residuals, or NULL
 *   solver  0: one GMRES per right-hand side (maxit / restart count Arnoldi
 *           steps, iters_out the steps to convergence);
 *           1: block GMRES over groups of up to 128 right-hand sides sharing one
 *           block Krylov space (maxit counts block iterations, restart caps the
 *           basis dimension, iters_out is the block iteration of convergence);
 *           each right-hand side still stops on its own residual criterion.
 * Returns CBFM_ENOCONV when some RHS did not converge within maxit.
 */
cbfm_status cbfm_solve(cbfm_red_t red, const double *exc, int32_t nrhs, double tol, int32_t maxit,
                       int32_t restart, int32_t precond, int32_t solver, double *j_out, const double *obs,
                       int32_t ndir, double *rcs_out, int32_t *iters_out, double *resid_out,
                       void *stream);

/* ---------------------------------------------------------------------
 * Solve sessions: block GMRES (paper Eqs. (CBFM_outer)/(CBFM_inner), the
 * right-preconditioned reduced system) on a set of right-hand sides that
 * may grow while the solve runs -- continuous batching in the serving loop.
 *
 * cbfm_session_create -- a session on a CMP-ready (or T-diagonal / plain)
 *   reduced system with its first 1-128 monostatic excitations exc
 *   (nrhs x (theta, phi, pol), host, copied); tol, maxit (block iterations),
 *   restart (basis dimensions) and precond as for cbfm_solve.  The session
 *   is owned by the caller until cbfm_free.
 * cbfm_session_join -- queue nrhs more excitations (host, copied); any
 *   thread, also while cbfm_session_run runs.  *first_slot (nullable)
 *   receives the slot of the first one; slots number the right-hand sides
 *   in the order they were accepted.  CBFM_EFULL once the session has
 *   finished or would exceed 128 right-hand sides.
 * cbfm_session_run -- runs the solve on the caller's stream: queued
 *   right-hand sides are taken at every block-iteration boundary (the
 *   running cycle restarts there with them added: their starting guess is
 *   zero, the others keep their iterate and the converged ones stay out of
 *   the new block); when every right-hand side has converged and nothing is
 *   queued the session closes.  Then currents and monostatic RCS for every
 *   slot.  Once per session; CBFM_ENOCONV as cbfm_solve.  Joins still
 *   queued when maxit ends the solve get no result (the slot count below
 *   tells).
 * cbfm_session_results -- after run: *nslots (nullable) = slots solved;
 *   with capacity >= that, rcs_out (nslots x 2, the |E_theta|^2 and
 *   |E_phi|^2 parts of the monostatic RCS as cbfm_solve), iters_out
 *   (block iterations since the slot joined) and resid_out (nullable each).
 */
cbfm_status cbfm_session_create(cbfm_red_t red, const double *exc, int32_t nrhs, double tol, int32_t maxit,
                                int32_t restart, int32_t precond, cbfm_session_t *out);
cbfm_status cbfm_session_join(cbfm_session_t sess, const double *exc, int32_t nrhs, int32_t *first_slot);
cbfm_status cbfm_session_run(cbfm_session_t sess, void *stream);
cbfm_status cbfm_session_results(cbfm_session_t sess, int32_t capacity, double *rcs_out, int32_t *iters_out,
                                 double *resid_out, int32_t *nslots);

/* Release any handle (mesh, cbf, reduced system or session); NULL is a no-op. */
void cbfm_free(void *handle);

/* Message of the last failed call on this thread ("" if none). */
const char *cbfm_last_error(void);

/* Kernel launches issued by this process so far (all entry points). */
int64_t cbfm_launch_count(void);

/*
 * cbfm_profile -- per-kernel timing with CUDA events recorded on the
 * launching stream around the main kernels (enable != 0 turns it on).
 * cbfm_profile_read writes a JSON object {name: {"launches": n, "ms": t,
 * "flop": f, "bytes": b}} (f, b: algorithmic floating-point operations and
 * bytes attributed to the kernel, 0 where not counted)
 * into buf (capacity cap, NUL-terminated, truncated if short), returns the
 * size needed, and clears the totals when reset != 0.
 */
void cbfm_profile(int32_t enable);
int64_t cbfm_profile_read(char *buf, int64_t cap, int32_t reset);

#ifdef __cplusplus
}
#endif
#endif /* CBFM_H */
