// internal.cuh -- handle structures and kernel entry points of the library.
#pragma once

#include <memory>
#include <string>
#include <vector>

#include "common.cuh"

namespace cbfm {

enum HandleKind : uint32_t { H_MESH = 0x4d455348u, H_CBF = 0x43424621u, H_RED = 0x52454421u };

struct HandleBase {
    uint32_t kind;
    int device;
};

// Host-side mesh tables (mesh_host.cpp).  Internal edge order: by cell,
// then canonical index, so every cell's edges are contiguous.
struct HostMesh {
    int64_t nv = 0, nt = 0, ne = 0;
    int ncell = 0;
    std::vector<double> verts;       // nv*3
    std::vector<int32_t> tris;       // nt*3
    std::vector<int32_t> canon_u, canon_v;      // canonical edges
    std::vector<int32_t> cell_of_canon;         // ne
    std::vector<int32_t> int_of_canon, canon_of_int;
    std::vector<int32_t> cell_off;              // ncell+1 (internal order)
    std::vector<int32_t> edge_tri, edge_loc;    // (ne,2) internal order: plus, minus
    std::vector<int32_t> tri_edge, tri_sign;    // (nt,3) internal edge ids
    std::vector<double> edge_len;               // internal order
};

void build_host_mesh(const double *verts, int64_t nv, const int32_t *tris, int64_t nt,
                     const int32_t *edge_cell, int32_t ncell, int32_t partition, HostMesh &hm);

struct FusedTables;   // k_fused.cu

struct Mesh : HandleBase {
    HostMesh h;
    double eps_re, eps_im, mu_r, alpha;
    z64 k1, k2, eta1, eta2;
    DevBuf<double> tri64;        // nt * TRI_REC
    DevBuf<float> tri32;         // nt * TRI_REC (centred coordinates)
    DevBuf<int32_t> tri_vid;     // nt*3 vertex ids
    DevBuf<int32_t> tri_edge;    // nt*3 internal edge id
    DevBuf<int32_t> tri_cell;    // nt*3 cell of each of the triangle's RWGs
    DevBuf<int32_t> edge_tri;    // ne*2
    DevBuf<int32_t> edge_loc;    // ne*2
    DevBuf<int32_t> edge_cell;   // ne, cell of each internal edge
    DevBuf<int32_t> near_pairs;  // n_near*2 (t, s), t <= s, both orders needed
    int64_t n_near = 0;
    std::shared_ptr<FusedTables> fused;   // triangle tables per cell (k_fused.cu), built on first use
    DevBuf<double> gram_val;     // ne*6 sparse RWG Gram row values
    DevBuf<int32_t> gram_col;    // ne*6 internal edge columns (-1 unused)
    double centre[3];
};

struct Cbf : HandleBase {
    Mesh *mesh;
    std::vector<int32_t> L;       // per cell
    std::vector<int64_t> coff;    // CBF offsets per cell (ncell+1), within one half
    std::vector<int64_t> boff;    // block offsets sum N_m L_m (ncell+1)
    int64_t nhalf = 0;            // sum L_m
    DevBuf<z64> CM, CJ;           // blocks N_m x L_m row-major, cells in order
    DevBuf<c32> CM32, CJ32;
};

struct Red : HandleBase {
    Mesh *mesh;
    Cbf *cbf;                     // NULL for the conventional MoM system (basis = the RWG functions)
    cbfm_precision prec;
    int64_t n = 0;                // N^CBF
    DevBuf<z64> A64;
    DevBuf<c32> A32;
    DevBuf<z64> G;                // G^CBF dense (n x n)
    DevBuf<z64> Ginv;             // its inverse (FP64)
    DevBuf<c32> Ginv32;
    DevBuf<z64> B64;              // B = A (G^CBF)^{-1}, the operator GMRES iterates with
    DevBuf<c32> B32;
    bool cmp_ready = false;
    // T-diagonal arrangement (Eq. (MoM_T)): Bt = A P D^{-1} (P swaps the column halves),
    // tdinv[k] = 1 / D_{p(k)}: the recovery x_k = y_{p(k)} tdinv[k]
    DevBuf<z64> Bt64;
    DevBuf<c32> Bt32;
    DevBuf<z64> tdinv;
    bool tdiag_ready = false;
    bool tdiag_jacobi = false;
    bool tdiag_swap = true;       // false: Jacobi scaling only (the inner system of the inexact CMP)
    // inexact CMP: G^CBF as a system of its own, iterated with its Jacobi operator G D^{-1}
    std::unique_ptr<Red> ginner;
    double inner_tol = 1e-5;
    int inner_maxit = 1000, inner_restart = 200;
    bool cmp_inexact_ready = false;
};

// ------------------------------------------------------------- kernels
// geometry (k_geom.cu)
void launch_tri_records(Mesh &m, const double *d_verts, const int32_t *d_tris, cudaStream_t st);
void launch_near_pairs(Mesh &m, cudaStream_t st);
void launch_gram_rows(Mesh &m, cudaStream_t st);
// f32: the plane-wave phase factors by FP32 reduced sin/cos (mixed-precision solve), else FP64
void launch_rhs(const Mesh &m, const double *d_waves, int nw, z64 *vE, z64 *vH, cudaStream_t st, bool f32 = false);
void launch_farfield(const Mesh &m, const z64 *j, int nrhs, const double *d_obs, int ndir, bool monostatic,
                     const double *d_exc, double *d_rcs, cudaStream_t st, bool f32 = false);

// assembly (k_assembly.cu): local blocks of all triangle pairs, then the RWG
// matrices Z_op (op = Ks, Ta, Tb), row-major ne x ne, internal edge order.
template <typename T>
void assemble_rwg(Mesh &m, cx<T> *Zrwg, cudaStream_t st, bool diag_cells = false);

// dense complex linear algebra (k_dense.cu)
struct GemmDesc {
    int64_t M, N, K;
    int64_t a_off, lda, b_off, ldb, c_off, ldc;
};
// C[g] = op(A[g]) * op(B[g]) (+ C when accumulate); opA/opB: 0 = N, 1 = T, 2 = H, 3 = conj
// alpha scales the product (C = alpha op(A) op(B) [+ C]).
template <typename T>
void gemm_grouped(const std::vector<GemmDesc> &g, int opA, int opB, const cx<T> *A, const cx<T> *B, cx<T> *C,
                  bool accumulate, cudaStream_t st, double alpha = 1.0);
// Profiling label of the FP64 products launched while an object is alive
// (reported as "site:<label>" beside the kernel's own record).
extern thread_local const char *g_gemm_site;
struct GemmSite {
    const char *prev;
    explicit GemmSite(const char *label) : prev(g_gemm_site) { g_gemm_site = label; }
    ~GemmSite() { g_gemm_site = prev; }
};
// Solve Z_b X_b = V_b in place (V overwritten by X) for nb independent systems of size n_b x n_b, s columns;
// Z and V are overwritten. Returns singular flag per system in d_info (1 = zero pivot).
void lu_solve_batched(int nb, const int64_t *h_zoff, const int64_t *h_voff, const int *h_n, int s, z64 *Z, z64 *V,
                      int *d_info, cudaStream_t st);
// Bounded-wait self-test (cbfm_wait_selftest); true when a wait expired.
bool wait_selftest(int kind, double limit_s, cudaStream_t st);
// One-sided Jacobi SVD of nb column-major s x s complex matrices X (overwritten by U Sigma), V out;
// singular values below keep * sigma_1 (0: none) are not kept by the caller and need not be resolved.
void jacobi_svd_batched(int nb, int s, z64 *X, z64 *V, double *sig, int *d_info, cudaStream_t st,
                        double keep = 0.0);
// In-place Gauss-Jordan inverse of an n x n FP64 complex matrix (row-major); info=1 on zero pivot.
// local blocks and RWG operators of several meshes, one launch per stage (k_assembly.cu)
// diag_cells: only triangle pairs that support RWGs of a common cell are
// evaluated (the cells' diagonal blocks of Z); every other entry is zero
template <typename T>
void assemble_rwg_batch(const std::vector<Mesh *> &ms, const std::vector<cx<T> *> &Z, cudaStream_t st,
                        bool diag_cells = false);
// near-pair blocks only, compact (27 complex64 per pair of each mesh's near list) (k_assembly.cu)
void near_blocks_compact(const std::vector<Mesh *> &ms, const std::vector<c32 *> &out, cudaStream_t st);
// Fused mixed-precision assembly and projection (k_fused.cu): A[k] = (C^JM)^H Z C^MJ
// for each mesh, with no RWG or local-block matrix in device memory.  fused_fits
// tells whether the scatterer's cells fit the kernel's tile limits.
bool fused_fits(const Mesh &m, const Cbf &c);
// the form CBFM_MIXED takes: fused when the unfused scratch (local blocks, RWG
// matrices, split operands) would not fit in a quarter of the free device memory and 16 GiB
bool mixed_takes_fused(const Mesh &m, const Cbf &c);
double unfused_scratch_bytes(const Mesh &m, const Cbf &c);
void assemble_project_fused(const std::vector<Mesh *> &ms, const std::vector<Cbf *> &cs, const std::vector<c32 *> &A,
                            cudaStream_t st);
// tuned launch parameters, per key (api.cu); 0 when not tuned yet
int tuning_get(const std::string &key);
void tuning_set(const std::string &key, int value);
// tensor-core projection of Z (3 x ne x ne, c32) onto the CBFs into A (k_tc.cu)
void project_tc(Mesh &m, Cbf &c, const c32 *Z, c32 *A, cudaStream_t st);
void project_tc_batch(const std::vector<Mesh *> &ms, const std::vector<Cbf *> &cs, const std::vector<const c32 *> &Z,
                      const std::vector<c32 *> &A, cudaStream_t st);
void gauss_jordan_inverse(int64_t n, int nbatch, z64 *Aug, z64 *inv, int *d_info, cudaStream_t st);

// GMRES (k_gmres.cu)
struct GmresOut {
    std::vector<int> iters;
    std::vector<double> resid;
};
// out[r] = M in[r] for rows with mask[r] != 0 (M32 != NULL: complex64 / FP32 arithmetic)
void apply_rows(const Red &rd, const z64 *M64, const c32 *M32, const z64 *in, z64 *out, int nrhs, const int *mask,
                cudaStream_t st);
GmresOut gmres_solve(Red &r, const z64 *d_b, int nrhs, double tol, int maxit, int restart, int pc,
                     z64 *d_x, cudaStream_t st);
// Block GMRES over all right-hand sides at once (k_bgmres.cu); maxit counts block iterations,
// restart caps the basis dimension; iters report the block iteration of convergence.
// Right-hand sides joining a running block solve (the serving loop): polled
// at every block-iteration boundary.
struct BgmresJoin {
    virtual ~BgmresJoin() = default;
    // some right-hand sides wait to join (cheap, any thread)
    virtual bool pending() = 0;
    // the waiting right-hand sides as rows of the reduced system (k x n, device), k returned
    virtual int take(cudaStream_t st, DevBuf<z64> &rows) = 0;
    // every right-hand side has converged: close to further joins unless some wait (then false)
    virtual bool close_if_idle() = 0;
};
// join == nullptr: the right-hand sides d_b (nrhs x n) are solved into d_x.
// With join, right-hand sides may join at block-iteration boundaries (the
// cycle restarts there with them added, y = 0 for the new ones); the
// solutions of all of them, in joining order, go to *x_all (allocated here).
GmresOut bgmres_solve(Red &r, const z64 *d_b, int nrhs, double tol, int maxit, int restart, int pc,
                      z64 *d_x, cudaStream_t st, BgmresJoin *join = nullptr, DevBuf<z64> *x_all = nullptr);
// pc (cbfm_precond): the operator GMRES iterates with, in the reduced system's precision
inline const z64 *pc_op64(const Red &r, int pc) {
    return pc == CBFM_PC_CMP ? r.B64.p : pc == CBFM_PC_TDIAG ? r.Bt64.p : r.A64.p;
}
inline const c32 *pc_op32(const Red &r, int pc) {
    return pc == CBFM_PC_CMP ? r.B32.p : pc == CBFM_PC_TDIAG ? r.Bt32.p : r.A32.p;
}

// T-diagonal arrangement (k_tdiag.cu): builds r.Bt*, r.tdinv (jacobi: D = diag(A P), else I;
// swap = false: P = I, a plain Jacobi scaling); returns false when a diagonal entry is zero
bool tdiag_build(Red &r, bool jacobi, cudaStream_t st, bool swap = true);
// x[q][k] = y[q][p(k)] tdinv[k] for nrhs rows of length r.n
void tdiag_recover(const Red &r, const z64 *y, z64 *x, int nrhs, cudaStream_t st);
// z ~ (G^CBF)^{-1} v for nrhs rows: inner GMRES on r.ginner (inexact CMP)
void cmp_inner_apply(Red &r, const z64 *v, z64 *z, int nrhs, cudaStream_t st);
// the conventional MoM matrix A = [[Ks, Ta], [Tb, Ks]] (2 ne x 2 ne) from Z (3 x ne x ne), internal edge order
template <typename T>
void mom_place(int64_t ne, const cx<T> *Z, cx<T> *A, cudaStream_t st);
// A (n x n, n = 2 ne, internal edge order) -> canonical edge order on both sides
void mom_to_canonical(int64_t ne, const int32_t *d_int_of_canon, const z64 *A, z64 *out, cudaStream_t st);

// export of the reduced matrix without device allocation (noalloc.cu)
void red_export_noalloc(Red &r, double *A, cudaStream_t st);
// loads the export's scratch array on the current device (once per device, from pool_setup)
void noalloc_prepare();

// Per-mesh triangle tables (k_fused.cu; built once per mesh, on first use): for
// every cell the triangles that carry one of its RWG functions (spatially
// ordered), the fused kernel's chunks of them, and the near list as a CSR.
struct FusedTables {
    std::vector<int32_t> tl_off, ch_off;   // per cell: offsets into tl and into the chunk table (host)
    DevBuf<int4> tl;                       // per list entry: {triangle, rows a0 | a1 << 16, row a2 | cols b0, b1 << 24, col b2}
    DevBuf<int32_t> dtl_off, dch_off;
    DevBuf<int2> chunk;                    // per chunk: [begin, end) into tl
    DevBuf<int16_t> chunk_cols;            // per chunk: the fused kernel's cell-local RWG columns (-1: padding)
    DevBuf<float> recT;                    // FP32 triangle records of the list entries, field-major (48 x entries)
    DevBuf<int32_t> vidT;                  // vertex ids of the list entries, field-major (3 x entries)
    DevBuf<int2> rwg_pos;                  // per internal edge: list positions (in its cell's list) of its + and - triangles
    DevBuf<int32_t> near_row;              // nt + 1: CSR of the near list over test triangles
    DevBuf<int2> near_ent;                 // {trial triangle, 2 l + transposed}
    int64_t n_near = 0;
    int nmax = 0;                          // largest N_m
};
FusedTables &fused_tables(Mesh &m, cudaStream_t st);
// near-pair blocks only, compact (27 complex per pair of each mesh's near list),
// FP64 closed forms with FP32 (T = float) or FP64 (T = double) smooth remainders (k_assembly.cu)
template <typename T>
void near_blocks_compact_t(const std::vector<Mesh *> &ms, const std::vector<cx<T> *> &out, cudaStream_t st);
// Z_mm of every cell in FP64, the 2 N_m x 2 N_m matrix [[Ks, Ta], [Tb, Ks]] of its RWG functions
// (row-major, at Zmm + zoff[c]), from the triangle pairs of the cell alone (k_celldiag.cu)
void assemble_cell_diag(Mesh &m, z64 *Zmm, const std::vector<int64_t> &zoff, cudaStream_t st);

// elementwise helpers (k_dense.cu)
void launch_z64_to_c32(const z64 *src, c32 *dst, int64_t n, cudaStream_t st);
void launch_c32_to_z64(const c32 *src, z64 *dst, int64_t n, cudaStream_t st);

}  // namespace cbfm
