// k_celldiag.cu -- the diagonal blocks Z_mm of the cells in FP64, for the
// primary CBFs (paper Eq. (pcbf): Z_mm J_m = V_m, Sec. III-A), with storage of
// the order of the cells themselves (no matrix over the whole mesh).
//
// For every cell m the triangles carrying one of its RWG functions (its list
// T_m, from the per-mesh triangle tables) are paired with each other:
//   stage 1 (k_diag_local): the 27 local entries (op x 3 x 3, op = Ks, Ta, Tb)
//     of every pair in T_m x T_m -- the far-pair quadrature of far_math.cuh in
//     FP64, or the FP64 block of the near-pair stage;
//   stage 2 (k_diag_gather): Z_op[i][j] for the cell's RWG functions i, j as
//     the sum over the 2 x 2 triangle pairs of their supports, written as the
//     2 N_m x 2 N_m matrix [[Ks, Ta], [Tb, Ks]] (row-major).
// The near/far classification and both evaluations are those of the full
// assembly, so Z_mm equals the corresponding block of the whole-mesh Z.
#include <algorithm>
#include <vector>

#include "far_math.cuh"

namespace cbfm {

namespace {

using namespace fm;

// Stage 1: one thread per pair (t, s) of a cell's list, grid-stride over all cells.
__global__ void k_diag_local(int nc, const int64_t *__restrict__ poff, const int32_t *__restrict__ tl_off,
                             const int4 *__restrict__ tl, const double *__restrict__ rec64,
                             const int32_t *__restrict__ vid, const int32_t *__restrict__ near_row,
                             const int2 *__restrict__ near_ent, const z64 *__restrict__ near_val, MediaT<double> md,
                             double alpha, z64 *__restrict__ Lb, int *__restrict__ err) {
    const int64_t total = poff[nc];
    for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < total; g += (int64_t)gridDim.x * blockDim.x) {
        int lo = 0, hi = nc - 1;   // cell of pair g
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (poff[mid] <= g) lo = mid;
            else hi = mid - 1;
        }
        const int c = lo;
        const int t0 = tl_off[c], nT = tl_off[c + 1] - t0;
        const int64_t q = g - poff[c];
        const int ti = (int)(q / nT), si = (int)(q - (int64_t)ti * nT);
        const int t = tl[t0 + ti].x, s = tl[t0 + si].x;
        z64 out[NCOMP];
        const int32_t vt[3] = {vid[3 * t], vid[3 * t + 1], vid[3 * t + 2]};
        const int32_t vs[3] = {vid[3 * s], vid[3 * s + 1], vid[3 * s + 2]};
        const double *rt = rec64 + (int64_t)t * TRI_REC, *rs = rec64 + (int64_t)s * TRI_REC;
        if (is_near(rt, rs, vt, vs, alpha)) {
            int code = -1;
            for (int e = near_row[t]; e < near_row[t + 1]; ++e)
                if (near_ent[e].x == s) {
                    code = near_ent[e].y;
                    break;
                }
            if (code < 0) {
                atomicExch(err, 1);
                for (int k = 0; k < NCOMP; ++k) out[k] = z64(0, 0);
            } else {
                const z64 *b = near_val + (int64_t)(code >> 1) * NCOMP;
                const bool tr = code & 1;
                for (int op = 0; op < 3; ++op)
                    for (int a = 0; a < 3; ++a)
                        for (int bb = 0; bb < 3; ++bb) out[op * 9 + 3 * a + bb] = b[op * 9 + (tr ? 3 * bb + a : 3 * a + bb)];
            }
        } else {
            far_entries<double>(rt, 1, rs, md, out);
        }
        z64 *dst = Lb + g * NCOMP;
        for (int k = 0; k < NCOMP; ++k) dst[k] = out[k];
    }
}

// Stage 2: one block per (slice of rows, cell).
__global__ void k_diag_gather(int nc, const int32_t *__restrict__ cell_off, const int32_t *__restrict__ tl_off,
                              const int64_t *__restrict__ poff, const int64_t *__restrict__ zoff,
                              const int2 *__restrict__ rwg_pos, const int32_t *__restrict__ edge_loc,
                              const z64 *__restrict__ Lb, z64 *__restrict__ Zmm) {
    const int c = blockIdx.y;
    const int64_t off = cell_off[c], N = cell_off[c + 1] - off, n2 = 2 * N;
    const int nT = tl_off[c + 1] - tl_off[c];
    const z64 *L = Lb + poff[c] * NCOMP;
    for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < N * N;
         idx += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = idx / N, j = idx - i * N;
        const int2 pi = rwg_pos[off + i], pj = rwg_pos[off + j];
        const int ai[2] = {edge_loc[2 * (off + i)], edge_loc[2 * (off + i) + 1]};
        const int aj[2] = {edge_loc[2 * (off + j)], edge_loc[2 * (off + j) + 1]};
        const int ti[2] = {pi.x, pi.y}, tj[2] = {pj.x, pj.y};
        z64 v[3] = {z64(0, 0), z64(0, 0), z64(0, 0)};
        for (int a = 0; a < 2; ++a)
            for (int b = 0; b < 2; ++b) {
                const z64 *e = L + ((int64_t)ti[a] * nT + tj[b]) * NCOMP + 3 * ai[a] + aj[b];
                for (int op = 0; op < 3; ++op) v[op] += e[op * 9];
            }
        z64 *Z = Zmm + zoff[c];
        Z[i * n2 + j] = v[0];               // Ks
        Z[i * n2 + N + j] = v[1];           // Ta
        Z[(N + i) * n2 + j] = v[2];         // Tb
        Z[(N + i) * n2 + N + j] = v[0];     // Ks
    }
}

}  // namespace

void assemble_cell_diag(Mesh &m, z64 *Zmm, const std::vector<int64_t> &zoff, cudaStream_t st) {
    const HostMesh &h = m.h;
    const int nc = h.ncell;
    FusedTables &ft = fused_tables(m, st);
    // FP64 near-pair blocks, compact
    DevBuf<z64> nearv;
    nearv.alloc((size_t)std::max<int64_t>(1, m.n_near) * NCOMP);
    near_blocks_compact_t<double>({&m}, {nearv.p}, st);
    std::vector<int64_t> poff(nc + 1, 0);
    for (int c = 0; c < nc; ++c) {
        const int64_t nT = ft.tl_off[c + 1] - ft.tl_off[c];
        poff[c + 1] = poff[c] + nT * nT;
    }
    DevBuf<int64_t> dpoff, dzoff;
    DevBuf<int32_t> dcoff, dloc;
    dpoff.alloc(nc + 1);
    dzoff.alloc(nc);
    dcoff.alloc(nc + 1);
    dloc.alloc(2 * h.ne);
    CBFM_CUDA(cudaMemcpyAsync(dpoff.p, poff.data(), 8 * (nc + 1), cudaMemcpyHostToDevice, st));
    CBFM_CUDA(cudaMemcpyAsync(dzoff.p, zoff.data(), 8 * nc, cudaMemcpyHostToDevice, st));
    CBFM_CUDA(cudaMemcpyAsync(dcoff.p, h.cell_off.data(), 4 * (nc + 1), cudaMemcpyHostToDevice, st));
    CBFM_CUDA(cudaMemcpyAsync(dloc.p, h.edge_loc.data(), 8 * h.ne, cudaMemcpyHostToDevice, st));
    DevBuf<z64> Lb;
    Lb.alloc((size_t)std::max<int64_t>(1, poff[nc]) * NCOMP);
    DevBuf<int> err;
    err.alloc(1);
    CBFM_CUDA(cudaMemsetAsync(err.p, 0, sizeof(int), st));
    const MediaT<double> md = media_t<double>(media_full(m.k1, m.k2, m.eta1, m.eta2));
    {
        const unsigned grid = (unsigned)std::max<int64_t>(1, std::min<int64_t>((poff[nc] + 127) / 128, 8 * (int64_t)sm_count()));
        ProfScope ps_("k_diag_local", st);
        k_diag_local<<<grid, 128, 0, st>>>(nc, dpoff.p, ft.dtl_off.p, ft.tl.p, m.tri64.p, m.tri_vid.p, ft.near_row.p,
                                           ft.near_ent.p, nearv.p, md, m.alpha, Lb.p, err.p);
        launched("k_diag_local");
        prof_add_work("k_diag_local", (double)poff[nc] * 49.0 * FAR_FLOP_PER_POINT_PAIR, 0.0);
    }
    {
        int nmax = 0;
        for (int c = 0; c < nc; ++c) nmax = std::max(nmax, h.cell_off[c + 1] - h.cell_off[c]);
        const unsigned gx = (unsigned)std::max<int64_t>(1, std::min<int64_t>(((int64_t)nmax * nmax + 255) / 256, 64));
        ProfScope ps_("k_diag_gather", st);
        k_diag_gather<<<dim3(gx, nc), 256, 0, st>>>(nc, dcoff.p, ft.dtl_off.p, dpoff.p, dzoff.p, ft.rwg_pos.p, dloc.p,
                                                   Lb.p, Zmm);
        launched("k_diag_gather");
    }
    int herr = 0;
    CBFM_CUDA(cudaMemcpyAsync(&herr, err.p, sizeof(int), cudaMemcpyDeviceToHost, st));
    CBFM_CUDA(cudaStreamSynchronize(st));
    if (herr) throw Fail{CBFM_ECUDA, "cell-diagonal assembly: a near pair is missing from the near list"};
}

}  // namespace cbfm
