// chol_blk.cuh -- blocked Cholesky factorisation and triangular inverse of
// small Hermitian positive definite matrices (the Gram matrices of the block
// GMRES orthogonalisation), FP64, on one thread-block cluster.
#pragma once

#include <cooperative_groups.h>

#include "cluster.cuh"
#include "common.cuh"

namespace cbfm {
namespace chol {

namespace cg = cooperative_groups;
constexpr int PCHOL_MAX = 128;   // largest block width (right-hand sides per block)

// Phase hook for timing experiments; empty in the library.
#ifndef CHOL_MARK
#define CHOL_MARK(phase)
#endif

// ------------------------------------------------ blocked Cholesky, no pivoting
// Cholesky of the Hermitian m x m matrix M (row-major, m <= PCHOL_MAX) in
// panels of CH_B columns, with the rows whose diagonal is exactly zero (rows
// the caller dropped) moved to the end in order: perm lists the r0 others
// first, and M[perm[a]][perm[b]] = sum_i conj(R[i][a]) R[i][b] for a, b < r0,
// R upper triangular (r0 x r0 in an m x m row-major array, zero elsewhere).
// It succeeds when every pivot exceeds tol * max(initial diagonal); at the
// first one that does not, *status = 1 and *rank = its position (the caller
// then runs the pivoted factorisation or reports the lost rank).
//
// One cluster of CC CTAs (one per SM); CTA c owns the columns j = c + CC l
// (cyclic, so the shrinking trailing matrix stays balanced), rows i <= j, in
// shared memory.  Per panel K = [kb, kb + b):
//   1. every CTA gathers the diagonal block M_KK from the owners of its
//      columns and factors the augmented block [M_KK | I] by row operations,
//      which turn it into [R_KK | R_KK^{-H}] (identical inputs, identical
//      results in every CTA: no broadcast);
//   2. each CTA forms its columns of the panel rows, R_K,j = R_KK^{-H} M_K,j,
//      and stores them into the panel-row buffer of every CTA of the cluster;
//   3. after one cluster synchronisation each CTA updates its own columns,
//      M_ij -= sum_{l in K} conj(R_li) R_lj (i <= j), before the next panel's
//      synchronisation.
// Two cluster synchronisations per panel instead of one per pivot; the FP64
// work of the trailing updates is spread over the CC SMs.  The inverse of
// each R_KK goes to Dinv for the inverse kernel below.
//
// FP64 instructions dominate: each warp instruction holds its SM
// sub-partition's FP64 pipe for ~64 clocks whatever the number of active
// lanes.  So the elimination of a diagonal block packs the live entries of
// each step densely into six warps of sub-partitions 0-2 (warps 0-2, 4-6),
// and the pivot chain (next pivot, its reciprocal square root) runs on warp 3
// while the entries are updated: one CTA barrier per step, the next pivot
// ready at its end.
constexpr int CH_B = 16;
constexpr int CH_THREADS = 256;
constexpr int CH_NPAN = PCHOL_MAX / CH_B;
constexpr int CH_NLEFT = CH_B * (CH_B - 1) / 2;   // upper entries of rows 1 .. CH_B-1

template <int CC>
__host__ __device__ constexpr int ch_ncl() { return (PCHOL_MAX + CC - 1) / CC; }
template <int CC>
constexpr size_t chol_cl_smem(int m) { return ((size_t)ch_ncl<CC>() * m + (size_t)CH_B * m) * sizeof(z64); }

// u -= conj(a) c (four FMAs)
__device__ __forceinline__ void ch_sub_conj(z64 &u, z64 a, z64 c) {
    u.re = fma(-a.re, c.re, u.re);
    u.re = fma(-a.im, c.im, u.re);
    u.im = fma(-a.re, c.im, u.im);
    u.im = fma(a.im, c.re, u.im);
}

template <int CC>
__global__ void __launch_bounds__(CH_THREADS)
    k_chol_cl(int m, const z64 *__restrict__ M, double tol, int *__restrict__ perm, z64 *__restrict__ R,
              z64 *__restrict__ Dinv, int *__restrict__ rank_out, int *__restrict__ status, int *__restrict__ err) {
    cg::cluster_group cl = cg::this_cluster();
    const int me = (int)cl.block_rank();
    constexpr int NCL = ch_ncl<CC>();
    extern __shared__ __align__(16) unsigned char ch_raw[];
    z64 *Mc = reinterpret_cast<z64 *>(ch_raw);   // [NCL][m]: own column j = me + CC lc, rows i <= j
    z64 *Rp = Mc + (size_t)NCL * m;              // [CH_B][m]: the panel rows of R over the trailing columns
    __shared__ z64 A[CH_B][2 * CH_B + 1];        // the augmented diagonal block [M_KK | I] under elimination
    __shared__ z64 Rk[CH_B][CH_B + 1];           // R_KK (upper triangular)
    __shared__ z64 Lk[CH_B][CH_B + 1];           // R_KK^{-H} (lower triangular)
    __shared__ double s_rs[2], s_inv[2], s_n2[2];   // 1/sqrt(pivot), 1/pivot, |A[k][k+1]|^2 by step parity
    __shared__ unsigned char s_tr[CH_NLEFT], s_tc[CH_NLEFT];   // left entries, rows descending, pivot last
    __shared__ int s_perm[PCHOL_MAX];
    __shared__ uint64_t cbar[2];
    __shared__ int s_abort, s_fail, s_r0;
    __shared__ double s_thr;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;

    // rows with a zero diagonal last (stable), and the pivot threshold
    if (warp == 0) {
        double mx = 0.0;
        int nz_total = 0;
        for (int pass = 0; pass < 2; ++pass) {
            int base = pass == 0 ? 0 : nz_total;
            for (int a0 = 0; a0 < m; a0 += 32) {
                const int a = a0 + lane;
                const double d = a < m ? M[(int64_t)a * m + a].re : 0.0;
                if (pass == 0 && a < m) mx = fmax(mx, d);
                const bool take = a < m && ((d != 0.0) == (pass == 0));
                const unsigned bal = __ballot_sync(0xffffffffu, take);
                if (take) s_perm[base + __popc(bal & ((1u << lane) - 1u))] = a;
                base += __popc(bal);
            }
            if (pass == 0) nz_total = base;
        }
        for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        if (lane == 0) {
            s_r0 = nz_total;
            s_thr = tol * mx;
            s_abort = 0;
            s_fail = -1;
            cl_bar_init(cbar, CC);
        }
    }
    // left-entry table: rows CH_B-1 down to 1, in each row the columns after the
    // diagonal and then the diagonal, so that the live entries of step k are a prefix
    if (tid < CH_NLEFT) {
        int r = CH_B - 1, start = 0;
        while (tid >= start + (CH_B - r)) {
            start += CH_B - r;
            --r;
        }
        const int o = tid - start;
        s_tr[tid] = (unsigned char)r;
        s_tc[tid] = (unsigned char)(o < CH_B - 1 - r ? r + 1 + o : r);
    }
    for (int idx = tid; idx < CH_B * (CH_B + 1); idx += CH_THREADS) {
        (&Rk[0][0])[idx] = z64(0.0, 0.0);
        (&Lk[0][0])[idx] = z64(0.0, 0.0);
    }
    __syncthreads();
    const int r0 = s_r0;
    const double thr = s_thr;
    const int ncl = me < r0 ? (r0 - 1 - me) / CC + 1 : 0;      // own columns below r0
    const int ncl_all = me < m ? (m - 1 - me) / CC + 1 : 0;    // own columns of the output
    for (int idx = tid; idx < ncl_all * m; idx += CH_THREADS) {
        const int lc = idx / m, i = idx - lc * m, j = me + CC * lc;
        R[(int64_t)i * m + j] = z64(0.0, 0.0);
        if (lc < ncl) Mc[(size_t)lc * m + i] = i <= j ? M[(int64_t)s_perm[i] * m + s_perm[j]] : z64(0.0, 0.0);
    }
    if (me == 0)
        for (int k = tid; k < m; k += CH_THREADS) perm[k] = s_perm[k];
    __syncthreads();
    cl.sync();   // barriers initialised and own columns loaded in every CTA

    // slot of this thread in the elimination (warps 0-2 and 4-6), -1 for warps 3 and 7
    const int slot = (warp & 3) == 3 ? -1 : ((warp < 4 ? warp : warp - 1) * 32 + lane);
    int ks = 0, fail = -1;
    bool alive = true;
    for (int kb = 0; kb < r0; kb += CH_B) {
        const int b = min(CH_B, r0 - kb), np = kb / CH_B;
        if (kb > 0 && !cl_sync(cbar, ks++, CC, &s_abort, err)) {
            alive = false;
            break;
        }
        CHOL_MARK(0);
        // 1. [M_KK | I], padded with the identity beyond b
        for (int idx = tid; idx < CH_B * 2 * CH_B; idx += CH_THREADS) {
            const int r = idx / (2 * CH_B), c = idx % (2 * CH_B);
            z64 v(0.0, 0.0);
            if (c < CH_B) {
                if (r <= c) {
                    if (c < b) {
                        const int j = kb + c;
                        const z64 *src = cl.map_shared_rank(Mc, j % CC);
                        v = src[(size_t)(j / CC) * m + kb + r];
                    } else if (r == c) {
                        v = z64(1.0, 0.0);
                    }
                }
            } else if (c - CH_B == r) {
                v = z64(1.0, 0.0);
            }
            A[r][c] = v;
        }
        __syncthreads();
        CHOL_MARK(1);
        if (tid == 0) {
            const double d = A[0][0].re;
            if (!(d > thr)) s_fail = kb;
            const double rs = d > 0.0 ? rsqrt(d) : 0.0;
            s_rs[0] = rs;
            s_inv[0] = rs * rs;
            s_n2[0] = norm2(A[0][1]);
        }
        __syncthreads();
        // step k: row k scaled by 1/sqrt(pivot) becomes row k of [R_KK | R_KK^{-H}];
        // rows r > k lose conj(A[k][r]) / pivot times row k; the chain thread forms
        // pivot k+1 from |A[k][k+1]|^2 (left by step k-1) and inverts it.
        for (int k = 0; k < CH_B && s_fail < 0; ++k) {
            const double rs = s_rs[k & 1], inv = s_inv[k & 1];
            const int nleft = max(0, (CH_B - 1 - k) * (CH_B - k) / 2 - 1);   // rows k+1.., without pivot k+1
            const int nright = (CH_B - 1 - k) * (k + 1);
            if (slot >= 0) {
                int e = slot;
                if (e < nleft) {
                    const int r = s_tr[e], c = s_tc[e];
                    const z64 f = conj(A[k][r]) * inv;
                    z64 v = A[r][c];
                    cfma(v, -f, A[k][c]);
                    A[r][c] = v;
                    if (r == k + 1 && c == k + 2) s_n2[(k + 1) & 1] = norm2(v);
                } else if ((e -= nleft) < nright) {
                    const int r = k + 1 + e / (k + 1), cc = e % (k + 1);
                    const z64 f = conj(A[k][r]) * inv;
                    z64 v = A[r][CH_B + cc];
                    cfma(v, -f, A[k][CH_B + cc]);
                    A[r][CH_B + cc] = v;
                } else if ((e -= nright) < CH_B + 1) {
                    if (e < CH_B - k) {
                        const int c = k + e;
                        Rk[k][c] = c == k ? z64(A[k][k].re * rs, 0.0) : A[k][c] * rs;
                    } else {
                        const int cc = e - (CH_B - k);
                        Lk[k][cc] = A[k][CH_B + cc] * rs;
                    }
                }
            } else if (warp == 3 && lane == 0 && k + 1 < CH_B) {
                const double piv = fma(-s_n2[k & 1], inv, A[k + 1][k + 1].re);
                if (k + 1 < b && !(piv > thr)) s_fail = kb + k + 1;
                const double rs1 = piv > 0.0 ? rsqrt(piv) : 0.0;
                s_rs[(k + 1) & 1] = rs1;
                s_inv[(k + 1) & 1] = rs1 * rs1;
                A[k + 1][k + 1] = z64(piv, 0.0);
            }
            __syncthreads();
        }
        CHOL_MARK(2);
        if (s_fail >= 0) {   // the same decision in every CTA: identical blocks
            fail = s_fail;
            break;
        }
        // R_KK^{-1} = (R_KK^{-H})^H for the inverse kernel
        if (me == 0)
            for (int idx = tid; idx < CH_B * CH_B; idx += CH_THREADS) {
                const int r = idx / CH_B, s = idx % CH_B;
                Dinv[((size_t)np * CH_B + r) * CH_B + s] = conj(Lk[s][r]);
            }
        // 2. own columns: rows K of R (the diagonal block's columns from Rk, the others
        // R_KK^{-H} M_K,j), to R and to the panel-row buffer of every CTA
        const bool trailing = kb + b < r0;
        for (int idx = tid; idx < ncl * CH_B; idx += CH_THREADS) {
            const int lc = idx / CH_B, r = idx % CH_B, j = me + CC * lc;
            if (j < kb || r >= b) continue;
            z64 v(0.0, 0.0);
            if (j < kb + b) {
                v = Rk[r][j - kb];
            } else {
                const z64 *mj = Mc + (size_t)lc * m + kb;
                for (int s = 0; s <= r; ++s) cfma(v, Lk[r][s], mj[s]);
            }
            R[(int64_t)(kb + r) * m + j] = v;
            if (trailing && j >= kb + b)
#pragma unroll 4
                for (int q = 0; q < CC; ++q) *cl.map_shared_rank(Rp + (size_t)r * m + j, q) = v;
        }
        CHOL_MARK(3);
        if (!trailing) break;   // no trailing matrix
        if (!cl_sync(cbar, ks++, CC, &s_abort, err)) {
            alive = false;
            break;
        }
        CHOL_MARK(4);
        CHOL_MARK(5);
        // 3. own trailing columns j >= kb + b, rows kb + b <= i <= j, one entry per thread
        {
            const int t0 = kb + b;
            const int lc0 = me >= t0 ? 0 : (t0 - me + CC - 1) / CC;   // first own column >= t0
            int total = 0;
            for (int lc = lc0; lc < ncl; ++lc) total += me + CC * lc - t0 + 1;
            for (int e = tid; e < total; e += CH_THREADS) {
                int lc = lc0, rem = e;
                while (rem >= me + CC * lc - t0 + 1) {
                    rem -= me + CC * lc - t0 + 1;
                    ++lc;
                }
                const int j = me + CC * lc, i = t0 + rem;
                z64 v = Mc[(size_t)lc * m + i];
#pragma unroll 4
                for (int l = 0; l < b; ++l) ch_sub_conj(v, Rp[(size_t)l * m + i], Rp[(size_t)l * m + j]);
                Mc[(size_t)lc * m + i] = v;
            }
        }
        CHOL_MARK(6);
        // the next panel's synchronisation orders these updates before any remote read
    }
    __syncthreads();
    cl.sync();   // every CTA done with the others' shared memory
    if (me == 0 && tid == 0) {
        *status = (fail >= 0 || !alive) ? 1 : 0;
        *rank_out = fail >= 0 ? fail : r0;
    }
}

// Rinv = R^{-1} for the blocked factor (r = *rank; R row-major, ld m; Dinv
// the inverses of its diagonal CH_B x CH_B blocks), zero elsewhere in the
// m x m output.  One CTA of 128 threads per column j; the column's part in
// its own block is read from Dinv, then block by block upwards
//   x_I = -R_II^{-1} sum_{l > block I} R[I][l] x_l,
// each sum split over 8 threads per row.  Nothing is written when *status
// reports a failed factorisation.
__global__ void __launch_bounds__(128) k_trinv_blk(int m, const z64 *__restrict__ R, const z64 *__restrict__ Dinv,
                                                   const int *__restrict__ rank, const int *__restrict__ status,
                                                   z64 *__restrict__ Rinv) {
    __shared__ z64 x[PCHOL_MAX];
    __shared__ z64 t[CH_B];
    if (*status != 0) return;
    const int j = blockIdx.x, tid = threadIdx.x, r0 = *rank;
    if (j >= r0) {
        for (int i = tid; i < m; i += blockDim.x) Rinv[(int64_t)i * m + j] = z64(0.0, 0.0);
        return;
    }
    const int J = j / CH_B, jb = J * CH_B;
    for (int i = tid; i < m; i += blockDim.x) x[i] = z64(0.0, 0.0);
    __syncthreads();
    if (tid < CH_B && jb + tid <= j) x[jb + tid] = Dinv[((size_t)J * CH_B + tid) * CH_B + (j - jb)];
    __syncthreads();
    const int r = tid >> 3, q = tid & 7;   // 16 rows x 8 threads
    for (int I = J - 1; I >= 0; --I) {
        const int ib = I * CH_B;
        z64 s(0.0, 0.0);
        for (int l = ib + CH_B + q; l <= j; l += 8) cfma(s, R[(int64_t)(ib + r) * m + l], x[l]);
        for (int o = 4; o > 0; o >>= 1) {
            s.re += __shfl_xor_sync(0xffffffffu, s.re, o);
            s.im += __shfl_xor_sync(0xffffffffu, s.im, o);
        }
        if (q == 0) t[r] = s;
        __syncthreads();
        z64 v(0.0, 0.0);
        for (int c = q; c < CH_B; c += 8) cfma(v, Dinv[((size_t)I * CH_B + r) * CH_B + c], t[c]);
        for (int o = 4; o > 0; o >>= 1) {
            v.re += __shfl_xor_sync(0xffffffffu, v.re, o);
            v.im += __shfl_xor_sync(0xffffffffu, v.im, o);
        }
        if (q == 0) x[ib + r] = -v;
        __syncthreads();
    }
    for (int i = tid; i < m; i += blockDim.x) Rinv[(int64_t)i * m + j] = x[i];
}


}  // namespace chol
}  // namespace cbfm
