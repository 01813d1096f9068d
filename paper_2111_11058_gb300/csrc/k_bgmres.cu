// k_bgmres.cu -- block GMRES: the right-preconditioned GMRES of paper Eqs.
// (CBFM_outer)/(CBFM_inner) run on all right-hand sides together, which share
// the operator B = A (G^CBF)^{-1}.  One block Krylov space
//   span{R0, B R0, B^2 R0, ...}   (R0 = the block of residuals)
// serves every right-hand side; each one still stops on its own criterion
// ||b_c - B y_c|| / ||b_c|| <= tol and the iteration ends when all have.
// With p right-hand sides the space grows by up to p directions per block
// iteration, so the orthogonalisation becomes matrix-matrix products.
//
// FP64 throughout except the operator product (complex64 B and FP32
// accumulation in CBFM_MIXED):
//   * block Arnoldi with block classical Gram-Schmidt, repeated where one
//     pass is not enough (BCGS2 with the second pass skipped when every
//     vector kept GS_KEEP of its norm, or applied only when its coefficients
//     exceed ORTH_TOL of the block);
//   * the new block is orthonormalised by Cholesky QR, the Cholesky pivoted
//     so that numerically dependent directions (saturation of the space,
//     dependent right-hand sides) are dropped, and repeated once (CholQR2)
//     unless the first pass already gives ||Q^H Q - I||_F <= ORTH_TOL;
//   * the block Hessenberg least-squares problem min ||E1 S - Hbar Z|| is
//     solved through a QR of Hbar kept up to date block column by block
//     column (block Gram-Schmidt and Cholesky QR, each repeated under the
//     same tests).
#include <cooperative_groups.h>

#include <algorithm>
#include <climits>
#include <cmath>
#include <atomic>
#include <vector>

#include "chol_blk.cuh"
#include "cluster.cuh"
#include "internal.cuh"

namespace cbfm {

namespace {

using namespace chol;
constexpr int PCHOL_THREADS = 256;
// ------------------------------------------------ pivoted Cholesky factor
// Pivoted Cholesky of the Hermitian m x m matrix M (row-major): with the order
// perm, M[perm[a]][perm[b]] = sum_i conj(R[i][a]) R[i][b], R upper trapezoidal
// (rank x m, row-major, ld m, rows >= rank zero).  pivot == 0 keeps the
// order.  A remaining diagonal below tol * max(initial diagonal) ends the
// factorisation (rank).
//
// It runs on a cluster of PC_CL CTAs (one per SM).  CTA c owns the rows of
// original index a = c + PC_CL l of the Schur complement U, stored in full in
// its shared memory (the diagonals also in a compact array).  For step i every
// CTA has proposed a candidate (its largest remaining diagonal, lowest
// position on ties; without pivoting only the owner of position i proposes):
// the row, unscaled, in its own shared memory, and its diagonal,
// 1 / sqrt(diagonal), position and index in the shared memory of every CTA.
// After the synchronisation of step i all CTAs pick the same winner q and read
// its row from the shared memory of its owner, CTA 0 writes row i of R (by
// original index; permuted to positions after the loop), and each CTA applies
//   U(a, b) -= conj(U(q, a)) U(q, b) / U(q, q)
// to its own rows.  The chain from one synchronisation to the next is kept
// short: a CTA updates the diagonals of its rows, picks its candidate for
// step i + 1, updates that row and stores it, sends the scalars, arrives, and
// only then updates the rest of its rows, overlapping the other CTAs' chains.
// A CTA can therefore write its proposal of step i + 2 while another still
// reads the one of step i: proposals rotate through three buffers.  The
// synchronisation of step k is the mbarrier pair of cluster.cuh, arrived on
// remotely by every CTA; its wait gives up after one second (error flag,
// loop ends).  Hardware cluster barriers are used only where every CTA
// arrives unconditionally: after set-up and before exit.
namespace cg = cooperative_groups;
constexpr int PC_CL = 8;
constexpr int PC_ROWS = (PCHOL_MAX + PC_CL - 1) / PC_CL;
constexpr int PC_NBUF = 3;

// dynamic shared memory: own rows [PC_ROWS][m] and own candidate rows [PC_NBUF][m]
constexpr size_t pchol_cl_smem(int m) { return (size_t)(PC_ROWS + PC_NBUF) * m * sizeof(z64); }

// u -= c r
__device__ __forceinline__ void pc_axpy(z64 &u, z64 c, z64 r) {
    u.re = fma(-c.re, r.re, u.re);
    u.re = fma(c.im, r.im, u.re);
    u.im = fma(-c.re, r.im, u.im);
    u.im = fma(-c.im, r.re, u.im);
}

__global__ void __cluster_dims__(PC_CL, 1, 1) __launch_bounds__(PCHOL_THREADS)
    k_pchol_cl(int m, const z64 *__restrict__ M, int *__restrict__ perm, z64 *__restrict__ R,
               int *__restrict__ rank_out, double tol, int pivot, int *__restrict__ err) {
    cg::cluster_group cl = cg::this_cluster();
    const int me = (int)cl.block_rank();
    extern __shared__ __align__(16) unsigned char pc_raw[];
    z64 *Uloc = reinterpret_cast<z64 *>(pc_raw);   // [PC_ROWS][m]
    z64 *crow = Uloc + (size_t)PC_ROWS * m;        // [PC_NBUF][m]: this CTA's candidate rows, by original index
    __shared__ uint64_t cbar[2];
    __shared__ double cval[PC_NBUF][PC_CL], crd[PC_NBUF][PC_CL];   // proposal: diagonal, 1 / sqrt(diagonal)
    __shared__ int cpos[PC_NBUF][PC_CL], cidx[PC_NBUF][PC_CL];     // proposal: position, original index
    __shared__ z64 s_coef[PC_ROWS];                                 // conj(U(q, a)) / U(q, q) per own row
    __shared__ double s_dg[PC_ROWS];                                // diagonal U(a, a) per own row
    __shared__ z64 rowq[PCHOL_MAX];                                 // the winning row of the step
    __shared__ int s_alive[PC_ROWS];                                // own row not yet eliminated
    __shared__ int piv[PCHOL_MAX], posof[PCHOL_MAX];
    __shared__ int s_abort, s_stop, s_cand, s_cpos;
    __shared__ double s_cd, s_crd;
    __shared__ double s_thr;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nth = blockDim.x;
    const int nloc = me < m ? (m - me + PC_CL - 1) / PC_CL : 0;
    for (int idx = threadIdx.x; idx < nloc * m; idx += nth) {
        const int ls = idx / m, b = idx - ls * m, a = me + PC_CL * ls;
        Uloc[idx] = M[(int64_t)a * m + b];
        R[(int64_t)a * m + b] = z64(0, 0);
    }
    for (int k = threadIdx.x; k < m; k += nth) {
        piv[k] = k;
        posof[k] = k;
    }
    if (threadIdx.x < nloc) {
        const int a = me + PC_CL * threadIdx.x;
        s_alive[threadIdx.x] = 1;
        s_dg[threadIdx.x] = M[(int64_t)a * m + a].re;
    }
    if (warp == 0) {
        double mx = 0.0;
        for (int k = lane; k < m; k += 32) mx = fmax(mx, M[(int64_t)k * m + k].re);
        for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        if (lane == 0) {
            s_thr = tol * mx;
            s_abort = 0;
            s_stop = m;
            cl_bar_init(cbar, PC_CL);
        }
    }
    __syncthreads();
    cl.sync();   // every CTA's barriers are initialised before the first remote arrive
    const double thr = s_thr;

    // warp 0: this CTA's candidate for step i (diagonals up to date)
    auto pick = [&](int i) {
        if (!pivot) {   // no row exchanges: position i is row i, owned by CTA i % PC_CL
            if (threadIdx.x == 0) {
                const int ls = (i % PC_CL == me) ? i / PC_CL : -1;
                const double d = ls >= 0 ? s_dg[ls] : -1.0;
                s_cand = ls;
                s_cpos = ls >= 0 ? i : INT_MAX;
                s_cd = d;
                s_crd = d > 0.0 ? 1.0 / sqrt(d) : 0.0;
            }
            return;
        }
        if (warp != 0) return;
        long long best = LLONG_MIN;
        int bp = INT_MAX, bls = -1;
        for (int ls = lane; ls < nloc; ls += 32) {
            const int a = me + PC_CL * ls, pa = posof[a];
            if (pa < i || (!pivot && pa != i)) continue;
            const long long v = __double_as_longlong(s_dg[ls]);   // orders positive doubles
            if (bls < 0 || v > best || (v == best && pa < bp)) {
                best = v;
                bp = pa;
                bls = ls;
            }
        }
        for (int o = 16; o > 0; o >>= 1) {
            const long long ov = __shfl_xor_sync(0xffffffffu, best, o);
            const int op = __shfl_xor_sync(0xffffffffu, bp, o), ol = __shfl_xor_sync(0xffffffffu, bls, o);
            if (ol >= 0 && (bls < 0 || ov > best || (ov == best && op < bp))) {
                best = ov;
                bp = op;
                bls = ol;
            }
        }
        if (lane == 0) {
            const double d = bls >= 0 ? __longlong_as_double(best) : -1.0;
            s_cand = bls;
            s_cpos = bls >= 0 ? bp : INT_MAX;
            s_cd = d;
            s_crd = d > 0.0 ? 1.0 / sqrt(d) : 0.0;
        }
    };
    // the candidate's scalars to buffer i % PC_NBUF of every CTA (one CTA per thread)
    auto send_scalars = [&](int i) {
        if (threadIdx.x < PC_CL) {
            const int r = threadIdx.x, buf = i % PC_NBUF, cls = s_cand;
            *cl.map_shared_rank(&cval[buf][me], r) = s_cd;
            *cl.map_shared_rank(&crd[buf][me], r) = s_crd;
            *cl.map_shared_rank(&cpos[buf][me], r) = s_cpos;
            *cl.map_shared_rank(&cidx[buf][me], r) = cls >= 0 ? me + PC_CL * cls : -1;
        }
    };

    // step 0: candidates from the initial diagonals
    pick(0);
    __syncthreads();
    if (s_cand >= 0)
        for (int b = threadIdx.x; b < m; b += nth) crow[b] = Uloc[s_cand * m + b];
    send_scalars(0);
    __syncthreads();
    cl_arrive(cbar, 0, PC_CL);

    for (int i = 0; i < m; ++i) {
        if (!cl_wait(cbar, i, &s_abort, err)) break;
        const int buf = i % PC_NBUF;
        // ---- the same decision in every CTA
        int w = -1, bpos = INT_MAX;
        long long bv = 0;
        for (int r = 0; r < PC_CL; ++r) {
            const int pr = cpos[buf][r];
            if (pr == INT_MAX) continue;
            const long long vb = __double_as_longlong(cval[buf][r]);
            if (w < 0 || vb > bv || (vb == bv && pr < bpos)) {
                w = r;
                bv = vb;
                bpos = pr;
            }
        }
        const double dq = w >= 0 ? cval[buf][w] : -1.0;
        if (w < 0 || !(dq > thr) || dq <= 0.0) {
            if (threadIdx.x == 0) s_stop = i;
            break;
        }
        const int q = cidx[buf][w];
        {   // row q of the Schur complement, unscaled, from the shared memory of its owner
            const z64 *src = cl.map_shared_rank(crow + (size_t)buf * m, w);
            for (int b = threadIdx.x; b < m; b += nth) rowq[b] = src[b];
        }
        __syncthreads();
        const z64 *Ri = rowq;
        const double rdq = crd[buf][w];                         // 1 / sqrt(U(q, q))
        if (threadIdx.x == 0 && bpos != i) {
            const int t = piv[i];
            piv[i] = piv[bpos];
            piv[bpos] = t;
            posof[piv[i]] = i;
            posof[piv[bpos]] = bpos;
        }
        if (threadIdx.x < nloc) {   // own row: coefficient, and its diagonal at once
            const int ls = threadIdx.x, a = me + PC_CL * ls;
            if (a == q) s_alive[ls] = 0;
            const z64 c = conj(Ri[a]) * (rdq * rdq);
            s_coef[ls] = c;
            if (s_alive[ls]) {   // real part of U(a, a) -= c U(q, a) (the diagonal is real)
                double d = s_dg[ls];
                d = fma(-c.re, Ri[a].re, d);
                d = fma(c.im, Ri[a].im, d);
                s_dg[ls] = d;
            }
        }
        __syncthreads();
        // row i of R = row q / sqrt(U(q, q)), by original index for now (permuted to positions after the loop)
        if (me == 0) {
            for (int b = threadIdx.x; b < m; b += nth)
                R[(int64_t)i * m + b] = posof[b] < i ? z64(0, 0) : (b == q ? z64(dq * rdq, 0) : Ri[b] * rdq);
        }
        if (i + 1 >= m) break;
        // ---- candidate for step i + 1: updated while it is sent, then the arrival
        pick(i + 1);
        __syncthreads();
        const int cls = s_cand;
        if (cls >= 0) {
            const int a = me + PC_CL * cls;
            const z64 c = s_coef[cls];
            z64 *dst = crow + (size_t)((i + 1) % PC_NBUF) * m;
            for (int b = threadIdx.x; b < m; b += nth) {
                z64 v = Uloc[cls * m + b];
                if (b != a && posof[b] > i) {
                    pc_axpy(v, c, Ri[b]);
                    Uloc[cls * m + b] = v;
                }
                dst[b] = v;
            }
        }
        send_scalars(i + 1);
        __syncthreads();
        cl_arrive(cbar, i + 1, PC_CL);
        // ---- the rest of this CTA's rows over the remaining positions (diagonals done)
        const int rem = m - i - 1;
        for (int idx = threadIdx.x; idx < nloc * rem; idx += nth) {
            const int ls = idx / rem, pos = i + 1 + (idx - ls * rem);
            if (ls == cls || !s_alive[ls]) continue;
            const int b = piv[pos], a = me + PC_CL * ls;
            if (b == a) continue;
            pc_axpy(Uloc[ls * m + b], s_coef[ls], Ri[b]);
        }
        __syncthreads();
    }
    __syncthreads();
    cl.sync();   // rows of R written by CTA 0 are visible to every CTA; no proposal is in flight any more
    // R[i][pos] = row i by original index at piv[pos] (rows distributed over the CTAs)
    const int rk = s_stop;
    for (int i = me; i < rk; i += PC_CL) {
        for (int b = threadIdx.x; b < m; b += nth) crow[b] = R[(int64_t)i * m + b];
        __syncthreads();
        for (int pos = threadIdx.x; pos < m; pos += nth) R[(int64_t)i * m + pos] = crow[piv[pos]];
        __syncthreads();
    }
    if (me == 0) {
        for (int k = threadIdx.x; k < m; k += nth) perm[k] = piv[k];
        if (threadIdx.x == 0) *rank_out = rk;
    }
    cl.sync();   // no CTA leaves while another may still use the cluster's shared memory
}

// Rinv = R11^{-1} for the leading r x r block of the upper-triangular Cholesky
// factor R (r = *rank; row-major, ld m, real positive diagonal), zero
// elsewhere in the m x m output.  One CTA of PCHOL_MAX threads per column j,
// thread t owning row t; column-oriented back substitution from b = e_j:
// for k = j .. 0, x_k = b_k / R[k][k] (the owner publishes it), then
// b_t -= R[t][k] x_k for the rows t < k.  The triangle R[0..j][0..j] is staged
// in shared memory first (column k packed at k(k+1)/2), so a step is one
// barrier, one shared-memory read and one complex multiply-add per row; the
// rows of a step are spread over the four warps (four FP64 pipes).
constexpr size_t trinv_smem(int m) { return (size_t)m * (m + 1) / 2 * sizeof(z64); }

__global__ void __launch_bounds__(PCHOL_MAX) k_trinv(int m, const z64 *__restrict__ R, const int *__restrict__ rank,
                                                     z64 *__restrict__ Rinv) {
    extern __shared__ __align__(16) unsigned char ti_raw[];
    z64 *Rs = reinterpret_cast<z64 *>(ti_raw);   // packed columns of the upper triangle
    __shared__ double s_inv[PCHOL_MAX];
    __shared__ z64 s_x[2];
    const int j = blockIdx.x, t = threadIdx.x;
    const int r = *rank;
    if (j < r) {
        // thread k loads column k: R[i][k], i <= k (consecutive threads, consecutive addresses)
        if (t <= j) {
            z64 *col = Rs + (size_t)t * (t + 1) / 2;
#pragma unroll 8
            for (int i = 0; i <= t; ++i) col[i] = R[(int64_t)i * m + t];
            s_inv[t] = 1.0 / R[(int64_t)t * m + t].re;
        }
        __syncthreads();
        z64 b(t == j ? 1.0 : 0.0, 0.0);
        for (int k = j; k >= 0; --k) {
            if (t == k) {
                b = b * s_inv[k];
                s_x[k & 1] = b;
            }
            __syncthreads();   // x_k published; the slot of step k + 2 is free again
            if (t < k) b -= Rs[(size_t)k * (k + 1) / 2 + t] * s_x[k & 1];
        }
        if (t < m) Rinv[(int64_t)t * m + j] = t <= j ? b : z64(0, 0);
    } else {
        if (t < m) Rinv[(int64_t)t * m + j] = z64(0, 0);
    }
}

// X (r x m): X[i][perm[l]] = Rinv[l][i] (l <= i < r), else 0  -> Q = X W for row vectors W.
// The zeroing is a launch of its own (k_zero2d) before this one; consecutive
// threads read consecutive entries of a row of Rinv.
__global__ void k_make_x(int m, int r, const int *__restrict__ perm, const z64 *__restrict__ Rinv,
                         z64 *__restrict__ X) {
    for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < (int64_t)r * r;
         idx += (int64_t)gridDim.x * blockDim.x) {
        const int l = (int)(idx / r), i = (int)(idx % r);
        if (l <= i) X[(int64_t)i * m + perm[l]] = Rinv[(int64_t)l * m + i];
    }
}

// Rfull (r x m, ld m): Rfull[i][perm[l]] = R[i][l]
__global__ void k_unpermute_r(int m, int r, const int *__restrict__ perm, const z64 *__restrict__ R,
                              z64 *__restrict__ Rfull) {
    for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < (int64_t)r * m;
         idx += (int64_t)gridDim.x * blockDim.x) {
        int i = (int)(idx / m), l = (int)(idx % m);
        Rfull[(int64_t)i * m + perm[l]] = R[idx];
    }
}

// dst[i * ldd + j] = src[j * lds + i] for i < rows, j < cols (transposing copy)
__global__ void k_copy_t(int rows, int cols, const z64 *__restrict__ src, int64_t lds, z64 *__restrict__ dst,
                         int64_t ldd) {
    for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < (int64_t)rows * cols;
         idx += (int64_t)gridDim.x * blockDim.x) {
        int i = (int)(idx / cols), j = (int)(idx % cols);
        dst[(int64_t)i * ldd + j] = src[(int64_t)j * lds + i];
    }
}

// dst[i * ldd + j] = src[i * lds + j] (+= when add)
__global__ void k_copy2d(int rows, int cols, const z64 *__restrict__ src, int64_t lds, z64 *__restrict__ dst,
                         int64_t ldd, int add) {
    for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < (int64_t)rows * cols;
         idx += (int64_t)gridDim.x * blockDim.x) {
        int i = (int)(idx / cols), j = (int)(idx % cols);
        if (add) dst[(int64_t)i * ldd + j] += src[(int64_t)i * lds + j];
        else dst[(int64_t)i * ldd + j] = src[(int64_t)i * lds + j];
    }
}

__global__ void k_zero2d(int rows, int cols, z64 *__restrict__ dst, int64_t ldd) {
    for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < (int64_t)rows * cols;
         idx += (int64_t)gridDim.x * blockDim.x) {
        int i = (int)(idx / cols), j = (int)(idx % cols);
        dst[(int64_t)i * ldd + j] = z64(0, 0);
    }
}

// column norms of a rows x cols row-major matrix (one block per column)
__global__ void k_colnorm(int rows, int cols, const z64 *__restrict__ X, int64_t ld, double *__restrict__ out) {
    const int c = blockIdx.x;
    double s = 0;
    for (int i = threadIdx.x; i < rows; i += blockDim.x) s += norm2(X[(int64_t)i * ld + c]);
    __shared__ double sh[32];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0;
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) a += sh[i];
        out[c] = sqrt(a);
    }
}

// row norms of a rows x n matrix (one block per row)
__global__ void k_rownorm(int64_t n, const z64 *__restrict__ X, double *__restrict__ out) {
    const int r = blockIdx.x;
    double s = 0;
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) s += norm2(X[(int64_t)r * n + i]);
    __shared__ double sh[32];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0;
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) a += sh[i];
        out[r] = sqrt(a);
    }
}

// Row scaling for the rank-revealing Cholesky QR: rows with norm <= drop * ref
// are zeroed (treated as exhausted directions), the others scaled to unit norm;
// scale[r] receives the factor to undo (norm, or 0 for dropped rows).
__global__ void k_scale_rows(int64_t n, z64 *__restrict__ X, const double *__restrict__ nrm, double ref, double drop,
                             double *__restrict__ scale) {
    const int r = blockIdx.y;
    const double v = nrm[r];
    const bool keep = v > drop * ref && v > 0.0;
    const double inv = keep ? 1.0 / v : 0.0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        X[(int64_t)r * n + i] = X[(int64_t)r * n + i] * inv;
    if (blockIdx.x == 0 && threadIdx.x == 0) scale[r] = keep ? v : 0.0;
}

// Rfull[i][c] *= scale[c] (r x m, ld m)
__global__ void k_scale_cols(int r, int m, z64 *__restrict__ R, const double *__restrict__ scale) {
    for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < (int64_t)r * m;
         idx += (int64_t)gridDim.x * blockDim.x)
        R[idx] = R[idx] * scale[idx % m];
}

__global__ void k_sub_rows(int64_t count, const z64 *__restrict__ a, const z64 *__restrict__ b, z64 *__restrict__ out) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < count) out[i] = a[i] - b[i];
}

// dst[r] = src[idx[r]] (rows of length n), r < k
__global__ void k_gather_rows(int k, int64_t n, const int *__restrict__ idx, const z64 *__restrict__ src,
                              z64 *__restrict__ dst) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < (int64_t)k * n;
         i += (int64_t)gridDim.x * blockDim.x)
        dst[i] = src[(int64_t)idx[i / n] * n + i % n];
}

// dst[idx[r]] (leading dimension ldd; 0: n) = src[r] (ld n) for r < k, += when ldd != 0
__global__ void k_scatter_rows(int k, int64_t n, const int *__restrict__ idx, const z64 *__restrict__ src,
                               z64 *__restrict__ dst, int64_t ldd) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < (int64_t)k * n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = i / n, c = i % n;
        if (ldd == 0) dst[(int64_t)idx[r] * n + c] = src[r * n + c];
        else dst[(int64_t)idx[r] * ldd + c] += src[r * ldd + c];
    }
}

// rows r of a rows x n matrix with mask[r] != 0 set to zero
__global__ void k_zero_rows_masked(int rows, int64_t n, const int *__restrict__ mask, z64 *__restrict__ X) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < (int64_t)rows * n;
         i += (int64_t)gridDim.x * blockDim.x)
        if (mask[i / n]) X[i] = z64(0.0, 0.0);
}

// Y += X (complex64 into complex128), n elements
__global__ void k_add32to64(int64_t n, const c32 *__restrict__ X, z64 *__restrict__ Y) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        Y[i] += z64(X[i].re, X[i].im);
}

// ||M - I||_F of a Hermitian m x m matrix from its upper triangle (one block;
// fixed summation order)
// Partial sums of ||M - I||_F^2 over the upper triangle (off-diagonal entries
// counted twice): CTA c takes rows a = c, c + GD_CTAS, ... and writes part[c];
// k_gram_dev_sum adds the GD_CTAS partials in a fixed order (same bits on
// every run, so the pass-2 decision does not depend on scheduling).
constexpr int GD_CTAS = 32;
__global__ void __launch_bounds__(256) k_gram_dev(int m, const z64 *__restrict__ M, double *__restrict__ part) {
    __shared__ double wp[8];
    double s = 0.0;
    for (int a = blockIdx.x; a < m; a += gridDim.x)
        for (int b = a + threadIdx.x; b < m; b += blockDim.x) {
            z64 v = M[(int64_t)a * m + b];
            if (a == b) v.re -= 1.0;
            s += (a == b ? 1.0 : 2.0) * (v.re * v.re + v.im * v.im);
        }
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) wp[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < 8; ++w) t += wp[w];
        part[blockIdx.x] = t;
    }
}
__global__ void k_gram_dev_sum(const double *__restrict__ part, double *__restrict__ out) {
    double s = threadIdx.x < GD_CTAS ? part[threadIdx.x] : 0.0;
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (threadIdx.x == 0) *out = sqrt(s);
}

// M[a][b] = conj(M[b][a]) for a > b: the lower triangle of a Hermitian matrix from its upper one
__global__ void k_mirror_lower(int m, z64 *__restrict__ M) {
    for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < m * m; idx += gridDim.x * blockDim.x) {
        const int a = idx / m, b = idx % m;
        if (a > b) M[idx] = conj(M[(int64_t)b * m + a]);
    }
}

// Part of a product: rows [r0, r0 + rows), columns [c0, c0 + cols) of op(A) op(B)
// over the summation range [k0, k0 + ks) (offsets in the storage of each op).
GemmDesc sub_desc(GemmDesc d, int opA, int opB, int64_t r0, int64_t rows, int64_t c0, int64_t cols, int64_t k0,
                  int64_t ks) {
    const bool rowA = opA == 0 || opA == 3, rowB = opB == 0 || opB == 3;
    d.a_off += rowA ? r0 * d.lda + k0 : r0 + k0 * d.lda;
    d.b_off += rowB ? k0 * d.ldb + c0 : k0 + c0 * d.ldb;
    d.c_off += r0 * d.ldc + c0;
    d.M = rows;
    d.N = cols;
    d.K = ks;
    return d;
}
constexpr int64_t TT = 32;   // tile edge of the FP64 product kernel
// The block upper triangle (tiles on or above the diagonal) of a Hermitian square product
std::vector<GemmDesc> upper_tiles(const GemmDesc &d, int opA, int opB) {
    std::vector<GemmDesc> g;
    for (int64_t r0 = 0; r0 < d.M; r0 += TT)
        g.push_back(sub_desc(d, opA, opB, r0, std::min(TT, d.M - r0), r0, d.N - r0, 0, d.K));
    return g;
}
// op(A) lower triangular (row i is zero beyond column i): row tiles summed up to their last row
std::vector<GemmDesc> lower_a_tiles(const GemmDesc &d, int opA, int opB) {
    std::vector<GemmDesc> g;
    for (int64_t r0 = 0; r0 < d.M; r0 += TT) {
        const int64_t rows = std::min(TT, d.M - r0);
        g.push_back(sub_desc(d, opA, opB, r0, rows, 0, d.N, 0, std::min(d.K, r0 + rows)));
    }
    return g;
}
// op(A) upper triangular (row i is zero before column i): row tiles summed from their first row
std::vector<GemmDesc> upper_a_tiles(const GemmDesc &d, int opA, int opB) {
    std::vector<GemmDesc> g;
    for (int64_t r0 = 0; r0 < d.M; r0 += TT)
        if (r0 < d.K) g.push_back(sub_desc(d, opA, opB, r0, std::min(TT, d.M - r0), 0, d.N, r0, d.K - r0));
    return g;
}
// op(B) upper triangular (column j is zero below row j): column tiles summed up to their last column
std::vector<GemmDesc> upper_b_tiles(const GemmDesc &d, int opA, int opB) {
    std::vector<GemmDesc> g;
    for (int64_t c0 = 0; c0 < d.N; c0 += TT) {
        const int64_t cols = std::min(TT, d.N - c0);
        g.push_back(sub_desc(d, opA, opB, 0, d.M, c0, cols, 0, std::min(d.K, c0 + cols)));
    }
    return g;
}

inline unsigned nb(int64_t work) { return (unsigned)std::max<int64_t>(1, std::min<int64_t>((work + 255) / 256, 4096)); }

struct Ctx {
    cudaStream_t st;
    DevBuf<z64> M, R, Rinv, X, T1, Rf, Dinv;
    DevBuf<int> perm, rank, err, status;
    DevBuf<double> rnrm, scale, dev;
    bool perm_id = true;   // the last factorisation kept the order (perm is the identity)
    std::vector<int> hperm;
};

// Cholesky QR applies its second pass only where the first leaves the block
// visibly non-orthonormal: the second pass changes Q by about ||Q1^H Q1 - I||,
// so below this bound on that Frobenius norm (and hence on the 2-norm) the
// first pass is kept.
constexpr double ORTH_TOL = 1e-12;
// Block Gram-Schmidt: one pass leaves a vector about u ||w0|| / ||w1|| away
// from orthogonal to the basis, so the second pass is skipped when every
// vector kept at least GS_KEEP of its norm (dimension factors included, well
// under ORTH_TOL); otherwise its coefficients are formed and applied when
// they exceed ORTH_TOL of the block.
constexpr double GS_KEEP = 0.1;

// ||M - I||_F of the m x m Gram matrix in ctx.M (host sync).
double gram_dev(Ctx &c, int m) {
    k_gram_dev<<<GD_CTAS, 256, 0, c.st>>>(m, c.M.p, c.dev.p + 1);
    launched("k_gram_dev");
    k_gram_dev_sum<<<1, 32, 0, c.st>>>(c.dev.p + 1, c.dev.p);
    launched("k_gram_dev_sum");
    double h = 0.0;
    CBFM_CUDA(cudaMemcpyAsync(&h, c.dev.p, sizeof(double), cudaMemcpyDeviceToHost, c.st));
    CBFM_CUDA(cudaStreamSynchronize(c.st));
    return h;
}

// Cluster size of the blocked Cholesky on this device: 16 CTAs where a
// cluster of 16 can be resident (non-portable size), else 8.
template <int CC>
cudaLaunchConfig_t chol_cfg(int m, cudaStream_t st, cudaLaunchAttribute *at) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(CC, 1, 1);
    cfg.blockDim = dim3(CH_THREADS, 1, 1);
    cfg.dynamicSmemBytes = chol_cl_smem<CC>(m);
    cfg.stream = st;
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = CC;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cfg;
}

int chol_cluster_size() {
    static std::atomic<int> size[64];   // zero-initialised: not yet chosen
    int dev = 0;
    CBFM_CUDA(cudaGetDevice(&dev));
    if (dev < 64) {
        const int known = size[dev].load(std::memory_order_acquire);
        if (known) return known;
    }
    CBFM_CUDA(cudaFuncSetAttribute(k_chol_cl<8>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   (int)chol_cl_smem<8>(PCHOL_MAX)));
    CBFM_CUDA(cudaFuncSetAttribute(k_chol_cl<16>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   (int)chol_cl_smem<16>(PCHOL_MAX)));
    int pick = 8;
    if (cudaFuncSetAttribute(k_chol_cl<16>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) == cudaSuccess) {
        cudaLaunchAttribute at[1];
        const cudaLaunchConfig_t cfg = chol_cfg<16>(PCHOL_MAX, 0, at);
        int nclusters = 0;
        if (cudaOccupancyMaxActiveClusters(&nclusters, k_chol_cl<16>, &cfg) == cudaSuccess && nclusters >= 1) pick = 16;
    }
    (void)cudaGetLastError();   // a refused non-portable size is not an error here
    if (dev < 64) size[dev].store(pick, std::memory_order_release);
    return pick;
}

// Cholesky on the m x m Gram matrix already in ctx.M; returns rank (host sync).
// First the blocked factorisation without pivoting (rows with a zero
// diagonal moved last); where one of its pivots falls below tol * max
// diagonal and `pivot` is set, the pivoted factorisation runs instead, which
// drops the dependent directions.  Without `pivot` the position of the
// failing pivot is returned as the rank.
int pchol(Ctx &c, int m, double tol, bool pivot) {
    static std::atomic<bool> attr_set[64];   // zero-initialised (static storage)
    int dev = 0;
    CBFM_CUDA(cudaGetDevice(&dev));
    if (dev < 64 && !attr_set[dev].load(std::memory_order_acquire)) {
        CBFM_CUDA(cudaFuncSetAttribute(k_pchol_cl, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)pchol_cl_smem(PCHOL_MAX)));
        CBFM_CUDA(cudaFuncSetAttribute(k_trinv, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)trinv_smem(PCHOL_MAX)));
        attr_set[dev].store(true, std::memory_order_release);
    }
    CBFM_REQUIRE(m >= 1 && m <= PCHOL_MAX, "Cholesky: block width out of range");
    const int cc = chol_cluster_size();
    {
        // algorithmic work of a full-rank factorisation and of the triangular inverse: m^3/6 complex MACs each
        prof_add_work("k_chol_blk", 8.0 * m * m * m / 6.0, 16.0 * m * m);
        ProfScope ps_("k_chol_blk", c.st);
        cudaLaunchAttribute at[1];
        if (cc == 16) {
            const cudaLaunchConfig_t cfg = chol_cfg<16>(m, c.st, at);
            CBFM_CUDA(cudaLaunchKernelEx(&cfg, k_chol_cl<16>, m, (const z64 *)c.M.p, tol, c.perm.p, c.R.p, c.Dinv.p,
                                         c.rank.p, c.status.p, c.err.p));
        } else {
            const cudaLaunchConfig_t cfg = chol_cfg<8>(m, c.st, at);
            CBFM_CUDA(cudaLaunchKernelEx(&cfg, k_chol_cl<8>, m, (const z64 *)c.M.p, tol, c.perm.p, c.R.p, c.Dinv.p,
                                         c.rank.p, c.status.p, c.err.p));
        }
        launched("k_chol_cl");
    }
    {
        prof_add_work("k_trinv_blk", 8.0 * m * m * m / 6.0, 32.0 * m * m);
        ProfScope ps_("k_trinv_blk", c.st);
        k_trinv_blk<<<m, 128, 0, c.st>>>(m, c.R.p, c.Dinv.p, c.rank.p, c.status.p, c.Rinv.p);
        launched("k_trinv_blk");
    }
    int hr[3] = {0, 0, 0};
    c.hperm.resize(m);
    CBFM_CUDA(cudaMemcpyAsync(&hr[0], c.rank.p, sizeof(int), cudaMemcpyDeviceToHost, c.st));
    CBFM_CUDA(cudaMemcpyAsync(&hr[1], c.err.p, sizeof(int), cudaMemcpyDeviceToHost, c.st));
    CBFM_CUDA(cudaMemcpyAsync(&hr[2], c.status.p, sizeof(int), cudaMemcpyDeviceToHost, c.st));
    CBFM_CUDA(cudaMemcpyAsync(c.hperm.data(), c.perm.p, sizeof(int) * m, cudaMemcpyDeviceToHost, c.st));
    CBFM_CUDA(cudaStreamSynchronize(c.st));
    if (hr[1]) throw Fail{CBFM_ETIMEOUT, "Cholesky: a cluster synchronisation expired"};
    c.perm_id = true;
    for (int i = 0; i < m; ++i) c.perm_id &= c.hperm[i] == i;
    if (hr[2] == 0 || !pivot) return hr[0];
    c.perm_id = false;
    k_mirror_lower<<<nb((int64_t)m * m), 256, 0, c.st>>>(m, c.M.p);   // the pivoted kernel reads whole rows
    launched("k_mirror_lower");
    {
        prof_add_work("k_pchol", 8.0 * m * m * m / 6.0, 16.0 * m * m);
        prof_add_work("k_trinv", 8.0 * m * m * m / 6.0, 32.0 * m * m);
        ProfScope ps_("k_pchol", c.st);
        k_pchol_cl<<<PC_CL, PCHOL_THREADS, pchol_cl_smem(m), c.st>>>(m, c.M.p, c.perm.p, c.R.p, c.rank.p, tol, 1,
                                                                     c.err.p);
        launched("k_pchol");
    }
    {
        ProfScope ps_("k_trinv", c.st);
        k_trinv<<<m, PCHOL_MAX, trinv_smem(m), c.st>>>(m, c.R.p, c.rank.p, c.Rinv.p);
        launched("k_trinv");
    }
    CBFM_CUDA(cudaMemcpyAsync(&hr[0], c.rank.p, sizeof(int), cudaMemcpyDeviceToHost, c.st));
    CBFM_CUDA(cudaMemcpyAsync(&hr[1], c.err.p, sizeof(int), cudaMemcpyDeviceToHost, c.st));
    CBFM_CUDA(cudaStreamSynchronize(c.st));
    if (hr[1]) throw Fail{CBFM_ETIMEOUT, "pivoted Cholesky: a cluster synchronisation expired"};
    return hr[0];
}

// Rank-revealing orthonormalisation of m row vectors W (m x n, ld n; W is
// overwritten): rows with norm <= drop * ref are treated as exhausted, the
// others are scaled to unit norm, then Cholesky QR (the Cholesky pivoted,
// dropping directions whose scaled Gram pivot falls below tol), repeated
// without pivoting unless the first pass is orthonormal to ORTH_TOL.
// Q (r x n) goes to Qdst and Rfull (r x m, ld m) satisfies
// W_in[c] = sum_i Rfull[i][c] Q[i] up to the dropped parts.  Returns r.
int cholqr2_rows(Ctx &c, z64 *W, int m, int64_t n, z64 *Qdst, z64 *Rfull, double tol, double ref, double drop) {
    GemmSite site_("site:cholqr_rows");
    k_rownorm<<<m, 256, 0, c.st>>>(n, W, c.rnrm.p);
    launched("k_rownorm");
    if (ref <= 0.0) {
        std::vector<double> h(m);
        CBFM_CUDA(cudaMemcpyAsync(h.data(), c.rnrm.p, sizeof(double) * m, cudaMemcpyDeviceToHost, c.st));
        CBFM_CUDA(cudaStreamSynchronize(c.st));
        for (double v : h) ref = std::max(ref, v);
        if (ref <= 0.0) return 0;
    }
    {
        dim3 g((unsigned)std::min<int64_t>((n + 255) / 256, 64), (unsigned)m);
        k_scale_rows<<<g, 256, 0, c.st>>>(n, W, c.rnrm.p, ref, drop, c.scale.p);
        launched("k_scale_rows");
    }
    // pass 1 (pivoted): M[a][b] = sum_k conj(W[a][k]) W[b][k], upper triangle
    gemm_grouped<double>(upper_tiles(GemmDesc{m, m, n, 0, n, 0, n, 0, m}, 3, 1), 3, 1, W, W, c.M.p, false, c.st);
    const int r = pchol(c, m, tol, true);
    if (r == 0) return 0;
    k_zero2d<<<nb((int64_t)r * m), 256, 0, c.st>>>(r, m, c.X.p, m);
    launched("k_zero2d");
    k_make_x<<<nb((int64_t)r * r), 256, 0, c.st>>>(m, r, c.perm.p, c.Rinv.p, c.X.p);
    launched("k_make_x");
    k_zero2d<<<nb((int64_t)r * m), 256, 0, c.st>>>(r, m, c.Rf.p, m);
    launched("k_zero2d");
    k_unpermute_r<<<nb((int64_t)r * m), 256, 0, c.st>>>(m, r, c.perm.p, c.R.p, c.Rf.p);
    launched("k_unpermute_r");
    // Q1 = X W  -> T1 (r x n); X is lower triangular when the order was kept
    {
        const GemmDesc dq{r, n, m, 0, m, 0, n, 0, n};
        gemm_grouped<double>(c.perm_id ? lower_a_tiles(dq, 0, 0) : std::vector<GemmDesc>{dq}, 0, 0, c.X.p, W, c.T1.p,
                             false, c.st);
    }
    // pass 2 (no pivoting) on Q1, unless Q1 is already orthonormal to ORTH_TOL
    gemm_grouped<double>(upper_tiles(GemmDesc{r, r, n, 0, n, 0, n, 0, r}, 3, 1), 3, 1, c.T1.p, c.T1.p, c.M.p, false,
                         c.st);
    if (gram_dev(c, r) <= ORTH_TOL) {
        CBFM_CUDA(cudaMemcpyAsync(Qdst, c.T1.p, sizeof(z64) * r * n, cudaMemcpyDeviceToDevice, c.st));
        k_copy2d<<<nb((int64_t)r * m), 256, 0, c.st>>>(r, m, c.Rf.p, m, Rfull, m, 0);
        launched("k_copy2d");
        k_scale_cols<<<nb((int64_t)r * m), 256, 0, c.st>>>(r, m, Rfull, c.scale.p);
        launched("k_scale_cols");
        return r;
    }
    const int r2 = pchol(c, r, 0.0, false);
    if (r2 != r) throw Fail{CBFM_ESINGULAR, "block GMRES: second Cholesky QR pass lost rank"};
    // Q = Rinv2^T Q1 : X2[i][l] = Rinv2[l][i]  (identity permutation)
    k_zero2d<<<nb((int64_t)r * r), 256, 0, c.st>>>(r, r, c.X.p, r);
    launched("k_zero2d");
    k_make_x<<<nb((int64_t)r * r), 256, 0, c.st>>>(r, r, c.perm.p, c.Rinv.p, c.X.p);
    launched("k_make_x");
    gemm_grouped<double>(lower_a_tiles(GemmDesc{r, n, r, 0, r, 0, n, 0, n}, 0, 0), 0, 0, c.X.p, c.T1.p, Qdst, false,
                         c.st);
    // Rfull = R2 Rfull1 diag(scale) (r x m), R2 is r x r upper triangular with leading dimension r
    gemm_grouped<double>(upper_a_tiles(GemmDesc{r, m, r, 0, r, 0, m, 0, m}, 0, 0), 0, 0, c.R.p, c.Rf.p, Rfull, false,
                         c.st);
    k_scale_cols<<<nb((int64_t)r * m), 256, 0, c.st>>>(r, m, Rfull, c.scale.p);
    launched("k_scale_cols");
    return r;
}

// Cholesky QR of the p columns of a d x p matrix H (ld ldh) in place,
// repeated unless the first pass is orthonormal to ORTH_TOL:
// H <- Q (d x p), Rout (p x p, ld ldr) with H_in = Q Rout; RinvOut (p x p, ld
// ldr) = Rout^{-1} (= R1^{-1} R2^{-1} after two passes).  The Cholesky
// factors of ctx have leading dimension p.
void cholqr2_cols(Ctx &c, z64 *H, int d, int p, int64_t ldh, z64 *Rout, z64 *RinvOut, int64_t ldr,
                  DevBuf<z64> &tmp) {
    GemmSite site_("site:cholqr_hess");
    for (int pass = 0; pass < 2; ++pass) {
        gemm_grouped<double>(upper_tiles(GemmDesc{p, p, d, 0, ldh, 0, ldh, 0, p}, 2, 0), 2, 0, H, H, c.M.p, false,
                             c.st);
        if (pass == 1 && gram_dev(c, p) <= ORTH_TOL) break;   // the first pass is orthonormal already
        const int r = pchol(c, p, 0.0, false);
        if (r != p) throw Fail{CBFM_ESINGULAR, "block GMRES: block Hessenberg lost column rank"};
        // H <- H Rinv  (via tmp, ld p)
        gemm_grouped<double>(upper_b_tiles(GemmDesc{d, p, p, 0, ldh, 0, p, 0, p}, 0, 0), 0, 0, H, c.Rinv.p, tmp.p,
                             false, c.st);
        k_copy2d<<<nb((int64_t)d * p), 256, 0, c.st>>>(d, p, tmp.p, p, H, ldh, 0);
        launched("k_copy2d");
        if (pass == 0) {
            k_copy2d<<<nb((int64_t)p * p), 256, 0, c.st>>>(p, p, c.R.p, p, Rout, ldr, 0);
            launched("k_copy2d");
            k_copy2d<<<nb((int64_t)p * p), 256, 0, c.st>>>(p, p, c.Rinv.p, p, RinvOut, ldr, 0);
            launched("k_copy2d");
        } else {
            // Rout = R2 R1, RinvOut = R1^{-1} R2^{-1}
            gemm_grouped<double>(upper_a_tiles(GemmDesc{p, p, p, 0, p, 0, ldr, 0, p}, 0, 0), 0, 0, c.R.p, Rout, tmp.p,
                                 false, c.st);
            k_copy2d<<<nb((int64_t)p * p), 256, 0, c.st>>>(p, p, tmp.p, p, Rout, ldr, 0);
            launched("k_copy2d");
            gemm_grouped<double>(upper_a_tiles(GemmDesc{p, p, p, 0, ldr, 0, p, 0, p}, 0, 0), 0, 0, RinvOut, c.Rinv.p,
                                 tmp.p, false, c.st);
            k_copy2d<<<nb((int64_t)p * p), 256, 0, c.st>>>(p, p, tmp.p, p, RinvOut, ldr, 0);
            launched("k_copy2d");
        }
    }
}

// Row vectors times a matrix, out[r] = M in[r] for r < rows (M n x n
// row-major, rows of length n), as one GEMM out = in M^T: complex64 M with
// the rows rounded to complex64 and FP32 accumulation when M32 is given,
// else FP64.  With `halves` only the two diagonal halves of M are used (M is
// block diagonal: the inverse of G^CBF).  s_in, s_out: rows x n scratch.
void rows_times(int64_t n, const z64 *M64, const c32 *M32, const z64 *in, z64 *out, int rows, bool halves,
                cudaStream_t st, c32 *s_in, c32 *s_out) {
    std::vector<GemmDesc> g;
    if (halves) {
        const int64_t h = n / 2;
        g.push_back(GemmDesc{rows, h, h, 0, n, 0, n, 0, n});
        g.push_back(GemmDesc{rows, h, h, h, n, h * n + h, n, h, n});
    } else {
        g.push_back(GemmDesc{rows, n, n, 0, n, 0, n, 0, n});
    }
    if (M32) {
        launch_z64_to_c32(in, s_in, (int64_t)rows * n, st);
        gemm_grouped<float>(g, 0, 1, s_in, M32, s_out, false, st);
        launch_c32_to_z64(s_out, out, (int64_t)rows * n, st);
    } else {
        gemm_grouped<double>(g, 0, 1, in, M64, out, false, st);
    }
}

}  // namespace

GmresOut bgmres_solve(Red &rd, const z64 *d_b, int nrhs, double tol, int maxit, int restart, int pc, z64 *d_x,
                      cudaStream_t st, BgmresJoin *join, DevBuf<z64> *x_all) {
    const int64_t n = rd.n;
    CBFM_REQUIRE(nrhs >= 1 && nrhs <= PCHOL_MAX, "block GMRES handles at most 128 right-hand sides per call");
    CBFM_REQUIRE(join == nullptr || x_all != nullptr, "block GMRES with joins needs an output buffer");
    int p = nrhs;
    const double rank_tol = 1e-14;   // pivot threshold of the scaled Gram matrix (unit diagonal)
    const double drop_tol = 1e-12;   // rows below this fraction of the reference norm are exhausted
    // Buffers whose size follows the number of right-hand sides p are set up by
    // setup() (again when right-hand sides join); the Cholesky factors of ctx
    // are sized for the largest block width.
    int64_t dcap = 0, dcap2 = 0;   // basis capacity (dimensions), at least one block beyond the first
    Ctx c;
    c.st = st;
    c.M.alloc((size_t)PCHOL_MAX * PCHOL_MAX);
    c.R.alloc((size_t)PCHOL_MAX * PCHOL_MAX);
    c.Rinv.alloc((size_t)PCHOL_MAX * PCHOL_MAX);
    c.X.alloc((size_t)PCHOL_MAX * PCHOL_MAX);
    c.Rf.alloc((size_t)PCHOL_MAX * PCHOL_MAX);
    c.perm.alloc(PCHOL_MAX);
    c.rank.alloc(1);
    c.err.alloc(1);
    c.status.alloc(1);
    c.Dinv.alloc((size_t)CH_NPAN * CH_B * CH_B);
    CBFM_CUDA(cudaMemsetAsync(c.err.p, 0, sizeof(int), st));
    c.rnrm.alloc(PCHOL_MAX);
    c.scale.alloc(PCHOL_MAX);
    c.dev.alloc(1 + GD_CTAS);   // the deviation and its per-CTA partials
    DevBuf<z64> V, W, HcT, Hn, Qh, Rh, Gv, E1S, Rv, Y, Z, tmp, tmp2, RinvBlk, Rw, Bm, Rout;
    DevBuf<double> bnorm, rnorm, rnorm0, fro_col;
    DevBuf<int> dmask, dsel;
    DevBuf<z64> Ws;            // the vectors of a selective second Gram-Schmidt pass
    DevBuf<c32> s_in, s_out;   // complex64 rows for the mixed-precision products
    DevBuf<c32> V32, Z32;      // complex64 basis and coefficients for the mixed-precision solution update
    DevBuf<z64> zin;           // inexact CMP: the inner GMRES's (G^CBF)^{-1} in, the input of the product with A
    std::vector<double> h_bn, h_rn, h_w1, h_h0, h_h1, h_col;
    auto setup = [&]() {
        dcap = std::max<int64_t>(2 * p, std::min<int64_t>((int64_t)std::max(restart, 2 * p), n + p));
        dcap2 = dcap + p;
        c.T1.alloc((size_t)p * n);
        Ws.alloc((size_t)p * n);
        V.alloc((size_t)dcap * n);
        W.alloc((size_t)p * n);
        HcT.alloc((size_t)p * dcap);
        Hn.alloc((size_t)dcap2 * p);
        Qh.alloc((size_t)dcap2 * dcap);
        Rh.alloc((size_t)dcap * dcap);
        Gv.alloc((size_t)dcap * p);
        E1S.alloc((size_t)dcap2 * p);
        Rv.alloc((size_t)dcap2 * p);
        Z.alloc((size_t)dcap * p);
        tmp.alloc((size_t)std::max<int64_t>(dcap2 * p, p * n));
        tmp2.alloc((size_t)dcap * p);
        RinvBlk.alloc((size_t)dcap * p);   // diagonal blocks of Rh^{-1}, stacked (p_j x p_j each, ld p)
        Rw.alloc((size_t)p * p);
        Rout.alloc((size_t)p * p);
        rnorm.alloc(p);
        rnorm0.alloc(p);
        fro_col.alloc((size_t)std::max<int64_t>(dcap, p));
        h_col.assign((size_t)std::max<int64_t>(dcap, p), 0.0);
        h_rn.assign(p, 0.0);
        h_w1.assign(p, 0.0);
        h_h0.assign(p, 0.0);
        h_h1.assign(p, 0.0);
        if (rd.prec != CBFM_FP64) {
            s_in.alloc((size_t)p * n);
            s_out.alloc((size_t)p * n);
        }
        V32.release();
        Z32.release();
        zin.release();
    };
    setup();
    // the right-hand sides (rows), their solutions y and norms
    Bm.alloc((size_t)p * n);
    CBFM_CUDA(cudaMemcpyAsync(Bm.p, d_b, sizeof(z64) * p * n, cudaMemcpyDeviceToDevice, st));
    Y.alloc((size_t)p * n);
    CBFM_CUDA(cudaMemsetAsync(Y.p, 0, sizeof(z64) * p * n, st));
    bnorm.alloc(PCHOL_MAX);
    k_rownorm<<<p, 256, 0, st>>>(n, Bm.p, bnorm.p);
    launched("k_rownorm");
    h_bn.assign(p, 0.0);
    // ||X||_F of a rows x cols block: column norms (one block each), summed on the host (host sync)
    auto fro = [&](int rows, int cols, const z64 *X, int64_t ld) {
        k_colnorm<<<cols, 256, 0, st>>>(rows, cols, X, ld, fro_col.p);
        launched("k_colnorm");
        CBFM_CUDA(cudaMemcpyAsync(h_col.data(), fro_col.p, sizeof(double) * cols, cudaMemcpyDeviceToHost, st));
        CBFM_CUDA(cudaStreamSynchronize(st));
        double a = 0.0;
        for (int c = 0; c < cols; ++c) a += h_col[c] * h_col[c];
        return std::sqrt(a);
    };
    // sqrt of the sum of squares of the first k norms; the smallest ratio
    // after / before over the vectors that had a norm
    auto norm_sum = [](const std::vector<double> &v, int k) {
        double a = 0.0;
        for (int i = 0; i < k; ++i) a += v[i] * v[i];
        return std::sqrt(a);
    };
    auto min_ratio = [](const std::vector<double> &after, const std::vector<double> &before, int k) {
        double r = 1.0;
        for (int i = 0; i < k; ++i)
            if (before[i] > 0.0) r = std::min(r, after[i] / before[i]);
        return r;
    };
    CBFM_CUDA(cudaMemcpyAsync(h_bn.data(), bnorm.p, sizeof(double) * p, cudaMemcpyDeviceToHost, st));
    CBFM_CUDA(cudaStreamSynchronize(st));

    auto applyB = [&](const z64 *in, z64 *out, int rows) {
        if (pc == CBFM_PC_CMP_INEXACT) {
            if (zin.p == nullptr) zin.alloc((size_t)p * n);
            cmp_inner_apply(rd, in, zin.p, rows, st);
            in = zin.p;
        }
        if (rd.prec != CBFM_FP64)
            rows_times(n, nullptr, pc_op32(rd, pc), in, out, rows, false, st, s_in.p, s_out.p);
        else rows_times(n, pc_op64(rd, pc), nullptr, in, out, rows, false, st, nullptr, nullptr);
    };

    GmresOut out;
    out.iters.assign(p, -1);
    out.resid.assign(p, 1.0);
    std::vector<int> conv_at(p, -1), join_at(p, 0);
    std::vector<char> frozen(p, 0);
    int total_blocks = 0;
    bool all_conv = false, breakdown = false;
    // Right-hand sides waiting to join: taken at a restart they asked for
    // (`asked`), or when the others are done and the session does not close
    // because some arrived meanwhile.  True when some were added (their
    // starting guess zero; the others keep their iterate).
    auto absorb_joins = [&](bool asked) {
        if (join == nullptr) return false;
        bool take = asked;
        if ((all_conv || breakdown) && !join->close_if_idle()) take = true;
        if (!take || total_blocks >= maxit) return false;
        DevBuf<z64> rows;
        const int k = join->take(st, rows);
        if (k <= 0) return false;
        CBFM_REQUIRE(p + k <= PCHOL_MAX, "block GMRES: more than 128 right-hand sides joined");
        DevBuf<z64> Bn, Yn;
        Bn.alloc((size_t)(p + k) * n);
        Yn.alloc((size_t)(p + k) * n);
        CBFM_CUDA(cudaMemcpyAsync(Bn.p, Bm.p, sizeof(z64) * p * n, cudaMemcpyDeviceToDevice, st));
        CBFM_CUDA(cudaMemcpyAsync(Bn.p + (int64_t)p * n, rows.p, sizeof(z64) * k * n, cudaMemcpyDeviceToDevice, st));
        CBFM_CUDA(cudaMemcpyAsync(Yn.p, Y.p, sizeof(z64) * p * n, cudaMemcpyDeviceToDevice, st));
        CBFM_CUDA(cudaMemsetAsync(Yn.p + (int64_t)p * n, 0, sizeof(z64) * k * n, st));
        k_rownorm<<<k, 256, 0, st>>>(n, rows.p, bnorm.p + p);
        launched("k_rownorm");
        h_bn.resize(p + k);
        CBFM_CUDA(cudaMemcpyAsync(h_bn.data() + p, bnorm.p + p, sizeof(double) * k, cudaMemcpyDeviceToHost, st));
        CBFM_CUDA(cudaStreamSynchronize(st));
        Bn.give(Bm);
        Yn.give(Y);
        out.iters.resize(p + k, -1);
        out.resid.resize(p + k, 1.0);
        conv_at.resize(p + k, -1);
        join_at.resize(p + k, total_blocks);
        frozen.resize(p + k, 0);
        p += k;
        setup();
        all_conv = breakdown = false;
        return true;
    };
    while (!all_conv && !breakdown && total_blocks < maxit) {
        // residual block R0 = Bm - B Y (rows), orthonormalised: R0[c] = sum_i S[i][c] V1[i]
        bool fresh = true;   // every right-hand side still at y = 0
        for (int q = 0; q < p; ++q) fresh &= (join_at[q] == total_blocks);
        if (fresh) {
            CBFM_CUDA(cudaMemcpyAsync(tmp.p, Bm.p, sizeof(z64) * p * n, cudaMemcpyDeviceToDevice, st));
        } else {
            applyB(Y.p, W.p, p);
            k_sub_rows<<<nb(p * n), 256, 0, st>>>(p * n, Bm.p, W.p, tmp.p);
            launched("k_sub_rows");
        }
        // with joins, a restart keeps the converged right-hand sides out of the new block
        bool any_frozen = false;
        for (int q = 0; q < p; ++q) {
            frozen[q] = join != nullptr && conv_at[q] >= 0;
            any_frozen |= frozen[q] != 0;
        }
        if (any_frozen) {
            std::vector<int> hm(frozen.begin(), frozen.end());
            dmask.alloc(p);
            CBFM_CUDA(cudaMemcpyAsync(dmask.p, hm.data(), sizeof(int) * p, cudaMemcpyHostToDevice, st));
            k_zero_rows_masked<<<nb(p * n), 256, 0, st>>>(p, n, dmask.p, tmp.p);
            launched("k_zero_rows_masked");
            CBFM_CUDA(cudaStreamSynchronize(st));   // hm is released on return from this block
        }
        bool joined = false;
        CBFM_CUDA(cudaMemsetAsync(E1S.p, 0, sizeof(z64) * dcap2 * p, st));
        CBFM_CUDA(cudaMemsetAsync(Qh.p, 0, sizeof(z64) * dcap2 * dcap, st));
        CBFM_CUDA(cudaMemsetAsync(Rh.p, 0, sizeof(z64) * dcap * dcap, st));
        const int p1 = cholqr2_rows(c, tmp.p, p, n, V.p, E1S.p, rank_tol, 0.0, drop_tol);
        CBFM_CUDA(cudaMemcpyAsync(Rv.p, E1S.p, sizeof(z64) * dcap2 * p, cudaMemcpyDeviceToDevice, st));
        if (p1 == 0) {   // residual block is zero: current iterate is exact
            for (int r = 0; r < p; ++r) {
                if (frozen[r]) continue;
                out.resid[r] = 0.0;
                if (conv_at[r] < 0) conv_at[r] = total_blocks;
            }
            all_conv = true;
            if (absorb_joins(false)) continue;
            break;
        }
        std::vector<int64_t> dims{0, p1};   // dims[i] = first basis index of block i
        int J = 0;                          // block columns of Hbar processed in this cycle
        while (true) {
            const int64_t d0 = dims[J], d1 = dims[J + 1];
            const int pjc = (int)(d1 - d0);
            if (dcap - d1 < pjc) break;   // no room for another block: solve and restart
            // W = B V_J; the norms before orthogonalisation set the scale for exhaustion
            applyB(V.p + d0 * n, W.p, pjc);
            // the norms before the orthogonalisation, read back with those after its first pass
            k_rownorm<<<pjc, 256, 0, st>>>(n, W.p, rnorm0.p);
            launched("k_rownorm");
            double wref = 0.0;
            // block classical Gram-Schmidt; HcT (pjc x d1) collects the coefficients.  The second
            // pass runs on the vectors that kept less than GS_KEEP of their norm in the first (the
            // others are orthogonal to the basis to ~10 u already), gathered into Ws
            {
                GemmSite site_("site:gs1");
                gemm_grouped<double>({GemmDesc{pjc, d1, n, 0, n, 0, n, 0, dcap}}, 0, 2, W.p, V.p, tmp2.p, false, st);
                gemm_grouped<double>({GemmDesc{pjc, n, d1, 0, dcap, 0, n, 0, n}}, 0, 0, tmp2.p, V.p, W.p, true, st,
                                     -1.0);
                k_copy2d<<<nb(pjc * d1), 256, 0, st>>>(pjc, (int)d1, tmp2.p, dcap, HcT.p, dcap, 0);
                launched("k_copy2d");
                k_rownorm<<<pjc, 256, 0, st>>>(n, W.p, rnorm.p);
                launched("k_rownorm");
                CBFM_CUDA(cudaMemcpyAsync(h_rn.data(), rnorm0.p, sizeof(double) * pjc, cudaMemcpyDeviceToHost, st));
                CBFM_CUDA(cudaMemcpyAsync(h_w1.data(), rnorm.p, sizeof(double) * pjc, cudaMemcpyDeviceToHost, st));
                CBFM_CUDA(cudaStreamSynchronize(st));
                for (int q = 0; q < pjc; ++q) wref = std::max(wref, h_rn[q]);
            }
            std::vector<int> sel;   // vectors that need the second pass
            std::vector<double> w1sel;
            for (int q = 0; q < pjc; ++q)
                if (h_rn[q] > 0.0 && h_w1[q] / h_rn[q] < GS_KEEP) {
                    sel.push_back(q);
                    w1sel.push_back(h_w1[q]);
                }
            if (!sel.empty()) {
                GemmSite site_("site:gs2");
                const int k = (int)sel.size();
                const bool all = k == pjc;
                if (!all) {
                    dsel.alloc(k);
                    CBFM_CUDA(cudaMemcpyAsync(dsel.p, sel.data(), sizeof(int) * k, cudaMemcpyHostToDevice, st));
                    k_gather_rows<<<nb((int64_t)k * n), 256, 0, st>>>(k, n, dsel.p, W.p, Ws.p);
                    launched("k_gather_rows");
                }
                z64 *Wk = all ? W.p : Ws.p;
                gemm_grouped<double>({GemmDesc{k, d1, n, 0, n, 0, n, 0, dcap}}, 0, 2, Wk, V.p, tmp2.p, false, st);
                if (fro(k, (int)d1, tmp2.p, dcap) > ORTH_TOL * norm_sum(w1sel, k)) {
                    gemm_grouped<double>({GemmDesc{k, n, d1, 0, dcap, 0, n, 0, n}}, 0, 0, tmp2.p, V.p, Wk, true, st,
                                         -1.0);
                    if (all) {
                        k_copy2d<<<nb(pjc * d1), 256, 0, st>>>(pjc, (int)d1, tmp2.p, dcap, HcT.p, dcap, 1);
                        launched("k_copy2d");
                    } else {
                        k_scatter_rows<<<nb((int64_t)k * n), 256, 0, st>>>(k, n, dsel.p, Ws.p, W.p, 0);
                        launched("k_scatter_rows");
                        k_scatter_rows<<<nb((int64_t)k * d1), 256, 0, st>>>(k, d1, dsel.p, tmp2.p, HcT.p, dcap);
                        launched("k_scatter_rows");
                    }
                }
                if (!all) CBFM_CUDA(cudaStreamSynchronize(st));   // sel is a host vector of this scope
            }
            // orthonormalise the new block (pivoted: drops dependent directions)
            const int r = wref > 0.0 ? cholqr2_rows(c, W.p, pjc, n, V.p + d1 * n, Rw.p, rank_tol, wref, drop_tol) : 0;
            const int rr = r;
            const int64_t d2 = d1 + rr;
            // new block column of Hbar (d2 x pjc, ld p): [C; R_W]
            k_copy_t<<<nb(d1 * pjc), 256, 0, st>>>((int)d1, pjc, HcT.p, dcap, Hn.p, p);
            launched("k_copy_t");
            if (rr > 0) {
                k_copy2d<<<nb(rr * pjc), 256, 0, st>>>(rr, pjc, Rw.p, pjc, Hn.p + d1 * p, p, 0);
                launched("k_copy2d");
            }
            // QR update of Hbar: project the new column block on the previous Q (twice).
            // Hbar is block upper Hessenberg, so column block i of its Q is zero
            // below row dims[i+2]: block i is projected over those rows only, and
            // row block r of the new column meets only the Q blocks i >= r - 1.
            if (d0 > 0) {
                std::vector<GemmDesc> proj, upd;
                for (int i = 0; i < J; ++i)
                    proj.push_back(GemmDesc{dims[i + 1] - dims[i], pjc, dims[i + 2], dims[i], dcap, 0, p,
                                            dims[i] * p, p});
                for (int r = 0; r <= J; ++r) {
                    const int64_t k0 = dims[std::max(0, r - 1)];
                    if (k0 >= d0) continue;
                    upd.push_back(GemmDesc{dims[r + 1] - dims[r], pjc, d0 - k0, dims[r] * dcap + k0, dcap, k0 * p,
                                           p, dims[r] * p, p});
                }
                // norms before the projection into rnorm0 (free again after the Gram-Schmidt
                // read), read together with those after the first pass: one host wait, not two
                k_colnorm<<<pjc, 256, 0, st>>>((int)d2, pjc, Hn.p, p, rnorm0.p);
                launched("k_colnorm");
                for (int pass = 0; pass < 2; ++pass) {
                    GemmSite site_(pass == 0 ? "site:hess_proj1" : "site:hess_proj2");
                    gemm_grouped<double>(proj, 2, 0, Qh.p, Hn.p, tmp2.p, false, st);
                    if (pass == 1 && fro((int)d0, pjc, tmp2.p, p) <= ORTH_TOL * norm_sum(h_h1, pjc)) break;
                    gemm_grouped<double>(upd, 0, 0, Qh.p, tmp2.p, Hn.p, true, st, -1.0);
                    k_copy2d<<<nb(d0 * pjc), 256, 0, st>>>((int)d0, pjc, tmp2.p, p, Rh.p + d0, dcap, pass);
                    launched("k_copy2d");
                    if (pass == 0) {
                        k_colnorm<<<pjc, 256, 0, st>>>((int)d2, pjc, Hn.p, p, rnorm.p);
                        launched("k_colnorm");
                        CBFM_CUDA(cudaMemcpyAsync(h_h0.data(), rnorm0.p, sizeof(double) * pjc, cudaMemcpyDeviceToHost,
                                                  st));
                        CBFM_CUDA(cudaMemcpyAsync(h_h1.data(), rnorm.p, sizeof(double) * pjc, cudaMemcpyDeviceToHost,
                                                  st));
                        CBFM_CUDA(cudaStreamSynchronize(st));
                        if (min_ratio(h_h1, h_h0, pjc) >= GS_KEEP) break;
                    }
                }
            }
            cholqr2_cols(c, Hn.p, (int)d2, pjc, p, Rout.p, RinvBlk.p + d0 * p, p, tmp);
            k_copy2d<<<nb(d2 * pjc), 256, 0, st>>>((int)d2, pjc, Hn.p, p, Qh.p + d0, dcap, 0);
            launched("k_copy2d");
            k_copy2d<<<nb(pjc * pjc), 256, 0, st>>>(pjc, pjc, Rout.p, p, Rh.p + d0 * dcap + d0, dcap, 0);
            launched("k_copy2d");
            // projected right-hand side rows and the residual of the least-squares
            // problem, updated with the new Q block only (Rv = E1S - Q Q^H E1S):
            //   G_J = Q_J^H Rv = Q_J^H E1S  (Q_J is orthogonal to the earlier Q blocks,
            //   and E1S is zero below its first p1 rows),  Rv <- Rv - Q_J G_J
            GemmSite site_ls_("site:ls_rhs");
            gemm_grouped<double>({GemmDesc{pjc, p, p1, 0, p, 0, p, d0 * p, p}}, 2, 0, Hn.p, E1S.p, Gv.p, false, st);
            gemm_grouped<double>({GemmDesc{d2, p, pjc, 0, p, d0 * p, p, 0, p}}, 0, 0, Hn.p, Gv.p, Rv.p, true, st,
                                 -1.0);
            k_colnorm<<<p, 256, 0, st>>>((int)d2, p, Rv.p, p, rnorm.p);
            launched("k_colnorm");
            CBFM_CUDA(cudaMemcpyAsync(h_rn.data(), rnorm.p, sizeof(double) * p, cudaMemcpyDeviceToHost, st));
            CBFM_CUDA(cudaStreamSynchronize(st));
            ++J;
            ++total_blocks;
            bool all = true;
            for (int q = 0; q < p; ++q) {
                if (frozen[q]) continue;   // converged before this cycle; y is final
                const double rel = h_bn[q] > 0 ? h_rn[q] / h_bn[q] : 0.0;
                out.resid[q] = rel;
                if (rel <= tol && conv_at[q] < 0) conv_at[q] = total_blocks;
                all &= (rel <= tol);
            }
            dims.push_back(d2);
            all_conv = all;
            if (r == 0) breakdown = !all;   // invariant subspace: least-squares solution is final
            if (all || r == 0 || total_blocks >= maxit) break;
            if (join != nullptr && join->pending()) {   // right-hand sides wait to join: restart here
                joined = true;
                break;
            }
        }
        // solve Rh Z = Gv (block back substitution) and update Y += Z^T V
        GemmSite site_sol_("site:solution");
        const int64_t dJ = dims[J];
        for (int i = J - 1; i >= 0; --i) {
            const int64_t a0 = dims[i], a1 = dims[i + 1];
            const int pi = (int)(a1 - a0);
            k_copy2d<<<nb(pi * p), 256, 0, st>>>(pi, p, Gv.p + a0 * p, p, tmp2.p, p, 0);
            launched("k_copy2d");
            if (a1 < dJ)
                gemm_grouped<double>({GemmDesc{pi, p, dJ - a1, a0 * dcap + a1, dcap, a1 * p, p, 0, p}}, 0, 0, Rh.p,
                                     Z.p, tmp2.p, true, st, -1.0);
            gemm_grouped<double>({GemmDesc{pi, p, pi, a0 * p, p, 0, p, a0 * p, p}}, 0, 0, RinvBlk.p, tmp2.p, Z.p,
                                 false, st);
        }
        if (rd.prec != CBFM_FP64) {
            // mixed precision: the solution update Y += Z^T V (not part of the orthogonalisation or the
            // residual) in FP32, like the operator product
            if (V32.p == nullptr) {
                V32.alloc((size_t)dcap * n);
                Z32.alloc((size_t)dcap * p);
            }
            launch_z64_to_c32(V.p, V32.p, dJ * n, st);
            launch_z64_to_c32(Z.p, Z32.p, dJ * p, st);
            gemm_grouped<float>({GemmDesc{p, n, dJ, 0, p, 0, n, 0, n}}, 1, 0, Z32.p, V32.p, s_out.p, false, st);
            k_add32to64<<<nb((int64_t)p * n), 256, 0, st>>>((int64_t)p * n, s_out.p, Y.p);
            launched("k_add32to64");
        } else {
            gemm_grouped<double>({GemmDesc{p, n, dJ, 0, p, 0, n, 0, n}}, 1, 0, Z.p, V.p, Y.p, true, st);
        }
        CBFM_CUDA(cudaStreamSynchronize(st));
        if (absorb_joins(joined)) continue;
        if (breakdown) break;
    }
    // x = P y
    if (join != nullptr) {
        x_all->alloc((size_t)p * n);
        d_x = x_all->p;
    }
    if (pc == CBFM_PC_CMP) {   // G^CBF^{-1} is block diagonal (its two halves)
        if (rd.prec != CBFM_FP64) rows_times(n, nullptr, rd.Ginv32.p, Y.p, d_x, p, true, st, s_in.p, s_out.p);
        else rows_times(n, rd.Ginv.p, nullptr, Y.p, d_x, p, true, st, nullptr, nullptr);
    }
    else if (pc == CBFM_PC_TDIAG) tdiag_recover(rd, Y.p, d_x, p, st);
    else if (pc == CBFM_PC_CMP_INEXACT) cmp_inner_apply(rd, Y.p, d_x, p, st);
    else CBFM_CUDA(cudaMemcpyAsync(d_x, Y.p, sizeof(z64) * p * n, cudaMemcpyDeviceToDevice, st));
    CBFM_CUDA(cudaStreamSynchronize(st));
    // iterations counted from the block iteration a right-hand side joined at
    for (int q = 0; q < p; ++q)
        out.iters[q] = conv_at[q] >= 0 ? conv_at[q] - join_at[q] : -(total_blocks - join_at[q]) - 1;
    if (breakdown)
        for (int q = 0; q < p; ++q)
            if (conv_at[q] < 0) out.iters[q] = total_blocks - join_at[q];   // exact within the saturated space
    return out;
}

}  // namespace cbfm
