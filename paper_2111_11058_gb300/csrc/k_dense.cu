// k_dense.cu -- dense complex linear algebra on the GPU: grouped GEMM,
// batched LU solves (primary CBFs, paper Eq. (pcbf)), batched one-sided
// Jacobi SVD (dual orthogonalisation, Eq. (gram_CBF_SVD)) and Gauss-Jordan
// inversion (CBF Gram matrix, Eq. (CBF_Gram_matrix)).
#include <algorithm>
#include <atomic>
#include <vector>

#include <cooperative_groups.h>

#include "cluster.cuh"
#include "internal.cuh"

namespace cbfm {

namespace cg = cooperative_groups;

namespace {

// ------------------------------------------------------------ grouped GEMM
constexpr int GB_M = 64, GB_N = 64, GB_K = 16;

// Up to GB_MAXG problems per launch travel in the kernel parameters (no
// device allocation, no host synchronisation).  When the output tiles of a
// launch are too few to fill the GPU, each problem is split along K into
// `ksplit[g]` slices whose partial results are summed in a fixed order by
// k_splitk_reduce (deterministic).
constexpr int GB_MAXG = 128;

struct GemmBatch {
    int ng;
    int64_t tile_off[GB_MAXG + 1];   // work items (output tiles x K slices) before problem g
    int64_t part_off[GB_MAXG + 1];   // first partial-sum element of problem g (split problems only)
    int64_t red_off[GB_MAXG + 1];    // first output element of problem g in the reduction (split problems only)
    int64_t kchunk[GB_MAXG];         // K range of one slice of problem g
    int ksplit[GB_MAXG];             // K slices of problem g (>= 1)
    GemmDesc d[GB_MAXG];
};

template <typename T>
__device__ __forceinline__ cx<T> load_op(const cx<T> *__restrict__ X, int64_t off, int64_t ld, int64_t r, int64_t c,
                                         int64_t R, int64_t C, int op) {
    // element (r, c) of op(X) where op(X) is R x C; op 0 = X, 1 = X^T, 2 = X^H, 3 = conj(X)
    if (r >= R || c >= C) return cx<T>(0, 0);
    if (op == 0) return X[off + r * ld + c];
    if (op == 3) return conj(X[off + r * ld + c]);
    cx<T> v = X[off + c * ld + r];
    return (op == 2) ? conj(v) : v;
}

template <typename T>
__global__ void __launch_bounds__(256) k_gemm(const __grid_constant__ GemmBatch bt, int opA, int opB,
                                              const cx<T> *__restrict__ A, const cx<T> *__restrict__ B,
                                              cx<T> *__restrict__ C, cx<T> *__restrict__ part, int accumulate,
                                              T alpha) {
    __shared__ cx<T> As[GB_K][GB_M + 1];
    __shared__ cx<T> Bs[GB_K][GB_N + 1];
    const int64_t item = blockIdx.x;
    int g = 0;
    {
        int lo = 0, hi = bt.ng - 1;
        while (lo < hi) {   // last problem with tile_off[g] <= item
            int mid = (lo + hi + 1) / 2;
            if (bt.tile_off[mid] <= item) lo = mid;
            else hi = mid - 1;
        }
        g = lo;
    }
    const GemmDesc d = bt.d[g];
    const int nsplit = bt.ksplit[g];
    int64_t local = item - bt.tile_off[g];
    const int ks = (int)(local % nsplit);
    local /= nsplit;
    const int64_t ntn = (d.N + GB_N - 1) / GB_N;
    const int64_t m0 = (local / ntn) * GB_M, n0 = (local % ntn) * GB_N;
    const int64_t kb = (nsplit > 1) ? (int64_t)ks * bt.kchunk[g] : 0;
    const int64_t ke = (nsplit > 1) ? min(d.K, kb + bt.kchunk[g]) : d.K;
    const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
    cx<T> acc[4][4];
    for (int i = 0; i < 4; ++i)
        for (int j = 0; j < 4; ++j) acc[i][j] = cx<T>(0, 0);
    for (int64_t k0 = kb; k0 < ke; k0 += GB_K) {
        // thread -> element maps chosen so that consecutive threads read consecutive addresses
        for (int idx = threadIdx.x; idx < GB_M * GB_K; idx += 256) {
            const bool rowA = (opA == 0 || opA == 3);
            int mm = rowA ? idx / GB_K : idx % GB_M;
            int kk = rowA ? idx % GB_K : idx / GB_M;
            As[kk][mm] = (k0 + kk < ke) ? load_op(A, d.a_off, d.lda, m0 + mm, k0 + kk, d.M, d.K, opA) : cx<T>(0, 0);
        }
        for (int idx = threadIdx.x; idx < GB_K * GB_N; idx += 256) {
            const bool rowB = (opB == 0 || opB == 3);
            int kk = rowB ? idx / GB_N : idx % GB_K;
            int nn = rowB ? idx % GB_N : idx / GB_K;
            Bs[kk][nn] = (k0 + kk < ke) ? load_op(B, d.b_off, d.ldb, k0 + kk, n0 + nn, d.K, d.N, opB) : cx<T>(0, 0);
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < GB_K; ++kk) {
            cx<T> a[4], b[4];
            for (int i = 0; i < 4; ++i) a[i] = As[kk][ty + 16 * i];
            for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx + 16 * j];
            for (int i = 0; i < 4; ++i)
                for (int j = 0; j < 4; ++j) cfma(acc[i][j], a[i], b[j]);
        }
        __syncthreads();
    }
    for (int i = 0; i < 4; ++i) {
        int64_t r = m0 + ty + 16 * i;
        if (r >= d.M) continue;
        for (int j = 0; j < 4; ++j) {
            int64_t c = n0 + tx + 16 * j;
            if (c >= d.N) continue;
            if (nsplit > 1) {
                part[bt.part_off[g] + ((int64_t)ks * d.M + r) * d.N + c] = acc[i][j];
            } else {
                cx<T> *p = C + d.c_off + r * d.ldc + c;
                cx<T> v = alpha * acc[i][j];
                if (accumulate) *p += v;
                else *p = v;
            }
        }
    }
}

// C[g] = alpha * sum_s part[g][s] (+ C[g]) for every split problem g: fixed
// summation order (deterministic).
template <typename T>
__global__ void k_splitk_reduce(const __grid_constant__ GemmBatch bt, const cx<T> *__restrict__ part,
                                cx<T> *__restrict__ C, int accumulate, T alpha) {
    const int64_t total = bt.red_off[bt.ng];
    for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
         idx += (int64_t)gridDim.x * blockDim.x) {
        int lo = 0, hi = bt.ng - 1;
        while (lo < hi) {   // last problem with red_off[g] <= idx (problems that are not split have no width)
            int mid = (lo + hi + 1) / 2;
            if (bt.red_off[mid] <= idx) lo = mid;
            else hi = mid - 1;
        }
        const GemmDesc &d = bt.d[lo];
        const int64_t e = idx - bt.red_off[lo], mn = d.M * d.N;
        const int64_t r = e / d.N, c = e % d.N;
        const cx<T> *pp = part + bt.part_off[lo] + e;
        cx<T> v(0, 0);
        for (int s = 0; s < bt.ksplit[lo]; ++s) v += pp[(int64_t)s * mn];
        cx<T> *p = C + d.c_off + r * d.ldc + c;
        v = alpha * v;
        if (accumulate) *p += v;
        else *p = v;
    }
}

// ------------------------------------------- stream-K grouped GEMM (FP64)
// FP64 products are limited by the FP64 pipe of each SM (about two DFMA per
// clock on GB300), so an FP64 GEMM runs at the speed of its busiest SM: the
// work must be spread evenly, whatever the shapes.  The problems of one launch
// are cut into units of one 32 x 32 output tile x 16 of K; the units, numbered
// problem by problem, tile by tile, K-step by K-step, are dealt out to G
// CTAs in equal contiguous runs (CTA c takes [c U / G, (c+1) U / G)).  A CTA
// writes every tile it covers completely straight to C; the (at most two)
// tiles cut at the ends of its run go to its two partial-sum slots.  The last
// CTA to finish its part of a cut tile (a counter per tile) adds the slots of
// the tile's CTAs in CTA order (deterministic) and writes C.
//
// Every FP64 warp instruction holds its SM sub-partition's FP64 pipe for
// about 64 clocks, so the complex products use three real multiplications
// instead of four (Higham, "Stability of a method for multiplying complex
// matrices with three real matrix multiplications", SIAM J. Matrix Anal.
// Appl. 13, 1992):  with t1 = sum a_re b_re, t2 = sum a_im b_im and
// t3 = sum (a_re + a_im)(b_re + b_im),  re = t1 - t2,  im = t3 - t1 - t2.
// The sums a_re + a_im and b_re + b_im are formed once per staged element;
// the error stays within a small multiple of the usual bound, normwise.
constexpr int SK_T = 32, SK_K = 16;

struct SkBatch {
    int ng;
    int G;                           // CTAs
    int defer;                       // 1: cut tiles are summed by k_sk_reduce after the launch
    int64_t U;                       // units
    int64_t unit_off[GB_MAXG + 1];   // first unit of problem g
    int64_t tile_off[GB_MAXG + 1];   // first tile of problem g (index of its cut-tile counter)
    int64_t ksteps[GB_MAXG];         // K-steps per tile of problem g
    GemmDesc d[GB_MAXG];
};

__device__ __forceinline__ int sk_group(const SkBatch &bt, int64_t u) {
    int lo = 0, hi = bt.ng - 1;
    while (lo < hi) {   // last problem with unit_off[g] <= u
        int mid = (lo + hi + 1) / 2;
        if (bt.unit_off[mid] <= u) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}
__device__ __forceinline__ int64_t sk_first(int64_t c, const SkBatch &bt) { return c * bt.U / bt.G; }
__device__ __forceinline__ int64_t sk_owner(int64_t u, const SkBatch &bt) { return ((u + 1) * bt.G - 1) / bt.U; }

// The slot a CTA cc used for the tile starting at unit tu0: 0 if the tile is
// where the CTA's units begin, else 1 (a CTA's last, cut tile).
__device__ __forceinline__ int sk_slot(int64_t cc, int64_t tu0, const SkBatch &bt) {
    return (sk_first(cc, bt) >= tu0) ? 0 : 1;
}
constexpr int SK_MAXP = 1024;   // pieces of a cut tile whose slots are looked up once per tile

// The last CTA of a cut tile: C tile = alpha * (sum of the tile's slots in CTA order) (+ C).
// Called by the whole CTA.
__device__ __noinline__ void sk_sum_tile(const SkBatch &bt, int g, int64_t m0, int64_t n0, int64_t tu0, int64_t cf,
                                         int64_t cl, const z64 *part, z64 *C, int accumulate, double alpha) {
    __shared__ unsigned char s_js[SK_MAXP];
    const GemmDesc &d = bt.d[g];
    const int np = (int)(cl - cf + 1);
    for (int q = threadIdx.x; q < np && q < SK_MAXP; q += blockDim.x) s_js[q] = (unsigned char)sk_slot(cf + q, tu0, bt);
    __syncthreads();
    for (int e = threadIdx.x; e < SK_T * SK_T; e += blockDim.x) {
        const int64_t r = m0 + e / SK_T, col = n0 + e % SK_T;
        if (r >= d.M || col >= d.N) continue;
        z64 v(0, 0);
        for (int64_t cc = cf; cc <= cl; ++cc) {
            const int q = (int)(cc - cf);
            const int jslot = q < SK_MAXP ? s_js[q] : sk_slot(cc, tu0, bt);
            const double2 pv = __ldcg(reinterpret_cast<const double2 *>(part) + (2 * cc + jslot) * (SK_T * SK_T) + e);
            v += z64(pv.x, pv.y);
        }
        z64 *pc = C + d.c_off + r * d.ldc + col;
        v = alpha * v;
        if (accumulate) *pc += v;
        else *pc = v;
    }
}

// The cut tiles of a deferred launch: CTA (tile, chunk) sums the tile's
// slots in CTA order for SK_RCH of its entries, one entry per thread, so the
// FP64 adds of a tile cut into many pieces are spread over many SMs.
constexpr int SK_RCH = 128;
__global__ void __launch_bounds__(SK_RCH) k_sk_reduce(const __grid_constant__ SkBatch bt, const z64 *__restrict__ part,
                                                      z64 *__restrict__ C, int accumulate, double alpha) {
    __shared__ unsigned char s_js[SK_MAXP];
    constexpr int nch = SK_T * SK_T / SK_RCH;
    const int64_t T = blockIdx.x / nch;
    const int e = (int)(blockIdx.x % nch) * SK_RCH + threadIdx.x;
    int g = 0;
    for (int lo = 0, hi = bt.ng - 1; lo <= hi;) {   // last problem with tile_off[g] <= T
        const int mid = (lo + hi) >> 1;
        if (bt.tile_off[mid] <= T) { g = mid; lo = mid + 1; } else hi = mid - 1;
    }
    const GemmDesc &d = bt.d[g];
    const int64_t t = T - bt.tile_off[g], ks = bt.ksteps[g];
    const int64_t tu0 = bt.unit_off[g] + t * ks;
    const int64_t cf = sk_owner(tu0, bt), cl = sk_owner(tu0 + ks - 1, bt);
    if (cf == cl) return;   // a whole tile, written by its CTA (uniform over the CTA)
    const int np = (int)(cl - cf + 1);
    for (int q = threadIdx.x; q < np && q < SK_MAXP; q += blockDim.x) s_js[q] = (unsigned char)sk_slot(cf + q, tu0, bt);
    __syncthreads();
    const int64_t ntn = (d.N + SK_T - 1) / SK_T;
    const int64_t r = (t / ntn) * SK_T + e / SK_T, col = (t % ntn) * SK_T + e % SK_T;
    if (r >= d.M || col >= d.N) return;
    z64 v(0, 0);
    for (int64_t cc = cf; cc <= cl; ++cc) {
        const int q = (int)(cc - cf);
        const int jslot = q < SK_MAXP ? s_js[q] : sk_slot(cc, tu0, bt);
        const double2 pv = __ldcg(reinterpret_cast<const double2 *>(part) + (2 * cc + jslot) * (SK_T * SK_T) + e);
        v += z64(pv.x, pv.y);
    }
    z64 *pc = C + d.c_off + r * d.ldc + col;
    v = alpha * v;
    if (accumulate) *pc += v;
    else *pc = v;
}

__global__ void __launch_bounds__(256) k_gemm_sk(const __grid_constant__ SkBatch bt, int opA, int opB,
                                                 const z64 *__restrict__ A, const z64 *__restrict__ B,
                                                 z64 *__restrict__ C, z64 *__restrict__ part,
                                                 unsigned *__restrict__ tile_cnt, int accumulate, double alpha) {
    __shared__ int s_last;
    __shared__ z64 As[SK_K][SK_T + 1];
    __shared__ z64 Bs[SK_K][SK_T + 1];
    __shared__ double Ass[SK_K][SK_T + 1];   // a_re + a_im
    __shared__ double Bss[SK_K][SK_T + 1];   // b_re + b_im
    const int64_t c = blockIdx.x;
    const int64_t u0 = sk_first(c, bt), u1 = sk_first(c + 1, bt);
    const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
    const bool rowA = (opA == 0 || opA == 3), rowB = (opB == 0 || opB == 3);
    for (int64_t u = u0; u < u1;) {
        const int g = sk_group(bt, u);
        const GemmDesc &d = bt.d[g];
        const int64_t ks = bt.ksteps[g];
        const int64_t local = u - bt.unit_off[g];
        const int64_t t = local / ks, kk0 = local % ks;
        const int64_t seg_end = min(u1, bt.unit_off[g] + (t + 1) * ks);
        const int64_t ntn = (d.N + SK_T - 1) / SK_T;
        const int64_t m0 = (t / ntn) * SK_T, n0 = (t % ntn) * SK_T;
        double t1[2][2], t2[2][2], t3[2][2];
        for (int i = 0; i < 2; ++i)
            for (int j = 0; j < 2; ++j) t1[i][j] = t2[i][j] = t3[i][j] = 0.0;
        for (int64_t kk = kk0; kk < kk0 + (seg_end - u); ++kk) {
            const int64_t k0 = kk * SK_K;
            for (int idx = threadIdx.x; idx < SK_T * SK_K; idx += 256) {
                const int mm = rowA ? idx / SK_K : idx % SK_T;
                const int kq = rowA ? idx % SK_K : idx / SK_T;
                const z64 va = load_op(A, d.a_off, d.lda, m0 + mm, k0 + kq, d.M, d.K, opA);
                As[kq][mm] = va;
                Ass[kq][mm] = va.re + va.im;
                const int kb = rowB ? idx / SK_T : idx % SK_K;
                const int nn = rowB ? idx % SK_T : idx / SK_K;
                const z64 vb = load_op(B, d.b_off, d.ldb, k0 + kb, n0 + nn, d.K, d.N, opB);
                Bs[kb][nn] = vb;
                Bss[kb][nn] = vb.re + vb.im;
            }
            __syncthreads();
#pragma unroll
            for (int kq = 0; kq < SK_K; ++kq) {
                const z64 a[2] = {As[kq][ty], As[kq][ty + 16]}, b[2] = {Bs[kq][tx], Bs[kq][tx + 16]};
                const double sa[2] = {Ass[kq][ty], Ass[kq][ty + 16]}, sb[2] = {Bss[kq][tx], Bss[kq][tx + 16]};
#pragma unroll
                for (int i = 0; i < 2; ++i)
#pragma unroll
                    for (int j = 0; j < 2; ++j) {
                        t1[i][j] = fma(a[i].re, b[j].re, t1[i][j]);
                        t2[i][j] = fma(a[i].im, b[j].im, t2[i][j]);
                        t3[i][j] = fma(sa[i], sb[j], t3[i][j]);
                    }
            }
            __syncthreads();
        }
        z64 acc[2][2];
        for (int i = 0; i < 2; ++i)
            for (int j = 0; j < 2; ++j) acc[i][j] = z64(t1[i][j] - t2[i][j], t3[i][j] - t1[i][j] - t2[i][j]);
        const bool whole = (kk0 == 0 && seg_end - u == ks);
        if (whole) {
            for (int i = 0; i < 2; ++i) {
                const int64_t r = m0 + ty + 16 * i;
                for (int j = 0; j < 2; ++j) {
                    const int64_t col = n0 + tx + 16 * j;
                    if (r < d.M && col < d.N) {
                        z64 *pc = C + d.c_off + r * d.ldc + col;
                        const z64 v = alpha * acc[i][j];
                        if (accumulate) *pc += v;
                        else *pc = v;
                    }
                }
            }
        } else {
            z64 *slot = part + (2 * c + (u == u0 ? 0 : 1)) * (SK_T * SK_T);
            for (int i = 0; i < 2; ++i)
                for (int j = 0; j < 2; ++j) slot[(ty + 16 * i) * SK_T + tx + 16 * j] = acc[i][j];
            if (bt.defer) {   // summed by k_sk_reduce after this launch
                u = seg_end;
                continue;
            }
            // the tile's CTAs are the owners of its first to its last unit
            const int64_t tu0 = bt.unit_off[g] + t * ks, tu1 = tu0 + ks;
            const int64_t cf = sk_owner(tu0, bt), cl = sk_owner(tu1 - 1, bt);
            __threadfence();   // this CTA's slot before its count
            __syncthreads();
            if (threadIdx.x == 0) {
                const unsigned prev = atomicAdd(&tile_cnt[bt.tile_off[g] + t], 1u);
                s_last = prev == (unsigned)(cl - cf) ? 1 : 0;
                __threadfence();
            }
            __syncthreads();
            if (s_last) sk_sum_tile(bt, g, m0, n0, tu0, cf, cl, part, C, accumulate, alpha);
        }
        u = seg_end;
    }
}

// ------------------------------------------------------ batched LU solve
// Gaussian elimination with partial pivoting on [Z | V], then backward
// substitution; one block per system.
__global__ void __launch_bounds__(256) k_lu_solve(const int64_t *__restrict__ zoff, const int64_t *__restrict__ voff,
                                                  const int *__restrict__ nsz, int s, z64 *__restrict__ Zall,
                                                  z64 *__restrict__ Vall, int *__restrict__ info) {
    const int b = blockIdx.x;
    const int n = nsz[b];
    z64 *Z = Zall + zoff[b];
    z64 *V = Vall + voff[b];
    __shared__ int piv;
    __shared__ z64 pinv;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int k = 0; k < n; ++k) {
        // pivot search by warp 0: largest |Z[i][k]|^2 (first on ties), bit patterns compared as integers
        if (warp == 0) {
            long long best = -1;
            int bi = k;
            for (int i = k + lane; i < n; i += 32) {
                const long long v = __double_as_longlong(norm2(Z[(int64_t)i * n + k]));
                if (v > best) {
                    best = v;
                    bi = i;
                }
            }
            for (int o = 16; o > 0; o >>= 1) {
                const long long ov = __shfl_xor_sync(0xffffffffu, best, o);
                const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
                if (ov > best || (ov == best && oi < bi)) {
                    best = ov;
                    bi = oi;
                }
            }
            if (lane == 0) {
                piv = bi;
                if (best <= 0) info[b] = 1;
            }
        }
        __syncthreads();
        const int p = piv;
        if (p != k) {
            for (int j = threadIdx.x; j < n; j += blockDim.x) {
                z64 t = Z[(int64_t)k * n + j];
                Z[(int64_t)k * n + j] = Z[(int64_t)p * n + j];
                Z[(int64_t)p * n + j] = t;
            }
            for (int j = threadIdx.x; j < s; j += blockDim.x) {
                z64 t = V[(int64_t)k * s + j];
                V[(int64_t)k * s + j] = V[(int64_t)p * s + j];
                V[(int64_t)p * s + j] = t;
            }
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            z64 d = Z[(int64_t)k * n + k];
            pinv = (norm2(d) > 0.0) ? cdiv(z64(1, 0), d) : z64(0, 0);
        }
        __syncthreads();
        // multipliers once per row, kept in column k
        for (int i = k + 1 + threadIdx.x; i < n; i += blockDim.x) Z[(int64_t)i * n + k] = Z[(int64_t)i * n + k] * pinv;
        __syncthreads();
        // eliminate below
        const int rows = n - k - 1;
        const int wcols = (n - k - 1) + s;
        for (int64_t idx = threadIdx.x; idx < (int64_t)rows * wcols; idx += blockDim.x) {
            int i = k + 1 + (int)(idx / wcols);
            int c = (int)(idx % wcols);
            const z64 l = Z[(int64_t)i * n + k];
            if (c < n - k - 1) {
                int j = k + 1 + c;
                Z[(int64_t)i * n + j] -= l * Z[(int64_t)k * n + j];
            } else {
                int j = c - (n - k - 1);
                V[(int64_t)i * s + j] -= l * V[(int64_t)k * s + j];
            }
        }
        __syncthreads();
    }
    // backward substitution, column oriented
    for (int k = n - 1; k >= 0; --k) {
        if (threadIdx.x == 0) {
            const z64 d = Z[(int64_t)k * n + k];
            pinv = (norm2(d) > 0.0) ? cdiv(z64(1, 0), d) : z64(0, 0);
        }
        __syncthreads();
        const z64 dinv = pinv;
        for (int j = threadIdx.x; j < s; j += blockDim.x) V[(int64_t)k * s + j] = V[(int64_t)k * s + j] * dinv;
        __syncthreads();
        for (int64_t idx = threadIdx.x; idx < (int64_t)k * s; idx += blockDim.x) {
            int i = (int)(idx / s), j = (int)(idx % s);
            V[(int64_t)i * s + j] -= Z[(int64_t)i * n + k] * V[(int64_t)k * s + j];
        }
        __syncthreads();
    }
}

// ---------------------------------------------- one-sided Jacobi SVD
// X (s x s, column-major, overwritten by U Sigma) and V (s x s, column-major).
// Round-robin pairing over n2 = s rounded up to even; disjoint pairs of a
// round are processed by different warps.  Stops after a sweep without any
// rotation, or after 60 sweeps (info = 2).
// One cluster of JS_CL CTAs per matrix: the s/2 column pairs of a round are
// spread over the cluster's warps (one pair per warp), the columns stay in
// global memory (read through L2 only, since other SMs write them), and the
// rounds are separated by a bounded cluster synchronisation.  Every CTA finds
// the same largest squared column norm and the same "anything rotated" answer
// (flags exchanged through distributed shared memory), so all CTAs run the
// same number of rounds and sweeps.  info[mat] = 2: no convergence in 60
// sweeps; 1: a cluster synchronisation expired.
constexpr int JS_CL = 8;

__device__ __forceinline__ double norm2d(double2 a) { return a.x * a.x + a.y * a.y; }

__global__ void __cluster_dims__(JS_CL, 1, 1) __launch_bounds__(256)
    k_jacobi_svd(int s, z64 *__restrict__ Xall, z64 *__restrict__ Vall, double *__restrict__ sig,
                 int *__restrict__ info, double tol, double keep) {
    cg::cluster_group cl = cg::this_cluster();
    const int me = (int)cl.block_rank(), mat = blockIdx.x / JS_CL;
    z64 *X = Xall + (int64_t)mat * s * s;
    z64 *V = Vall + (int64_t)mat * s * s;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int gw = me * nw + warp, ngw = JS_CL * nw;
    __shared__ uint64_t cbar[2];
    __shared__ int s_abort, rot_local, rotflag[JS_CL];
    __shared__ double s_wmax[32], s_big;
    for (int64_t i = (int64_t)me * blockDim.x + threadIdx.x; i < (int64_t)s * s; i += (int64_t)JS_CL * blockDim.x)
        V[i] = z64((i % s) == (i / s) ? 1.0 : 0.0, 0.0);
    if (threadIdx.x == 0) {
        cl_bar_init(cbar, JS_CL);
        s_abort = 0;
    }
    __syncthreads();
    cl.sync();   // barriers initialised and V set in every CTA (unconditional)
    const int n2 = s + (s & 1);
    int step = 0;   // cluster synchronisation count
    bool ok = true;
    int sweep = 0;
    for (; sweep < 60; ++sweep) {
        // largest squared column norm: a pair whose coupling is below f times it is
        // left alone, f = max(tol^2, (1e-5 keep)^2) with keep the relative size of the
        // smallest singular value the caller keeps.  Below tol^2 both columns are at
        // the rounding level of the largest; below (1e-5 keep)^2 both columns are far
        // below every kept singular value (sigma >= keep sigma_1), which such a
        // coupling turns by at most 1e-10: rotating them would only sort directions
        // that are discarded.  Every pair above f is rotated to the relative
        // criterion, so the kept singular values and vectors keep full accuracy (a
        // floor of tol |x|max^2 left pairs of columns near 1e-7 sigma_1 coupled and
        // their singular values wrong at their own size)
        double mx = 0.0;
        for (int i = warp; i < s; i += nw) {
            double al = 0;
            for (int r = lane; r < s; r += 32) al += norm2d(__ldcg(reinterpret_cast<const double2 *>(X) + (int64_t)i * s + r));
            for (int o = 16; o > 0; o >>= 1) al += __shfl_xor_sync(0xffffffffu, al, o);
            mx = fmax(mx, al);
        }
        if (lane == 0) s_wmax[warp] = mx;
        if (threadIdx.x == 0) rot_local = 0;
        __syncthreads();
        if (threadIdx.x == 0) {
            double bmax = 0.0;
            for (int w = 0; w < nw; ++w) bmax = fmax(bmax, s_wmax[w]);
            s_big = bmax;
        }
        __syncthreads();
        const double floor_abs = fmax(tol * tol, 1e-10 * keep * keep) * s_big;
        for (int round = 0; round < n2 - 1 && ok; ++round) {
            for (int pr = gw; pr < n2 / 2; pr += ngw) {
                // round-robin: position 0 fixed, others rotate
                int a = (pr == 0) ? 0 : 1 + (pr - 1 + round) % (n2 - 1);
                int b = 1 + (n2 - 2 - pr + round) % (n2 - 1);
                int i = min(a, b), j = max(a, b);
                if (j >= s) continue;   // dummy column of odd sizes
                z64 *xi = X + (int64_t)i * s, *xj = X + (int64_t)j * s;
                double al = 0, be = 0;
                z64 ga(0, 0);
                for (int r = lane; r < s; r += 32) {
                    const double2 u2 = __ldcg(reinterpret_cast<const double2 *>(xi) + r);
                    const double2 v2 = __ldcg(reinterpret_cast<const double2 *>(xj) + r);
                    const z64 u(u2.x, u2.y), v(v2.x, v2.y);
                    al += norm2(u);
                    be += norm2(v);
                    cfmaconj(ga, u, v);
                }
                for (int o = 16; o > 0; o >>= 1) {
                    al += __shfl_xor_sync(0xffffffffu, al, o);
                    be += __shfl_xor_sync(0xffffffffu, be, o);
                    ga.re += __shfl_xor_sync(0xffffffffu, ga.re, o);
                    ga.im += __shfl_xor_sync(0xffffffffu, ga.im, o);
                }
                double ag = sqrt(norm2(ga));
                if (ag <= tol * sqrt(al * be) || ag <= floor_abs || ag == 0.0) continue;
                if (lane == 0) rot_local = 1;
                double zeta = (be - al) / (2.0 * ag);
                double t = 1.0 / (zeta + copysign(sqrt(1.0 + zeta * zeta), zeta));
                double c = 1.0 / sqrt(1.0 + t * t), sn = c * t;
                z64 e(ga.re / ag, ga.im / ag);   // e^{i phi}
                z64 sem = sn * conj(e), sep = sn * e;
                z64 *vi = V + (int64_t)i * s, *vj = V + (int64_t)j * s;
                for (int r = lane; r < s; r += 32) {
                    const double2 u2 = __ldcg(reinterpret_cast<const double2 *>(xi) + r);
                    const double2 v2 = __ldcg(reinterpret_cast<const double2 *>(xj) + r);
                    const z64 u(u2.x, u2.y), v(v2.x, v2.y);
                    xi[r] = c * u - sem * v;
                    xj[r] = sep * u + c * v;
                    const double2 p2 = __ldcg(reinterpret_cast<const double2 *>(vi) + r);
                    const double2 q2 = __ldcg(reinterpret_cast<const double2 *>(vj) + r);
                    const z64 vu(p2.x, p2.y), vv(q2.x, q2.y);
                    vi[r] = c * vu - sem * vv;
                    vj[r] = sep * vu + c * vv;
                }
            }
            ok = cl_sync(cbar, step++, JS_CL, &s_abort, info + mat);
        }
        if (!ok) break;
        // has any CTA rotated in this sweep?  (flags to every CTA, then one synchronisation)
        if (threadIdx.x < JS_CL) *cl.map_shared_rank(&rotflag[me], threadIdx.x) = rot_local;
        if (!(ok = cl_sync(cbar, step++, JS_CL, &s_abort, info + mat))) break;
        int any = 0;
        for (int r = 0; r < JS_CL; ++r) any |= rotflag[r];
        if (!any) break;
    }
    if (ok && me == 0 && threadIdx.x == 0 && sweep >= 60) info[mat] = 2;
    for (int i = gw; i < s; i += ngw) {
        double al = 0;
        for (int r = lane; r < s; r += 32)
            al += norm2d(__ldcg(reinterpret_cast<const double2 *>(X) + (int64_t)i * s + r));
        for (int o = 16; o > 0; o >>= 1) al += __shfl_xor_sync(0xffffffffu, al, o);
        if (lane == 0) sig[(int64_t)mat * s + i] = sqrt(al);
    }
    cl.sync();   // no CTA leaves while another may still write into its shared memory
}

// ------------------------------------------------- Gauss-Jordan inverse
// In-place Gauss-Jordan ("sweep") with row interchanges and ping-pong
// buffers.  With O the matrix after swapping rows k and p, pinv = 1 / O[k][k],
// f_i = O[i][k] pinv:
//   new[i][j] = O[i][j] - f_i O[k][j]   (i != k, j != k)
//   new[i][k] = -f_i,  new[k][j] = O[k][j] pinv,  new[k][k] = pinv.
// After n sweeps the matrix is the inverse of the row-permuted input; undoing
// the interchanges on the columns, last first, gives A^{-1}.  Each sweep also
// finds the pivot of the next column (largest |.|^2 below the diagonal, lowest
// row on ties) through a 64-bit atomicMax on key = (|v|^2 bits, ~row).
constexpr int GJ_IBITS = 20;
constexpr unsigned long long GJ_IMASK = (1ull << GJ_IBITS) - 1;

__device__ __forceinline__ unsigned long long gj_key(double v2, int row) {
    if (!(v2 > 0.0)) return 0ull;
    const unsigned long long b = (unsigned long long)__double_as_longlong(v2);
    return ((b >> GJ_IBITS) << GJ_IBITS) | (GJ_IMASK - (unsigned long long)row);
}

// block-wide max of a key, then one atomicMax
__device__ __forceinline__ void gj_push_key(unsigned long long key, unsigned long long *dst) {
    __shared__ unsigned long long s_k[32];
    const int t = threadIdx.y * blockDim.x + threadIdx.x, lane = t & 31, w = t >> 5;
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long other = __shfl_xor_sync(0xffffffffu, key, o);
        key = other > key ? other : key;
    }
    if (lane == 0) s_k[w] = key;
    __syncthreads();
    if (t == 0) {
        unsigned long long best = 0;
        for (int i = 0; i < (int)(blockDim.x * blockDim.y + 31) / 32; ++i) best = s_k[i] > best ? s_k[i] : best;
        if (best) atomicMax(dst, best);
    }
}

// copy A into the first buffer and find the pivot of column 0
__global__ void __launch_bounds__(256) k_gj_init(int n, const z64 *__restrict__ A, z64 *__restrict__ X,
                                                 unsigned long long *__restrict__ keys) {
    // matrix blockIdx.y of the batch
    A += (int64_t)blockIdx.y * n * n;
    X += (int64_t)blockIdx.y * n * n;
    keys += (int64_t)blockIdx.y * n;
    unsigned long long key = 0;
    for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < (int64_t)n * n;
         idx += (int64_t)gridDim.x * blockDim.x) {
        const z64 v = A[idx];
        X[idx] = v;
        if (idx % n == 0) {
            const unsigned long long kk = gj_key(norm2(v), (int)(idx / n));
            key = kk > key ? kk : key;
        }
    }
    gj_push_key(key, &keys[0]);
}

// All n sweeps in one cooperative launch: persistent CTAs stride over the
// 32 x 32 tiles of every matrix of the batch and meet at a grid barrier after
// each sweep (a counter and a generation word in global memory; the wait gives
// up after one second, sets *err and ends the kernel).  The ping-pong buffers
// and the pivot keys are written by other SMs, so they are read through L2
// only.  16 x 16 threads per CTA, each 2 rows x 2 columns of a 32 x 32 tile.
constexpr int GJ_MAXB = 4;   // matrices per batch (pivot data cached per CTA)

__device__ __forceinline__ bool gj_grid_sync(unsigned *cnt, unsigned *gen, unsigned nblocks, unsigned &g, int *abort_flag,
                                             int *err) {
    __syncthreads();
    if (threadIdx.x == 0 && threadIdx.y == 0) {
        __threadfence();   // this CTA's writes before the arrival
        const unsigned my = g;
        if (atomicAdd(cnt, 1u) == nblocks - 1) {
            atomicExch(cnt, 0u);
            __threadfence();
            atomicExch(gen, my + 1);
        } else {
            uint64_t t0;
            asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t0));
            for (;;) {   // acquire loads: the waiting CTAs do not queue atomics on the line
                unsigned cur;
                asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(cur) : "l"(gen) : "memory");
                if (cur != my) break;
                uint64_t t;
                asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
                if (t - t0 > 1000000000ull) {
                    *abort_flag = 1;
                    atomicExch(err, 1);
                    break;
                }
                __nanosleep(20);
            }
        }
        __threadfence();   // the others' writes after it
    }
    ++g;
    __syncthreads();
    return *(volatile int *)abort_flag == 0;
}

__global__ void __launch_bounds__(256) k_gj_persistent(int n, int nbatch, z64 *__restrict__ b0, z64 *__restrict__ b1,
                                                       unsigned long long *__restrict__ keys,
                                                       int *__restrict__ pivrow, int *__restrict__ info,
                                                       unsigned *__restrict__ bar, int *__restrict__ err) {
    __shared__ z64 s_pinv[GJ_MAXB];
    __shared__ int s_p[GJ_MAXB];
    __shared__ int s_abort;
    const int tn = (n + 31) / 32;
    const int64_t nn = (int64_t)n * n;
    const int ntiles = nbatch * tn * tn;
    if (threadIdx.x == 0 && threadIdx.y == 0) s_abort = 0;
    unsigned g = 0;
    for (int k = 0; k < n; ++k) {
        const z64 *Ain = (k & 1) ? b1 : b0;
        z64 *Aout = (k & 1) ? b0 : b1;
        if (threadIdx.y == 0 && threadIdx.x < nbatch) {   // pivot of column k of every matrix
            const int mb = threadIdx.x;
            const unsigned long long key = __ldcg(keys + (int64_t)mb * n + k);
            int p = k;
            z64 pinv(0, 0);
            if (key == 0ull) {
                if (blockIdx.x == 0) info[0] = 1;   // no non-zero pivot in column k
            } else {
                p = (int)(GJ_IMASK - (key & GJ_IMASK));
                const double2 v = __ldcg(reinterpret_cast<const double2 *>(Ain + mb * nn) + (int64_t)p * n + k);
                pinv = cdiv(z64(1, 0), z64(v.x, v.y));
            }
            if (blockIdx.x == 0) pivrow[(int64_t)mb * n + k] = p;
            s_p[mb] = p;
            s_pinv[mb] = pinv;
        }
        __syncthreads();
        for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
            const int mb = tile / (tn * tn), rem = tile - mb * tn * tn, by = rem / tn, bx = rem - by * tn;
            const z64 *A = Ain + mb * nn;
            z64 *O = Aout + mb * nn;
            const int p = s_p[mb];
            const z64 pinv = s_pinv[mb];
            const int j0 = bx * 32 + threadIdx.x, i0 = by * 32 + threadIdx.y;
            z64 r[2];
#pragma unroll
            for (int c = 0; c < 2; ++c) {
                const int j = j0 + 16 * c;
                const double2 v = j < n ? __ldcg(reinterpret_cast<const double2 *>(A) + (int64_t)p * n + j)
                                        : make_double2(0.0, 0.0);
                r[c] = z64(v.x, v.y);   // O[k][j]
            }
            unsigned long long key = 0;
#pragma unroll
            for (int rr = 0; rr < 2; ++rr) {
                const int i = i0 + 16 * rr;
                if (i >= n) continue;
                z64 *out = O + (int64_t)i * n;
                if (i == k) {
#pragma unroll
                    for (int c = 0; c < 2; ++c) {
                        const int j = j0 + 16 * c;
                        if (j < n) out[j] = j == k ? pinv : r[c] * pinv;
                    }
                } else {
                    const int src = i == p ? k : i;
                    const double2 *in = reinterpret_cast<const double2 *>(A + (int64_t)src * n);
                    const double2 fk = __ldcg(in + k);
                    const z64 f = z64(fk.x, fk.y) * pinv;
#pragma unroll
                    for (int c = 0; c < 2; ++c) {
                        const int j = j0 + 16 * c;
                        if (j >= n) continue;
                        const double2 a = __ldcg(in + j);
                        const z64 v = j == k ? -f : z64(a.x, a.y) - f * r[c];
                        out[j] = v;
                        if (j == k + 1 && i > k) {
                            const unsigned long long kk = gj_key(norm2(v), i);
                            key = kk > key ? kk : key;
                        }
                    }
                }
            }
            if (k + 1 < n && (k + 1) / 32 == bx) gj_push_key(key, keys + (int64_t)mb * n + k + 1);
        }
        if (!gj_grid_sync(bar, bar + 1, gridDim.x, g, &s_abort, err)) return;
    }
}

// column order of the result: undo the interchanges, last first (one thread)
__global__ void k_gj_perm(int n, const int *__restrict__ pivrow, int *__restrict__ src) {
    if (threadIdx.x != 0) return;
    pivrow += (int64_t)blockIdx.x * n;   // one block per matrix of the batch
    src += (int64_t)blockIdx.x * n;
    for (int j = 0; j < n; ++j) src[j] = j;
    for (int k = n - 1; k >= 0; --k) {
        const int p = pivrow[k], t = src[k];
        src[k] = src[p];
        src[p] = t;
    }
}

__global__ void k_gj_unpack(int n, const z64 *__restrict__ X, const int *__restrict__ src, z64 *__restrict__ inv) {
    X += (int64_t)blockIdx.y * n * n;
    inv += (int64_t)blockIdx.y * n * n;
    src += (int64_t)blockIdx.y * n;
    for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < (int64_t)n * n;
         idx += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = idx / n, j = idx % n;
        inv[idx] = X[i * n + src[j]];
    }
}

__global__ void k_to32(const z64 *__restrict__ s, c32 *__restrict__ d, int64_t n) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) d[i] = c32((float)s[i].re, (float)s[i].im);
}
__global__ void k_to64(const c32 *__restrict__ s, z64 *__restrict__ d, int64_t n) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) d[i] = z64(s[i].re, s[i].im);
}

void gemm_sk(const std::vector<GemmDesc> &g, int opA, int opB, const z64 *A, const z64 *B, z64 *C, bool accumulate,
             cudaStream_t st, double alpha) {
    static std::atomic<int> s_grid[64];   // CTAs per launch, per device (zero: not yet queried)
    int dev = 0;
    CBFM_CUDA(cudaGetDevice(&dev));
    int G0 = dev < 64 ? s_grid[dev].load(std::memory_order_relaxed) : 0;
    if (G0 == 0) {
        int nsm = 0, occ = 0;
        CBFM_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
        CBFM_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_gemm_sk, 256, 0));
        // two CTAs per SM: one keeps the FP64 pipe busy while the other
        // stages its next K-step; more would only cut more tiles
        G0 = std::max(1, nsm * std::max(1, std::min(occ, 2)));
        if (dev < 64) s_grid[dev].store(G0, std::memory_order_relaxed);
    }
    for (size_t g0 = 0; g0 < g.size(); g0 += GB_MAXG) {
        SkBatch bt;
        bt.ng = (int)std::min<size_t>(GB_MAXG, g.size() - g0);
        bt.unit_off[0] = bt.tile_off[0] = 0;
        for (int i = 0; i < bt.ng; ++i) {
            const GemmDesc &d = g[g0 + i];
            bt.d[i] = d;
            const int64_t tiles = (d.M > 0 && d.N > 0) ? ((d.M + SK_T - 1) / SK_T) * ((d.N + SK_T - 1) / SK_T) : 0;
            bt.ksteps[i] = std::max<int64_t>(1, (d.K + SK_K - 1) / SK_K);   // K = 0: one step of zeros
            bt.unit_off[i + 1] = bt.unit_off[i] + tiles * bt.ksteps[i];
            bt.tile_off[i + 1] = bt.tile_off[i] + tiles;
        }
        bt.U = bt.unit_off[bt.ng];
        if (bt.U == 0) continue;
        bt.G = (int)std::min<int64_t>(G0, bt.U);
        // few tiles for many CTAs (a Gram of few columns over a long K): each tile is cut
        // into ~G / tiles pieces, too many for one CTA to add; a second launch spreads
        // the sums over many CTAs
        const int64_t ntiles = bt.tile_off[bt.ng];
        bt.defer = (int64_t)bt.G > 2 * ntiles ? 1 : 0;
        // partial-sum slots (two per CTA) and one arrival counter per tile, zeroed
        const size_t slot_bytes = sizeof(z64) * 2 * (size_t)bt.G * SK_T * SK_T;
        const size_t cnt_bytes = sizeof(unsigned) * (size_t)ntiles;
        unsigned char *scratch = nullptr;
        CBFM_CUDA(cudaMallocAsync((void **)&scratch, slot_bytes + cnt_bytes, st));
        z64 *part = reinterpret_cast<z64 *>(scratch);
        unsigned *tile_cnt = reinterpret_cast<unsigned *>(scratch + slot_bytes);
        if (!bt.defer) CBFM_CUDA(cudaMemsetAsync(tile_cnt, 0, cnt_bytes, st));
        {
            ProfScope ps_("k_gemm_z64", st);
            ProfScope site_(g_gemm_site ? g_gemm_site : "site:other", st);
            k_gemm_sk<<<bt.G, 256, 0, st>>>(bt, opA, opB, A, B, C, part, tile_cnt, accumulate ? 1 : 0, alpha);
            launched("k_gemm_sk");
            if (bt.defer) {
                k_sk_reduce<<<(unsigned)(ntiles * (SK_T * SK_T / SK_RCH)), SK_RCH, 0, st>>>(bt, part, C,
                                                                                             accumulate ? 1 : 0, alpha);
                launched("k_sk_reduce");
            }
        }
        CBFM_CUDA(cudaFreeAsync(scratch, st));
    }
}

// ------------------------------------------------ blocked Gauss-Jordan
// Inverse by Gauss-Jordan with GJB x GJB block pivots and no row exchanges
// between blocks:  with D = A_kk^{-1},
//   A_kj <- D A_kj,  A_ij <- A_ij - A_ik D A_kj,  A_ik <- -A_ik D,  A_kk <- D.
// The products are the FP64 stream-K GEMMs; only the diagonal-block
// inverses are serial.  Used where the block pivots are safe (checked), else
// the pivoted sweep above.
constexpr int GJB = 16;   // small diagonal blocks: their serial inverses are cheap, the GEMMs carry the work

// column panel C = A[:, k0:k0+b] (n x b, ld b) and row panel Rw = A[k0:k0+b, :] (b x n, ld n), per matrix
__global__ void k_gjb_panels(int n, int k0, int b, const z64 *__restrict__ A, z64 *__restrict__ C,
                             z64 *__restrict__ Rw) {
    const int t = blockIdx.y;
    A += (int64_t)t * n * n;
    C += (int64_t)t * n * b;
    Rw += (int64_t)t * b * n;
    for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < (int64_t)n * b;
         idx += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = idx / b, j = idx % b;
        C[idx] = A[i * n + k0 + j];
        const int64_t r = idx / n, c = idx % n;
        Rw[idx] = A[(k0 + r) * n + c];
    }
}

// D = inverse of the b x b diagonal block Rw[:, k0:k0+b] (ld n), one CTA per
// matrix: Gauss-Jordan with partial pivoting inside the block (row exchanges
// undone on the columns when D is stored).  A pivot below 1e-13 of the
// block's largest entry sets *flag.  The column block k of A is zeroed (it is
// accumulated into next; its old values are in the panel copy).
//
// Each step is two phases over ping-pong copies of the block: warp 0 finds the
// pivot, inverts it and scales the pivot row (the new row k); then every
// entry of the other rows is updated from the old copy with four FMAs.  FP64
// warp instructions are the cost here (each holds a sub-partition's FP64 pipe
// for ~64 clocks whatever its active lanes), so the pivot-row work is done
// once, by one warp, instead of once per entry.
// The elimination itself, by the GJB x GJB threads of a CTA: blk[r * ld + c]
// (r, c < b) is the block, read through L2 (other SMs may have written it).
__device__ void gjb_block_inverse(int b, const z64 *__restrict__ blk, int64_t ld, z64 *__restrict__ D,
                                  int *__restrict__ flag) {
    __shared__ z64 buf[2][GJB][GJB + 1];
    __shared__ z64 nrow[GJB];   // row k of the next copy: pivot row times 1/pivot, 1/pivot at k
    __shared__ z64 s_pinv;
    __shared__ int perm[GJB];
    __shared__ int s_p;
    __shared__ double s_amax;
    const int tid = threadIdx.x, lane = tid & 31;
    const int r = tid / GJB, c = tid % GJB;
    if (r < b && c < b) {
        const double2 v = __ldcg(reinterpret_cast<const double2 *>(blk + (int64_t)r * ld + c));
        buf[0][r][c] = z64(v.x, v.y);
    } else {
        buf[0][r][c] = z64(0.0, 0.0);
    }
    __syncthreads();
    if (tid < 32) {
        double m = 0.0;
        for (int idx = lane; idx < b * b; idx += 32) m = fmax(m, norm2(buf[0][idx / b][idx % b]));
        for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
        if (lane == 0) s_amax = m;
    }
    __syncthreads();
    int cur = 0;
    for (int k = 0; k < b; ++k) {
        const z64(*X)[GJB + 1] = buf[cur];
        z64(*Y)[GJB + 1] = buf[cur ^ 1];
        if (tid < 32) {   // pivot: largest |X[r][k]|^2, r >= k (first on ties); bit patterns of
                          // non-negative doubles order as integers
            long long bv = -1;
            int bp = k;
            if (lane >= k && lane < b) {
                bv = __double_as_longlong(norm2(X[lane][k]));
                bp = lane;
            }
            for (int o = 16; o > 0; o >>= 1) {
                const long long ov = __shfl_xor_sync(0xffffffffu, bv, o);
                const int op = __shfl_xor_sync(0xffffffffu, bp, o);
                if (ov > bv || (ov == bv && op < bp)) {
                    bv = ov;
                    bp = op;
                }
            }
            z64 pinv(0.0, 0.0);
            if (lane == 0) {
                const double d = __longlong_as_double(bv);
                if (!(d > 1e-26 * s_amax)) atomicExch(flag, 1);   // |pivot| < 1e-13 max|entry|
                const z64 piv = X[bp][k];
                const double id = d > 0.0 ? __drcp_rn(d) : 0.0;
                pinv = z64(piv.re * id, -piv.im * id);
                s_p = bp;
                s_pinv = pinv;
                perm[k] = bp;
            }
            pinv.re = __shfl_sync(0xffffffffu, pinv.re, 0);
            pinv.im = __shfl_sync(0xffffffffu, pinv.im, 0);
            if (lane < b) nrow[lane] = lane == k ? pinv : X[bp][lane] * pinv;
        }
        __syncthreads();
        const int p = s_p;
        if (r < b && c < b) {
            if (r == k) {
                Y[k][c] = nrow[c];
            } else {
                const int src = r == p ? k : r;   // rows k and p exchanged
                const z64 f = X[src][k];
                z64 v;
                if (c == k) {
                    v = -(f * s_pinv);
                } else {
                    v = X[src][c];
                    const z64 w = nrow[c];
                    v.re = fma(-f.re, w.re, v.re);
                    v.re = fma(f.im, w.im, v.re);
                    v.im = fma(-f.re, w.im, v.im);
                    v.im = fma(-f.im, w.re, v.im);
                }
                Y[r][c] = v;
            }
        }
        __syncthreads();
        cur ^= 1;
    }
    // undo the row exchanges as column exchanges, in reverse order: column j of
    // the inverse is column idx[j] of the eliminated block
    __shared__ int colsrc[GJB];
    if (tid == 0) {
        for (int j = 0; j < GJB; ++j) colsrc[j] = j;
        for (int k = b - 1; k >= 0; --k) {
            const int q = perm[k];
            const int u = colsrc[k];
            colsrc[k] = colsrc[q];
            colsrc[q] = u;
        }
    }
    __syncthreads();
    D[r * GJB + c] = (r < b && c < b) ? buf[cur][r][colsrc[c]] : z64(0.0, 0.0);
}

__global__ void __launch_bounds__(GJB * GJB) k_gjb_inv(int n, int k0, int b, const z64 *__restrict__ Rw,
                                                 z64 *__restrict__ D, int *__restrict__ flag,
                                                 z64 *__restrict__ A) {
    const int t = blockIdx.x;
    Rw += (int64_t)t * b * n;
    D += (int64_t)t * GJB * GJB;
    A += (int64_t)t * n * n;
    for (int idx = threadIdx.x; idx < n * b; idx += blockDim.x)
        A[(int64_t)(idx / b) * n + k0 + idx % b] = z64(0.0, 0.0);
    gjb_block_inverse(b, Rw + k0, n, D, flag);
}

// All block steps of the blocked Gauss-Jordan inverse in one cooperative
// launch (nbatch matrices, in place).  Before the first step CTA t inverts
// the first diagonal block of matrix t and every CTA copies its share of the
// first column block; then per block step K, two phases separated by the
// bounded grid barrier of k_gj_persistent:
//   (B) Rwp = D_K A[K, :] (b x n) by 16 x 8 tiles staged in shared memory;
//   (C) every 32 x 32 tile of A: A[K, K] = D_K, A[K, j] = Rwp[:, j],
//       A[i, K] = -C_K[i, :] D_K, A[i, j] -= C_K[i, :] Rwp[:, j] for i, j outside
//       K (complex products in three real multiplications: t1 = sum re re,
//       t2 = sum im im, t3 = sum (re + im)(re + im)); the owner of a tile that
//       holds columns of block K + 1 copies their new values into C_{K+1}.
// Look-ahead: CTA t copies block K + 1 of matrix t in phase B (before any
// update of this step), forms its updated values in phase C with the same
// arithmetic as the tile update (so the same bits) and inverts it into
// D_{K+1}, while the other CTAs update every tile: the serial inverse runs
// beside the update instead of between two barriers.  C and D are
// double-buffered by the parity of K; Sb holds, per matrix, the old block and
// its update.
// Buffers written by other SMs are read through L2.  *flag as k_gjb_inv.
__global__ void __launch_bounds__(256, 2) k_gjb_persistent(int n, int nbatch, z64 *__restrict__ A, z64 *__restrict__ Cb,
                                                            z64 *__restrict__ Rwp, z64 *__restrict__ Db,
                                                            z64 *__restrict__ Sb, int *__restrict__ flag,
                                                            unsigned *__restrict__ bar, int *__restrict__ err,
                                                            int *__restrict__ smids, unsigned *__restrict__ tilectr) {
    __shared__ double sC[3][32][GJB + 1];   // 32 rows of C: re, im, re + im
    __shared__ double sR[3][GJB][32 + 1];   // b rows of the right operand (Rwp, or D in the columns of K)
    __shared__ int s_abort, s_idle, s_tile;
    if (threadIdx.x == 0) s_abort = 0;
    unsigned smid;
    asm volatile("mov.u32 %0, %%smid;" : "=r"(smid));
    if (blockIdx.x < nbatch && threadIdx.x == 0) smids[blockIdx.x] = (int)smid;   // read after the first barrier
    unsigned g = 0;
    const int64_t nn = (int64_t)n * n;
    const int tn = (n + 31) / 32;
    const int64_t nthr = (int64_t)gridDim.x * blockDim.x;
    const int64_t gtid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t csz = (int64_t)nbatch * n * GJB, dsz = (int64_t)nbatch * GJB * GJB;
    const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
    auto ld2 = [](const z64 *p) {
        const double2 v = __ldcg(reinterpret_cast<const double2 *>(p));
        return z64(v.x, v.y);
    };
    // before the first step: C_0 and D_0
    {
        const int b = min(GJB, n);
        for (int64_t idx = gtid; idx < (int64_t)nbatch * n * b; idx += nthr) {
            const int t = (int)(idx / ((int64_t)n * b));
            const int64_t rem = idx - (int64_t)t * n * b, i = rem / b, l = rem - i * b;
            Cb[((int64_t)t * n + i) * GJB + l] = ld2(A + t * nn + i * n + l);
        }
        if (blockIdx.x < nbatch) gjb_block_inverse(b, A + blockIdx.x * nn, n, Db + (int64_t)blockIdx.x * GJB * GJB, flag);
        if (!gj_grid_sync(bar, bar + 1, gridDim.x, g, &s_abort, err)) return;
    }
    // a CTA that shares its SM with a look-ahead CTA takes no tiles, so that the
    // serial inverse has the SM's FP64 pipes to itself
    if (threadIdx.x == 0) {   // (with more than 4 CTAs per look-ahead CTA, so others remain for the tiles)
        int idle = 0;
        for (int t = 0; t < nbatch && blockIdx.x >= nbatch && (int)gridDim.x > 4 * nbatch; ++t)
            idle |= __ldcg(smids + t) == (int)smid;
        s_idle = idle;
    }
    __syncthreads();
    const bool idle = s_idle != 0;
    for (int k0 = 0, par = 0; k0 < n; k0 += GJB, par ^= 1) {
        const int b = min(GJB, n - k0);
        const int kn = k0 + GJB, bn = min(GJB, n - kn);   // block K + 1 (bn <= 0: none)
        const z64 *Ck = Cb + par * csz, *Dk = Db + par * dsz;
        z64 *Cn = Cb + (par ^ 1) * csz, *Dn = Db + (par ^ 1) * dsz;
        // (B): tiles of 16 rows x 8 columns, one output per thread of the first 128
        {
            const int tn8 = (n + 7) / 8;
            for (int tile = blockIdx.x; tile < nbatch * tn8; tile += gridDim.x) {
                const int t = tile / tn8, j0 = (tile - t * tn8) * 8;
                const z64 *At = A + t * nn, *Dt = Dk + (int64_t)t * GJB * GJB;
                __syncthreads();
                {   // D_K into sC[0..2][l][m], the row block tile into sR[0..2][m][c] (re, im, re + im)
                    const int l = threadIdx.x / 16, m = threadIdx.x % 16;
                    const z64 d = (l < b && m < b) ? ld2(Dt + l * GJB + m) : z64(0.0, 0.0);
                    sC[0][l][m] = d.re;
                    sC[1][l][m] = d.im;
                    sC[2][l][m] = d.re + d.im;
                    if (threadIdx.x < GJB * 8) {
                        const int mm = threadIdx.x / 8, c = threadIdx.x % 8, j = j0 + c;
                        const z64 v = (mm < b && j < n) ? ld2(At + (int64_t)(k0 + mm) * n + j) : z64(0.0, 0.0);
                        sR[0][mm][c] = v.re;
                        sR[1][mm][c] = v.im;
                        sR[2][mm][c] = v.re + v.im;
                    }
                }
                __syncthreads();
                if (threadIdx.x < GJB * 8) {
                    const int l = threadIdx.x / 8, c = threadIdx.x % 8, j = j0 + c;
                    if (l < b && j < n) {
                        double t1 = 0.0, t2 = 0.0, t3 = 0.0;
#pragma unroll
                        for (int m = 0; m < GJB; ++m) {
                            t1 = fma(sC[0][l][m], sR[0][m][c], t1);
                            t2 = fma(sC[1][l][m], sR[1][m][c], t2);
                            t3 = fma(sC[2][l][m], sR[2][m][c], t3);
                        }
                        Rwp[((int64_t)t * GJB + l) * n + j] = z64(t1 - t2, t3 - t1 - t2);
                    }
                }
            }
        }
        if (blockIdx.x < nbatch && bn > 0) {   // block K + 1 before this step's update
            const int r = threadIdx.x / GJB, c = threadIdx.x % GJB;
            if (r < bn && c < bn)
                Sb[(int64_t)blockIdx.x * 2 * GJB * GJB + r * GJB + c] =
                    ld2(A + blockIdx.x * nn + (int64_t)(kn + r) * n + kn + c);
        }
        if (!gj_grid_sync(bar, bar + 1, gridDim.x, g, &s_abort, err)) return;
        // (C): the update of one tile; CTA t < nbatch takes the diagonal tile of
        // matrix t holding block K + 1 and then inverts that block
        // C[i, :] Rwp[:, j] from the staging, one order of operations for every caller
        auto cprod = [&](int ri, int cj) {
            double t1 = 0.0, t2 = 0.0, t3 = 0.0;
#pragma unroll
            for (int l = 0; l < GJB; ++l) {
                t1 = fma(sC[0][ri][l], sR[0][l][cj], t1);
                t2 = fma(sC[1][ri][l], sR[1][l][cj], t2);
                t3 = fma(sC[2][ri][l], sR[2][l][cj], t3);
            }
            return z64(t1 - t2, t3 - t1 - t2);
        };
        auto stage = [&](int t, int i0, int j0) {   // C rows i0.., right-operand columns j0.. (32 each)
            const z64 *Ct = Ck + (int64_t)t * n * GJB, *Rt = Rwp + (int64_t)t * GJB * n, *Dt = Dk + (int64_t)t * GJB * GJB;
            __syncthreads();   // the previous reads of the staging are done
            for (int e = threadIdx.x; e < 32 * GJB; e += blockDim.x) {
                const int rr = e / GJB, l = e - rr * GJB, i = i0 + rr;
                const z64 v = (i < n && l < b) ? ld2(Ct + (int64_t)i * GJB + l) : z64(0.0, 0.0);
                sC[0][rr][l] = v.re;
                sC[1][rr][l] = v.im;
                sC[2][rr][l] = v.re + v.im;
            }
            for (int e = threadIdx.x; e < GJB * 32; e += blockDim.x) {
                const int l = e / 32, cc = e - l * 32, j = j0 + cc;
                z64 v(0.0, 0.0);
                if (l < b && j < n)
                    v = (j >= k0 && j < k0 + b) ? ld2(Dt + l * GJB + (j - k0)) : ld2(Rt + (int64_t)l * n + j);
                sR[0][l][cc] = v.re;
                sR[1][l][cc] = v.im;
                sR[2][l][cc] = v.re + v.im;
            }
            __syncthreads();
        };
        const int dtile = bn > 0 ? kn / 32 : -1;
        auto update = [&](int t, int bi, int bj) {
            const int i0 = bi * 32, j0 = bj * 32;
            z64 *At = A + t * nn;
            const z64 *Rt = Rwp + (int64_t)t * GJB * n, *Dt = Dk + (int64_t)t * GJB * GJB;
            z64 *Cnt = Cn + (int64_t)t * n * GJB;
            stage(t, i0, j0);
#pragma unroll
            for (int rr = 0; rr < 2; ++rr) {
#pragma unroll
                for (int cc = 0; cc < 2; ++cc) {
                    const int ri = ty + 16 * rr, cj = tx + 16 * cc, i = i0 + ri, j = j0 + cj;
                    if (i >= n || j >= n) continue;
                    const bool ki = i >= k0 && i < k0 + b, kj = j >= k0 && j < k0 + b;
                    z64 *out = At + (int64_t)i * n + j;
                    z64 v;
                    if (ki) {
                        v = kj ? ld2(Dt + (i - k0) * GJB + (j - k0)) : ld2(Rt + (int64_t)(i - k0) * n + j);
                    } else {
                        const z64 prod = cprod(ri, cj);
                        v = kj ? -prod : ld2(out) - prod;
                    }
                    *out = v;
                    if (j >= kn && j < kn + bn) Cnt[(int64_t)i * GJB + (j - kn)] = v;
                }
            }
        };
        if (blockIdx.x < nbatch) {
            if (dtile >= 0) {   // block K + 1 after this step, from its copy, then its inverse
                const int t = blockIdx.x, i0 = (kn / 32) * 32, off = kn - i0;
                z64 *S = Sb + (int64_t)t * 2 * GJB * GJB;
                stage(t, i0, i0);
                const int r = threadIdx.x / GJB, c = threadIdx.x % GJB;
                if (r < bn && c < bn) S[GJB * GJB + r * GJB + c] = S[r * GJB + c] - cprod(off + r, off + c);
                __threadfence();   // the block in L2, where the inverse reads it
                __syncthreads();
                gjb_block_inverse(bn, S + GJB * GJB, GJB, Dn + (int64_t)t * GJB * GJB, flag);
            }
        } else if (!idle) {   // tiles from this step's counter
            const int ntc = nbatch * tn * tn;
            for (;;) {
                __syncthreads();   // s_tile of the previous claim has been read
                if (threadIdx.x == 0) s_tile = (int)atomicAdd(tilectr + k0 / GJB, 1u);
                __syncthreads();
                const int tile = s_tile;
                if (tile >= ntc) break;
                const int t = tile / (tn * tn), rem = tile - t * tn * tn, bi = rem / tn, bj = rem - bi * tn;
                update(t, bi, bj);
            }
        }
        if (!gj_grid_sync(bar, bar + 1, gridDim.x, g, &s_abort, err)) return;
    }
}

// ------------------------------------------------ bounded waits, self-test
// Grid barrier of the persistent kernels waited on for `target` arrivals by
// gridDim.x CTAs: with target > gridDim.x nothing completes it, every CTA
// gives up after the barrier's one-second limit and sets *err.
__global__ void k_wait_grid_selftest(unsigned target, unsigned *__restrict__ bar, int *__restrict__ err) {
    __shared__ int s_abort;
    if (threadIdx.x == 0) s_abort = 0;
    __syncthreads();
    unsigned g = 0;
    gj_grid_sync(bar, bar + 1, target, g, &s_abort, err);
}

// Cluster mbarriers initialised for `expect` arrivals per phase, arrived at by
// the cluster's CTAs: with expect > cluster size the phase never completes and
// each CTA's wait gives up after limit_ns (sets *err); with expect equal to it
// the barrier completes.  The closing hardware cluster barrier is reached by
// every CTA either way.
__global__ void __cluster_dims__(2, 1, 1) k_wait_cluster_selftest(int expect, unsigned long long limit_ns,
                                                                 int *__restrict__ err) {
    cg::cluster_group cl = cg::this_cluster();
    __shared__ uint64_t cbar[2];
    __shared__ int s_abort;
    if (threadIdx.x == 0) {
        s_abort = 0;
        cl_bar_init(cbar, expect);
    }
    __syncthreads();
    cl.sync();
    cl_sync(cbar, 0, (int)cl.num_blocks(), &s_abort, err, limit_ns);
    cl.sync();
}

// row block k of A <- Rwp (b x n); then A_kk <- D
__global__ void k_gjb_place(int n, int k0, int b, const z64 *__restrict__ Rwp, const z64 *__restrict__ D,
                            z64 *__restrict__ A) {
    const int t = blockIdx.y;
    A += (int64_t)t * n * n;
    Rwp += (int64_t)t * b * n;
    D += (int64_t)t * GJB * GJB;
    for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < (int64_t)b * n;
         idx += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = idx / n, c = idx % n;
        const bool diag = c >= k0 && c < k0 + b;
        A[(k0 + r) * n + c] = diag ? D[r * GJB + (c - k0)] : Rwp[idx];
    }
}

// probe vector x_i = cos(i) + j sin(2 i), and err[t] = ||y_t - x|| / ||x||
__global__ void k_gjb_probe(int n, z64 *__restrict__ x) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        x[i] = z64(cos((double)i), sin(2.0 * i));
}
__global__ void __launch_bounds__(256) k_gjb_err(int n, const z64 *__restrict__ y, const z64 *__restrict__ x,
                                                 double *__restrict__ err) {
    __shared__ double p0[8], p1[8];
    const int t = blockIdx.x;
    y += (int64_t)t * n;
    double e = 0.0, r = 0.0;
    for (int i = threadIdx.x; i < n; i += 256) {
        e += norm2(y[i] - x[i]);
        r += norm2(x[i]);
    }
    for (int o = 16; o > 0; o >>= 1) {
        e += __shfl_xor_sync(0xffffffffu, e, o);
        r += __shfl_xor_sync(0xffffffffu, r, o);
    }
    if ((threadIdx.x & 31) == 0) {
        p0[threadIdx.x >> 5] = e;
        p1[threadIdx.x >> 5] = r;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double se = 0.0, sr = 0.0;
        for (int w = 0; w < 8; ++w) {
            se += p0[w];
            sr += p1[w];
        }
        err[t] = (se == se && sr > 0.0) ? sqrt(se / sr) : 1e300;   // NaN -> failure
    }
}

// Blocked Gauss-Jordan of nbatch n x n matrices in place (inv: A on entry);
// true when no diagonal block had a pivot below 1e-13 of its largest entry
// and A^{-1} (A x) reproduces a fixed probe x to 1e-8 for every matrix.
bool gj_blocked(int64_t n, int nbatch, const z64 *Aorig, z64 *inv, cudaStream_t st) {
    DevBuf<z64> C, Rw, RD, x, z, y;
    DevBuf<int> flag;
    DevBuf<double> err;
    C.alloc((size_t)nbatch * n * GJB);
    Rw.alloc((size_t)nbatch * GJB * n);
    // D A_kj (nbatch x b x n) followed by D (nbatch x GJB x GJB): one base
    // pointer, so the update and the column block share a launch
    RD.alloc((size_t)nbatch * GJB * n + (size_t)nbatch * GJB * GJB);
    z64 *const Rwp = RD.p, *const D = RD.p + (size_t)nbatch * GJB * n;
    const int64_t doff = (int64_t)nbatch * GJB * n;
    flag.alloc(1);
    CBFM_CUDA(cudaMemsetAsync(flag.p, 0, sizeof(int), st));
    const unsigned nbk = (unsigned)std::min<int64_t>((n * GJB + 255) / 256, 1024);
    GemmSite site_("site:gauss_jordan");
    // every block step in one cooperative launch (the per-step launches below remain
    // for a device without cooperative launch)
    int dev = 0, coop = 0, occ = 0;
    CBFM_CUDA(cudaGetDevice(&dev));
    CBFM_CUDA(cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev));
    CBFM_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_gjb_persistent, 256, 0));
    const int64_t tn = (n + 31) / 32;
    const bool persistent = coop && occ > 0 && (int64_t)occ * sm_count() > nbatch;
    if (persistent) {
        DevBuf<unsigned> bar, tilectr;
        DevBuf<int> perr, smids;
        DevBuf<z64> Cb, Db, Sb;   // C and D, double-buffered; the look-ahead block
        Cb.alloc((size_t)2 * nbatch * n * GJB);
        Db.alloc((size_t)2 * nbatch * GJB * GJB);
        Sb.alloc((size_t)2 * nbatch * GJB * GJB);
        bar.alloc(2);
        perr.alloc(1);
        smids.alloc(nbatch);
        const int64_t nsteps = (n + GJB - 1) / GJB;
        tilectr.alloc(nsteps);
        CBFM_CUDA(cudaMemsetAsync(tilectr.p, 0, sizeof(unsigned) * nsteps, st));
        CBFM_CUDA(cudaMemsetAsync(bar.p, 0, 2 * sizeof(unsigned), st));
        CBFM_CUDA(cudaMemsetAsync(perr.p, 0, sizeof(int), st));
        const unsigned grid =
            (unsigned)std::min<int64_t>((int64_t)nbatch * (tn * tn + 1), (int64_t)occ * sm_count());
        int ni = (int)n, nb = nbatch;
        z64 *Ap = inv, *Cq = Cb.p, *Rq = Rwp, *Dq = Db.p, *Sq = Sb.p;
        void *args[] = {&ni, &nb, &Ap, &Cq, &Rq, &Dq, &Sq, &flag.p, &bar.p, &perr.p, &smids.p, &tilectr.p};
        prof_add_work("k_gjb_persistent", 6.0 * nbatch * (double)n * n * n, 16.0 * nbatch * (double)n * n * 2);
        {
            ProfScope ps_("k_gjb_persistent", st);
            CBFM_CUDA(cudaLaunchCooperativeKernel((const void *)k_gjb_persistent, dim3(grid), dim3(256), args, 0, st));
            launched("k_gjb_persistent");
        }
        int herr = 0;
        CBFM_CUDA(cudaMemcpyAsync(&herr, perr.p, sizeof(int), cudaMemcpyDeviceToHost, st));
        CBFM_CUDA(cudaStreamSynchronize(st));
        if (herr) throw Fail{CBFM_ETIMEOUT, "Gauss-Jordan: a grid barrier wait expired"};
    }
    for (int64_t k0 = 0; !persistent && k0 < n; k0 += GJB) {
        const int b = (int)std::min<int64_t>(GJB, n - k0);
        k_gjb_panels<<<dim3(nbk, nbatch), 256, 0, st>>>((int)n, (int)k0, b, inv, C.p, Rw.p);
        launched("k_gjb_panels");
        {   // one thread per entry of the block in the elimination: GJB x GJB threads
            prof_add_work("k_gjb_inv", 8.0 * nbatch * (double)b * b * b, 32.0 * nbatch * (double)b * b);
            ProfScope ps_("k_gjb_inv", st);
            k_gjb_inv<<<nbatch, GJB * GJB, 0, st>>>((int)n, (int)k0, b, Rw.p, D, flag.p, inv);
            launched("k_gjb_inv");
        }
        std::vector<GemmDesc> dr, du;
        const int64_t k1 = k0 + b;
        for (int t = 0; t < nbatch; ++t) {
            const int64_t tb = (int64_t)t * b * n, tc = (int64_t)t * n * b, td = (int64_t)t * GJB * GJB,
                          tn = (int64_t)t * n * n;
            dr.push_back(GemmDesc{b, n, b, td, GJB, tb, n, tb, n});   // Rwp = D Rw
            // one launch, disjoint columns of A: A -= C Rwp left and right of column block k, and
            // A[:, k] -= C D (the block was zeroed, so it becomes -C D)
            if (k0 > 0) du.push_back(GemmDesc{n, k0, b, tc, b, tb, n, tn, n});
            if (k1 < n) du.push_back(GemmDesc{n, n - k1, b, tc, b, tb + k1, n, tn + k1, n});
            du.push_back(GemmDesc{n, b, b, tc, b, doff + td, GJB, tn + k0, n});
        }
        gemm_grouped<double>(dr, 0, 0, D, Rw.p, Rwp, false, st);
        gemm_grouped<double>(du, 0, 0, C.p, RD.p, inv, true, st, -1.0);
        k_gjb_place<<<dim3(nbk, nbatch), 256, 0, st>>>((int)n, (int)k0, b, Rwp, D, inv);
        launched("k_gjb_place");
    }
    // probe: y = A^{-1} (A x)
    x.alloc((size_t)n);
    z.alloc((size_t)nbatch * n);
    y.alloc((size_t)nbatch * n);
    err.alloc((size_t)nbatch);
    k_gjb_probe<<<(unsigned)((n + 255) / 256), 256, 0, st>>>((int)n, x.p);
    launched("k_gjb_probe");
    std::vector<GemmDesc> d1, d2;
    for (int t = 0; t < nbatch; ++t) {
        d1.push_back(GemmDesc{n, 1, n, (int64_t)t * n * n, n, 0, 1, (int64_t)t * n, 1});
        d2.push_back(GemmDesc{n, 1, n, (int64_t)t * n * n, n, (int64_t)t * n, 1, (int64_t)t * n, 1});
    }
    gemm_grouped<double>(d1, 0, 0, Aorig, x.p, z.p, false, st);
    gemm_grouped<double>(d2, 0, 0, inv, z.p, y.p, false, st);
    k_gjb_err<<<nbatch, 256, 0, st>>>((int)n, y.p, x.p, err.p);
    launched("k_gjb_err");
    int hflag = 0;
    std::vector<double> herr(nbatch);
    CBFM_CUDA(cudaMemcpyAsync(&hflag, flag.p, sizeof(int), cudaMemcpyDeviceToHost, st));
    CBFM_CUDA(cudaMemcpyAsync(herr.data(), err.p, sizeof(double) * nbatch, cudaMemcpyDeviceToHost, st));
    CBFM_CUDA(cudaStreamSynchronize(st));
    if (hflag) return false;
    for (double e : herr)
        if (!(e <= 1e-8)) return false;
    return true;
}

}  // namespace

template <typename T>
void gemm_grouped(const std::vector<GemmDesc> &g, int opA, int opB, const cx<T> *A, const cx<T> *B, cx<T> *C,
                  bool accumulate, cudaStream_t st, double alpha) {
    if (g.empty()) return;
    {
        double fl = 0, by = 0;
        // complex MACs: 3 real multiply-adds each in the FP64 kernel (three-multiplication form), 4 in FP32
        const double flop_per_cmac = sizeof(T) == 8 ? 6.0 : 8.0;
        for (auto &d : g) {
            fl += flop_per_cmac * d.M * d.N * d.K;
            by += (double)(d.M * d.K + d.K * d.N + d.M * d.N) * sizeof(cx<T>);
        }
        prof_add_work(sizeof(T) == 8 ? "k_gemm_z64" : "k_gemm_c32", fl, by);
        if (sizeof(T) == 8) prof_add_work(g_gemm_site ? g_gemm_site : "site:other", fl, by);   // per solver step
    }
    if constexpr (sizeof(T) == 8) {
        gemm_sk(g, opA, opB, A, B, C, accumulate, st, alpha);
    } else {
        for (size_t g0 = 0; g0 < g.size(); g0 += GB_MAXG) {
            GemmBatch bt;
            bt.ng = (int)std::min<size_t>(GB_MAXG, g.size() - g0);
            int64_t tiles = 0;
            std::vector<int64_t> tg(bt.ng);
            for (int i = 0; i < bt.ng; ++i) {
                const GemmDesc &d = g[g0 + i];
                bt.d[i] = d;
                tg[i] = (d.M > 0 && d.N > 0) ? ((d.M + GB_M - 1) / GB_M) * ((d.N + GB_N - 1) / GB_N) : 0;
                tiles += tg[i];
            }
            if (tiles == 0) continue;
            // few output tiles: split K (slices of at least GB_K) until about two
            // CTAs per SM exist
            const int64_t nsm2 = 2 * (int64_t)sm_count();
            const int64_t want = (tiles < nsm2) ? (nsm2 + tiles - 1) / tiles : 1;
            bt.tile_off[0] = bt.part_off[0] = bt.red_off[0] = 0;
            for (int i = 0; i < bt.ng; ++i) {
                const GemmDesc &d = bt.d[i];
                int64_t S = 1, chunk = 0;
                if (want > 1 && tg[i] > 0 && d.K > GB_K) {
                    S = std::min<int64_t>(want, (d.K + GB_K - 1) / GB_K);
                    chunk = (d.K + S - 1) / S;
                    chunk = (chunk + GB_K - 1) / GB_K * GB_K;
                    S = (d.K + chunk - 1) / chunk;
                }
                bt.ksplit[i] = (int)S;
                bt.kchunk[i] = S > 1 ? chunk : 0;
                bt.tile_off[i + 1] = bt.tile_off[i] + tg[i] * S;
                bt.part_off[i + 1] = bt.part_off[i] + (S > 1 ? S * d.M * d.N : 0);
                bt.red_off[i + 1] = bt.red_off[i] + (S > 1 ? d.M * d.N : 0);
            }
            const int64_t items = bt.tile_off[bt.ng];
            cx<T> *part = nullptr;
            if (bt.part_off[bt.ng] > 0) {
                CBFM_CUDA(cudaMallocAsync((void **)&part, sizeof(cx<T>) * bt.part_off[bt.ng], st));
            }
            {
                ProfScope ps_("k_gemm_c32", st);
                k_gemm<T><<<(unsigned)items, 256, 0, st>>>(bt, opA, opB, A, B, C, part, accumulate ? 1 : 0, (T)alpha);
                launched("k_gemm");
            }
            if (part) {
                const int64_t mn = bt.red_off[bt.ng];
                k_splitk_reduce<T><<<(unsigned)std::min<int64_t>((mn + 255) / 256, 4096), 256, 0, st>>>(
                    bt, part, C, accumulate ? 1 : 0, (T)alpha);
                launched("k_splitk_reduce");
                CBFM_CUDA(cudaFreeAsync(part, st));
            }
        }
    }
}

thread_local const char *g_gemm_site = nullptr;

template void gemm_grouped<double>(const std::vector<GemmDesc> &, int, int, const z64 *, const z64 *, z64 *, bool,
                                   cudaStream_t, double);
template void gemm_grouped<float>(const std::vector<GemmDesc> &, int, int, const c32 *, const c32 *, c32 *, bool,
                                  cudaStream_t, double);

void lu_solve_batched(int nb, const int64_t *h_zoff, const int64_t *h_voff, const int *h_n, int s, z64 *Z, z64 *V,
                      int *d_info, cudaStream_t st) {
    DevBuf<int64_t> zo, vo;
    DevBuf<int> nn;
    zo.alloc(nb);
    vo.alloc(nb);
    nn.alloc(nb);
    CBFM_CUDA(cudaMemcpyAsync(zo.p, h_zoff, nb * sizeof(int64_t), cudaMemcpyHostToDevice, st));
    CBFM_CUDA(cudaMemcpyAsync(vo.p, h_voff, nb * sizeof(int64_t), cudaMemcpyHostToDevice, st));
    CBFM_CUDA(cudaMemcpyAsync(nn.p, h_n, nb * sizeof(int), cudaMemcpyHostToDevice, st));
    {
        ProfScope ps_("k_lu_solve", st);
        k_lu_solve<<<nb, 256, 0, st>>>(zo.p, vo.p, nn.p, s, Z, V, d_info);
        launched("k_lu_solve");
    }
    CBFM_CUDA(cudaStreamSynchronize(st));
}

void jacobi_svd_batched(int nb, int s, z64 *X, z64 *V, double *sig, int *d_info, cudaStream_t st, double keep) {
    // rotation threshold: a few units of round-off in the column dot products
    {
        ProfScope ps_("k_jacobi_svd", st);
        k_jacobi_svd<<<nb * JS_CL, 256, 0, st>>>(s, X, V, sig, d_info, 1e-15 * (s > 8 ? s : 8), keep);
        launched("k_jacobi_svd");
    }
}

void gauss_jordan_inverse(int64_t n, int nbatch, z64 *Aug, z64 *inv, int *d_info, cudaStream_t st) {
    // nbatch matrices n x n, consecutive in `inv` (A on entry, A^{-1} on
    // return); Aug holds 2 nbatch n x n scratch matrices.  The batch shares
    // every launch.
    //
    // First the blocked form (block pivots, no exchanges between blocks: its
    // work is GEMMs), kept when it passes its checks; otherwise the pivoted
    // sweep below runs on the original matrices.
    if (n <= 0 || nbatch <= 0) return;
    CBFM_REQUIRE(n < (int64_t)GJ_IMASK, "Gauss-Jordan: matrix too large for the pivot key");
    CBFM_REQUIRE(nbatch <= 65535, "Gauss-Jordan: batch too large");
    const size_t bytes = sizeof(z64) * (size_t)nbatch * n * n;
    CBFM_CUDA(cudaMemcpyAsync(Aug, inv, bytes, cudaMemcpyDeviceToDevice, st));   // the originals
    if (gj_blocked(n, nbatch, Aug, inv, st)) return;
    CBFM_CUDA(cudaMemcpyAsync(inv, Aug, bytes, cudaMemcpyDeviceToDevice, st));
    z64 *b0 = Aug, *b1 = Aug + (int64_t)nbatch * n * n;
    DevBuf<unsigned long long> keys;
    DevBuf<int> pivrow, src;
    keys.alloc((size_t)nbatch * n);
    pivrow.alloc((size_t)nbatch * n);
    src.alloc((size_t)nbatch * n);
    CBFM_CUDA(cudaMemsetAsync(keys.p, 0, sizeof(unsigned long long) * nbatch * n, st));
    const unsigned nb = (unsigned)std::min<int64_t>((n * n + 255) / 256, 2 * (int64_t)sm_count());
    {
        ProfScope ps_("k_gj_init", st);
        k_gj_init<<<dim3(nb, nbatch), 256, 0, st>>>((int)n, inv, b0, keys.p);
        launched("k_gj_init");
    }
    CBFM_REQUIRE(nbatch <= GJ_MAXB, "Gauss-Jordan: at most 4 matrices per batch");
    DevBuf<unsigned> bar;
    DevBuf<int> err;
    bar.alloc(2);
    err.alloc(1);
    CBFM_CUDA(cudaMemsetAsync(bar.p, 0, 2 * sizeof(unsigned), st));
    CBFM_CUDA(cudaMemsetAsync(err.p, 0, sizeof(int), st));
    int dev = 0, nsm = 0, occ = 0;
    CBFM_CUDA(cudaGetDevice(&dev));
    CBFM_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    CBFM_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_gj_persistent, 256, 0));
    const int tiles = nbatch * (int)(((n + 31) / 32) * ((n + 31) / 32));
    const unsigned grid = (unsigned)std::max(1, std::min(tiles, std::max(1, occ) * nsm));
    {
        int ni = (int)n;
        void *args[] = {&ni, &nbatch, &b0, &b1, &keys.p, &pivrow.p, &d_info, &bar.p, &err.p};
        ProfScope ps_("k_gj_sweep", st);
        CBFM_CUDA(cudaLaunchCooperativeKernel((const void *)k_gj_persistent, dim3(grid), dim3(16, 16), args, 0, st));
        launched("k_gj_sweep");
    }
    if (n & 1) std::swap(b0, b1);   // the last sweep wrote b1 when n is odd
    {
        int herr = 0;
        CBFM_CUDA(cudaMemcpyAsync(&herr, err.p, sizeof(int), cudaMemcpyDeviceToHost, st));
        CBFM_CUDA(cudaStreamSynchronize(st));
        if (herr) throw Fail{CBFM_ETIMEOUT, "Gauss-Jordan: a grid barrier wait expired"};
    }
    prof_add_work("k_gj_sweep", 8.0 * nbatch * (double)n * n * n, 32.0 * nbatch * (double)n * n * n);
    k_gj_perm<<<nbatch, 32, 0, st>>>((int)n, pivrow.p, src.p);
    launched("k_gj_perm");
    {
        ProfScope ps_("k_gj_unpack", st);
        k_gj_unpack<<<dim3(nb, nbatch), 256, 0, st>>>((int)n, b0, src.p, inv);
        launched("k_gj_unpack");
    }
    CBFM_CUDA(cudaStreamSynchronize(st));   // the scratch arrays are released on return
}

void launch_z64_to_c32(const z64 *src, c32 *dst, int64_t n, cudaStream_t st) {
    if (n <= 0) return;
    {
        ProfScope ps_("k_to32", st);
        k_to32<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(src, dst, n);
        launched("k_to32");
    }
}
void launch_c32_to_z64(const c32 *src, z64 *dst, int64_t n, cudaStream_t st) {
    if (n <= 0) return;
    {
        ProfScope ps_("k_to64", st);
        k_to64<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(src, dst, n);
        launched("k_to64");
    }
}

// Bounded-wait self-test (see cbfm_wait_selftest): kind 0 grid barrier never
// completed, 1 cluster barrier never completed, 2 cluster barrier completed.
// Returns whether a wait expired.
bool wait_selftest(int kind, double limit_s, cudaStream_t st) {
    DevBuf<unsigned> bar;
    DevBuf<int> err;
    bar.alloc(2);
    err.alloc(1);
    CBFM_CUDA(cudaMemsetAsync(bar.p, 0, 2 * sizeof(unsigned), st));
    CBFM_CUDA(cudaMemsetAsync(err.p, 0, sizeof(int), st));
    if (kind == 0) {
        k_wait_grid_selftest<<<4, 32, 0, st>>>(5u, bar.p, err.p);   // 4 CTAs, 5 arrivals awaited
        launched("k_wait_grid_selftest");
    } else {
        const unsigned long long ns = (unsigned long long)(limit_s * 1e9);
        k_wait_cluster_selftest<<<2, 32, 0, st>>>(kind == 1 ? 3 : 2, ns, err.p);
        launched("k_wait_cluster_selftest");
    }
    int h = 0;
    CBFM_CUDA(cudaMemcpyAsync(&h, err.p, sizeof(int), cudaMemcpyDeviceToHost, st));
    CBFM_CUDA(cudaStreamSynchronize(st));
    return h != 0;
}

}  // namespace cbfm
