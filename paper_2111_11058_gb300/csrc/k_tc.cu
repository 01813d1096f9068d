// k_tc.cu -- projection of the RWG operators onto the CBFs on the 5th-generation
// tensor cores (Sec. IV, reduced matrix A = (C^JM)^H Z C^MJ), mixed-precision
// path: split-TF32 ("3xTF32") products accumulated in FP32 in tensor memory.
//
// Complex products as real GEMMs.  A complex row a (interleaved re, im in
// memory) times a complex column c is the real dot product of the interleaved
// row with the "expanded" column rows (c_re, -c_im, ...) for the real part and
// (c_im, c_re, ...) for the imaginary part.  So every operand is a K-major
// FP32 matrix read straight from its interleaved complex storage, and the
// accumulator columns come in (re, im) pairs.
//
// Split TF32.  Each operand x is stored as two planes hi = tf32(x),
// lo = tf32(x - hi) (round to nearest, low 13 mantissa bits zero).  The
// product uses hi*hi + hi*lo + lo*hi; the dropped lo*lo term and the rounding
// of lo leave a relative error of about 2^-21 per product.
//
// Two launches of one kernel (k_tc_gemm) per reduced matrix:
//   GEMM1  Y_c = Z_op[:, Lambda_k] C_k for every cell k, operator op and
//          coefficient set (C^M or C^J) that the four blocks of A need; the
//          epilogue writes Y transposed and expanded (hi/lo) for GEMM2.
//   GEMM2  A[rows of cell k, :] = C_k^H Y_c[Lambda_k, :], computed per tile of
//          128 CBF rows against a compact block-diagonal panel of conj(C).
//
// Kernel structure (one output tile of 128 x n per CTA, 4 warps):
//   warp 0 lane 0  TMA producer: 128B-swizzled tiles of A hi/lo and B hi/lo
//                  into a ring of stages (cp.async.bulk.tensor, mbarrier tx)
//   warp 1 lane 0  MMA issuer: tcgen05.mma kind::tf32, accumulator in TMEM,
//                  tcgen05.commit frees a stage when its MMAs are done
//   all 4 warps    epilogue: tcgen05.ld of the warp's 32 TMEM lanes (rows)
// Every mbarrier wait is bounded (wall clock); on expiry the CTA records an
// error, drains its own copies and MMAs (bounded), frees TMEM and returns.
#include <cuda.h>   // CUtensorMap and its enums (the encoder is looked up in the driver at run time)

#include <algorithm>
#include <memory>
#include <atomic>
#include <vector>

#include "internal.cuh"
#include "tc_ptx.cuh"

namespace cbfm {

namespace {

using namespace tc;

constexpr int TC_KB = 32;              // floats per K block = one 128-byte swizzle row
constexpr int TC_BROWS = 64;           // rows per B box
constexpr int TC_NMAX = 256;           // largest MMA N
constexpr int TC_THREADS = 128;
constexpr uint32_t TC_TMEM_COLS = 256;
constexpr size_t TC_A_BYTES = (size_t)TC_M * TC_KB * 4;        // 16 KB per plane
constexpr size_t TC_B_BOX_BYTES = (size_t)TC_BROWS * TC_KB * 4;  // 8 KB per box and plane
constexpr size_t TC_SMEM_BUDGET = 200 * 1024;

enum TcMap { MAP_Z = 0, MAP_BP = 1, MAP_CP = 2, MAP_YT = 3 };

struct TcMaps {
    CUtensorMap m[4];
};

// One output tile.  Coordinates of the 4-D maps are (k, row, c2, plane).
struct TcTask {
    int32_t amap, bmap, a_c2, b_c2;
    int32_t a_row0, b_row0, a_k0, b_k0;
    int32_t nk, n, mode, sidx;   // sidx: scatterer of the task (batched launches)
    int32_t e[6];   // epilogue parameters (see k_tc_gemm)
};

struct TcParams {
    int64_t ne, nh, nred;   // RWGs, CBFs per half, reduced order
    int64_t ldz;            // floats per row of Z and YT planes
    float *yt;              // YT planes [plane][chain][2 nh][ldz]
    c32 *A;                 // reduced matrix (nred x nred row-major)
    int *err;
    int stages;
    int stage_bytes;
};

// ------------------------------------------------------------------ kernel
// mode 0 (GEMM1, rows = RWGs):  e = {op, L_k, P_k, coff_k, row of the first
//   accumulator column within the cell's panel, unused}; accumulator column
//   pair (2j, 2j+1) of panel row pr: set M if pr < P_k else J, CBF coff_k + j.
// mode 1 (GEMM2, rows = CBFs of one half): e = {A row offset, A column offset,
//   valid rows, unused...}; accumulator column pair j -> A column b_row0/2 + j.
// BATCH: the task's scatterer selects its tensor maps and parameters from
// global-memory arrays (stages and stage size stay launch-wide).
template <bool BATCH>
__global__ void __launch_bounds__(TC_THREADS, 1) k_tc_gemm(const __grid_constant__ TcMaps maps,
                                                           const TcTask *__restrict__ tasks, const TcParams P0,
                                                           const TcMaps *__restrict__ maps_g,
                                                           const TcParams *__restrict__ params_g) {
    extern __shared__ uint8_t smem_raw[];
    __shared__ uint64_t full_bar[8], empty_bar[8], done_bar;
    __shared__ uint32_t s_tmem;
    __shared__ int s_abort;
    uint8_t *smem = (uint8_t *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const TcTask t = tasks[blockIdx.x];
    const TcParams P = BATCH ? params_g[t.sidx] : P0;
    const TcMaps *mp = BATCH ? &maps_g[t.sidx] : &maps;
    const int S = P0.stages;
    const int nb = (t.n + TC_BROWS - 1) / TC_BROWS;   // B boxes per plane
    const uint32_t tx_bytes = (uint32_t)(2 * TC_A_BYTES + 2 * nb * TC_B_BOX_BYTES);

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&s_tmem)),
                     "r"(TC_TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (threadIdx.x == 32) {
        for (int s = 0; s < S; ++s) {
            mbar_init(&full_bar[s], 1);
            mbar_init(&empty_bar[s], 1);
        }
        mbar_init(&done_bar, 1);
        s_abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = s_tmem;

    auto stage_a = [&](int s, int plane) { return smem + (size_t)s * P0.stage_bytes + plane * TC_A_BYTES; };
    auto stage_b = [&](int s, int plane) {
        return smem + (size_t)s * P0.stage_bytes + 2 * TC_A_BYTES + (size_t)plane * nb * TC_B_BOX_BYTES;
    };

    if (warp == 0 && lane == 0) {
        // ---------------- TMA producer
        const CUtensorMap *ma = &mp->m[t.amap], *mb = &mp->m[t.bmap];
        if (BATCH) {   // maps written by the host into global memory: acquire them for the tensor proxy
            asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"((uint64_t)ma) : "memory");
            asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"((uint64_t)mb) : "memory");
        }
        int issued = 0;
        for (int kb = 0; kb < t.nk; ++kb) {
            const int s = kb % S, it = kb / S;
            if (kb >= S && !mbar_wait(&empty_bar[s], (it - 1) & 1)) {
                s_abort = 1;
                atomicExch(P.err, 1);
                break;
            }
            if (*(volatile int *)&s_abort) break;
            mbar_expect_tx(&full_bar[s], tx_bytes);
            const int ka = t.a_k0 + kb * TC_KB, kbb = t.b_k0 + kb * TC_KB;
            for (int pl = 0; pl < 2; ++pl) {
                tma_load_4d(stage_a(s, pl), ma, &full_bar[s], ka, t.a_row0, t.a_c2, pl);
                for (int q = 0; q < nb; ++q)
                    tma_load_4d(stage_b(s, pl) + q * TC_B_BOX_BYTES, mb, &full_bar[s], kbb, t.b_row0 + q * TC_BROWS,
                                t.b_c2, pl);
            }
            issued = kb + 1;
        }
        // drain: the last phase issued on every stage has landed before the CTA may exit
        for (int kb = issued > S ? issued - S : 0; kb < issued; ++kb)
            if (!mbar_wait(&full_bar[kb % S], (kb / S) & 1)) atomicExch(P.err, 2);
    } else if (warp == 1 && lane == 0) {
        // ---------------- MMA issuer
        const uint32_t id = idesc_tf32(t.n);
        for (int kb = 0; kb < t.nk; ++kb) {
            const int s = kb % S, it = kb / S;
            if (!mbar_wait(&full_bar[s], it & 1)) {
                s_abort = 1;
                atomicExch(P.err, 3);
                break;
            }
            tc_fence_after();
            const uint32_t a_hi = smem_u32(stage_a(s, 0)), a_lo = smem_u32(stage_a(s, 1));
            const uint32_t b_hi = smem_u32(stage_b(s, 0)), b_lo = smem_u32(stage_b(s, 1));
#pragma unroll
            for (int kk = 0; kk < TC_KB / 8; ++kk) {
                const uint32_t o = kk * 32;   // 8 TF32 = 32 bytes along K inside the swizzled row
                mma_tf32(tmem, sdesc(a_hi + o), sdesc(b_hi + o), id, (kb | kk) != 0);
                mma_tf32(tmem, sdesc(a_hi + o), sdesc(b_lo + o), id, 1);
                mma_tf32(tmem, sdesc(a_lo + o), sdesc(b_hi + o), id, 1);
            }
            mma_commit(&empty_bar[s]);
        }
        if (t.nk > 0) mma_commit(&done_bar);   // all MMAs issued above (and only those) are complete
        else mbar_arrive(&done_bar);
    }
    __syncwarp();

    // ---------------- epilogue
    const bool ok = mbar_wait(&done_bar, 0);
    if (!ok) atomicExch(P.err, 4);
    // one decision for the whole block: tcgen05.ld is warp-collective
    const bool go = __syncthreads_and(ok && t.nk > 0 && !*(volatile int *)&s_abort) != 0;
    tc_fence_after();
    const int row = warp * 32 + lane;
    if (go) {
        const uint32_t tbase = tmem + ((uint32_t)(warp * 32) << 16);
        if (t.mode == 0) {
            const int64_t e = t.a_row0 + row;   // RWG (row of Z)
            const int op = t.e[0], L = t.e[1], Pk = t.e[2], coff = t.e[3], pr0 = t.e[4];
            const int64_t plane = 4 * 2 * P.nh * P.ldz;   // floats per YT plane
            for (int c0 = 0; c0 < t.n; c0 += 16) {
                uint32_t v[16];
                tmem_ld16(tbase + c0, v);
                if (e >= P.ne) continue;
#pragma unroll
                for (int h = 0; h < 8; ++h) {
                    const int pr = pr0 + c0 + 2 * h;
                    const bool setJ = pr >= Pk;
                    const int j = (setJ ? pr - Pk : pr) >> 1;
                    if (j >= L) continue;
                    int chain = -1;
                    if (op == 0) chain = setJ ? 3 : 0;
                    else if (op == 1 && setJ) chain = 1;
                    else if (op == 2 && !setJ) chain = 2;
                    if (chain < 0) continue;
                    const float yr = __uint_as_float(v[2 * h]), yi = __uint_as_float(v[2 * h + 1]);
                    float rh, rl, ih, il;
                    split(yr, rh, rl);
                    split(yi, ih, il);
                    const int64_t J = coff + j;
                    float *base = P.yt + ((int64_t)chain * 2 * P.nh + 2 * J) * P.ldz + 2 * e;
                    // expanded rows: (J, re) = (y_re, -y_im), (J, im) = (y_im, y_re)
                    *reinterpret_cast<float2 *>(base) = make_float2(rh, -ih);
                    *reinterpret_cast<float2 *>(base + P.ldz) = make_float2(ih, rh);
                    *reinterpret_cast<float2 *>(base + plane) = make_float2(rl, -il);
                    *reinterpret_cast<float2 *>(base + plane + P.ldz) = make_float2(il, rl);
                }
            }
        } else {
            const int64_t l = t.a_row0 + row;   // CBF row within the half
            const int r0 = t.e[0], cc0 = t.e[1], nrow = t.e[2];
            for (int c0 = 0; c0 < t.n; c0 += 16) {
                uint32_t v[16];
                tmem_ld16(tbase + c0, v);
                if (l >= nrow) continue;
#pragma unroll
                for (int h = 0; h < 8; ++h) {
                    const int64_t J = (t.b_row0 + c0 + 2 * h) >> 1;
                    if (J >= P.nh) continue;
                    P.A[(r0 + l) * P.nred + cc0 + J] = c32(__uint_as_float(v[2 * h]), __uint_as_float(v[2 * h + 1]));
                }
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TC_TMEM_COLS)
                     : "memory");
}

// ----------------------------------------------------------- operand builders
// Z planes: Zs[plane][op][e][f] = hi/lo of the interleaved float f of row e
// of Z_op (f < 2 ne), zero in the padding up to ldz.
__global__ void k_split_z(int64_t ne, int64_t ldz, const c32 *__restrict__ Z, float *__restrict__ Zs) {
    const int64_t rows = 3 * ne, per = ldz / 2;   // complex slots per row
    const int64_t plane = rows * ldz;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < rows * per;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = i / per, c = i - r * per;
        float2 hi = make_float2(0.f, 0.f), lo = hi;
        if (c < ne) {
            const c32 z = Z[r * ne + c];
            split(z.re, hi.x, lo.x);
            split(z.im, hi.y, lo.y);
        }
        *reinterpret_cast<float2 *>(Zs + r * ldz + 2 * c) = hi;
        *reinterpret_cast<float2 *>(Zs + plane + r * ldz + 2 * c) = lo;
    }
}

// GEMM1 B panels: for cell k, rows [0, P_k) expand C^M_k, rows [P_k, 2 P_k)
// expand C^J_k ((j, re) row then (j, im) row per CBF j; zero rows up to P_k),
// columns kk of the cell's K frame: float kk0_k + kk of a Z row.
// Bp[plane][prow_k + r][kk] with ld ldb.
__global__ void k_build_bpanel(int ncell, const int32_t *__restrict__ cell_off, const int64_t *__restrict__ boff,
                               const int32_t *__restrict__ Ls, const int32_t *__restrict__ Pk,
                               const int32_t *__restrict__ prow, const int32_t *__restrict__ kk0, int64_t ldb,
                               int64_t rows, const z64 *__restrict__ CM, const z64 *__restrict__ CJ,
                               float *__restrict__ Bp) {
    const int k = blockIdx.y;
    const int Pc = Pk[k], L = Ls[k];
    const int64_t off = cell_off[k], N = cell_off[k + 1] - off;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < 2 * Pc * ldb;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int r = (int)(i / ldb);
        const int64_t kk = i - (int64_t)r * ldb;
        const bool setJ = r >= Pc;
        const int q = setJ ? r - Pc : r, j = q >> 1, reim = q & 1;
        const int64_t f = kk0[k] + kk, e = f >> 1;
        const int comp = (int)(f & 1);
        double v = 0.0;
        if (j < L && e >= off && e < off + N) {
            const z64 c = (setJ ? CJ : CM)[boff[k] + (e - off) * L + j];
            v = reim == 0 ? (comp == 0 ? c.re : -c.im) : (comp == 0 ? c.im : c.re);
        }
        float hi, lo;
        split64(v, hi, lo);
        const int64_t o = ((int64_t)prow[k] + r) * ldb + kk;
        Bp[o] = hi;
        Bp[rows * ldb + o] = lo;
    }
}

// GEMM2 A panels: tile t covers CBF rows [128 t, 128 t + 128) of a half and K
// floats [ks_t, ks_t + ldc) of a Z row; entry = interleaved conj(C)
// (c_re, -c_im) of the row's own cell, zero elsewhere.  Cp[plane][half][128 t + r][kk].
__global__ void k_build_cpanel(int64_t nh, int ntile, int64_t ldc, const int32_t *__restrict__ cell_of_cbf,
                               const int32_t *__restrict__ cell_off, const int64_t *__restrict__ coff,
                               const int64_t *__restrict__ boff, const int32_t *__restrict__ Ls,
                               const int32_t *__restrict__ ks, const z64 *__restrict__ CM, const z64 *__restrict__ CJ,
                               float *__restrict__ Cp) {
    const int half = blockIdx.y;
    const z64 *C = half == 0 ? CM : CJ;
    const int64_t rows = (int64_t)ntile * TC_M;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < rows * ldc;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = i / ldc, kk = i - r * ldc;
        double v = 0.0;
        if (r < nh) {
            const int k = cell_of_cbf[r];
            const int64_t j = r - coff[k], off = cell_off[k], N = cell_off[k + 1] - off;
            const int64_t f = ks[r / TC_M] + kk, e = f >> 1;
            if (e >= off && e < off + N) {
                const z64 c = C[boff[k] + (e - off) * Ls[k] + j];
                v = (f & 1) == 0 ? c.re : -c.im;
            }
        }
        float hi, lo;
        split64(v, hi, lo);
        const int64_t o = ((int64_t)half * rows + r) * ldc + kk;
        Cp[o] = hi;
        Cp[2 * rows * ldc + o] = lo;
    }
}

// ------------------------------------------------------------ host helpers
using EncodeFn = CUresult (*)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                              const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                              CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeFn encoder() {
    // thread-safe one-time lookup (a failed lookup is retried on the next call)
    static const EncodeFn fn = [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        CBFM_CUDA(cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q));
        CBFM_REQUIRE(q == cudaDriverEntryPointSuccess && p, "cuTensorMapEncodeTiled not available from the driver");
        return (EncodeFn)p;
    }();
    return fn;
}

// 4-D FP32 map over [d3][d2][d1][d0] (d0 innermost, a multiple of 32), box (32, box_rows, 1, 1), 128B swizzle.
void make_map(CUtensorMap *m, float *base, int64_t d0, int64_t d1, int64_t d2, int64_t d3, int box_rows) {
    CBFM_REQUIRE(d0 % TC_KB == 0, "tensor map: row length must be a multiple of 32 floats");
    CBFM_REQUIRE(((uintptr_t)base & 15) == 0, "tensor map: base not 16-byte aligned");
    cuuint64_t dims[4] = {(cuuint64_t)d0, (cuuint64_t)d1, (cuuint64_t)d2, (cuuint64_t)d3};
    cuuint64_t strides[3] = {(cuuint64_t)d0 * 4, (cuuint64_t)(d0 * d1) * 4, (cuuint64_t)(d0 * d1 * d2) * 4};
    cuuint32_t box[4] = {(cuuint32_t)TC_KB, (cuuint32_t)box_rows, 1, 1};
    cuuint32_t es[4] = {1, 1, 1, 1};
    CUresult r = encoder()(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, base, dims, strides, box, es,
                           CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                           CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) throw Fail{CBFM_ECUDA, "cuTensorMapEncodeTiled failed (" + std::to_string((int)r) + ")"};
}

inline int64_t up(int64_t x, int64_t a) { return (x + a - 1) / a * a; }

// One launch over `tasks`.  maps_g / params_g non-null: batched launch (the
// tasks' sidx index those arrays); otherwise the single-scatterer maps and P.
void launch_tc(const TcMaps &maps, const TcMaps *maps_g, const TcParams *params_g, const std::vector<TcTask> &tasks,
               TcParams P, cudaStream_t st, const char *name) {
    if (tasks.empty()) return;
    int nbmax = 1;
    for (auto &t : tasks) {
        CBFM_REQUIRE(t.n >= 16 && t.n <= TC_NMAX && t.n % 16 == 0, "tensor-core tile: bad N");
        CBFM_REQUIRE(t.a_k0 % TC_KB == 0 && t.b_k0 % TC_KB == 0, "tensor-core tile: K origin not 32-aligned");
        CBFM_REQUIRE(t.a_k0 >= 0 && t.b_k0 >= 0 && t.a_row0 >= 0 && t.b_row0 >= 0, "tensor-core tile: negative origin");
        nbmax = std::max(nbmax, (t.n + TC_BROWS - 1) / TC_BROWS);
    }
    P.stage_bytes = (int)(2 * TC_A_BYTES + 2 * (size_t)nbmax * TC_B_BOX_BYTES);
    P.stages = (int)std::min<size_t>(4, TC_SMEM_BUDGET / P.stage_bytes);
    CBFM_REQUIRE(P.stages >= 2, "tensor-core tile: stages do not fit in shared memory");
    const size_t smem = (size_t)P.stages * P.stage_bytes + 1024;   // + alignment slack
    static std::atomic<bool> attr[64];   // zero-initialised (static storage)
    int dev = 0;
    CBFM_CUDA(cudaGetDevice(&dev));
    if (dev < 64 && !attr[dev].load(std::memory_order_acquire)) {
        CBFM_CUDA(cudaFuncSetAttribute(k_tc_gemm<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)(TC_SMEM_BUDGET + 1024)));
        CBFM_CUDA(cudaFuncSetAttribute(k_tc_gemm<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)(TC_SMEM_BUDGET + 1024)));
        attr[dev].store(true, std::memory_order_release);
    }
    DevBuf<TcTask> dt;
    dt.alloc(tasks.size());
    CBFM_CUDA(cudaMemcpyAsync(dt.p, tasks.data(), sizeof(TcTask) * tasks.size(), cudaMemcpyHostToDevice, st));
    {
        ProfScope ps_(name, st);
        if (maps_g)
            k_tc_gemm<true><<<(unsigned)tasks.size(), TC_THREADS, smem, st>>>(maps, dt.p, P, maps_g, params_g);
        else
            k_tc_gemm<false><<<(unsigned)tasks.size(), TC_THREADS, smem, st>>>(maps, dt.p, P, nullptr, nullptr);
        launched(name);
    }
    CBFM_CUDA(cudaStreamSynchronize(st));   // dt is released on return
}

}  // namespace

namespace {

// Per-scatterer operands of the projection (split planes, panels, index
// tables), its tensor maps and launch parameters, and its work counts.
struct TcPrep {
    DevBuf<float> Zs, Bp, Cp, YT;
    DevBuf<int32_t> dLs, dPk, dprow, dkk0, dcell_off, dcell_of_cbf, dks;
    DevBuf<int64_t> dboff, dcoff;
    TcMaps maps;
    TcParams P;
    double fl1 = 0, fl2 = 0, by1 = 0, by2 = 0;
};

// Builds the operands and appends the scatterer's GEMM1 and GEMM2 tasks
// (tagged sidx).  Returns false when the scatterer has no CBFs.
bool tc_prepare(Mesh &m, Cbf &c, const c32 *Z, c32 *A, int sidx, int *errp, TcPrep &pp, std::vector<TcTask> &t1,
                std::vector<TcTask> &t2, cudaStream_t st) {
    const int nc = m.h.ncell;

    const int64_t ne = m.h.ne, nh = c.nhalf, nred = 2 * nh;
    if (nh == 0) return false;
    const int64_t ldz = up(2 * ne, TC_KB);
    CBFM_REQUIRE(ne < (1ll << 30) / 2 && ldz < (1ll << 31), "mesh too large for 32-bit tile coordinates");

    // --- Z hi/lo planes
    DevBuf<float> &Zs = pp.Zs;
    Zs.alloc((size_t)2 * 3 * ne * ldz);
    {
        ProfScope ps_("k_split_z", st);
        k_split_z<<<4 * sm_count(), 256, 0, st>>>(ne, ldz, Z, Zs.p);
        launched("k_split_z");
        prof_add_work("k_split_z", 0.0, (double)3 * ne * ne * 8 + (double)2 * 3 * ne * ldz * 4);
    }

    // --- GEMM1 B panels (per cell K frame, aligned to 32 floats)
    std::vector<int32_t> Ls(nc), Pk(nc), prow(nc), kk0(nc);
    int64_t ldb = TC_KB, brows = 0;
    for (int k = 0; k < nc; ++k) {
        const int64_t off = m.h.cell_off[k], N = m.h.cell_off[k + 1] - off;
        Ls[k] = c.L[k];
        Pk[k] = (int32_t)up(2 * (int64_t)c.L[k], 16);
        prow[k] = (int32_t)brows;
        brows += 2 * Pk[k];
        kk0[k] = (int32_t)(2 * off / TC_KB * TC_KB);
        ldb = std::max<int64_t>(ldb, up(2 * (off + N), TC_KB) - kk0[k]);
    }
    brows = std::max<int64_t>(brows, 1);
    DevBuf<int32_t> &dLs = pp.dLs, &dPk = pp.dPk, &dprow = pp.dprow, &dkk0 = pp.dkk0, &dcell_off = pp.dcell_off;
    DevBuf<int64_t> &dboff = pp.dboff, &dcoff = pp.dcoff;
    dLs.alloc(nc); dPk.alloc(nc); dprow.alloc(nc); dkk0.alloc(nc); dcell_off.alloc(nc + 1);
    dboff.alloc(nc + 1); dcoff.alloc(nc + 1);
    CBFM_CUDA(cudaMemcpyAsync(dLs.p, Ls.data(), 4 * nc, cudaMemcpyHostToDevice, st));
    CBFM_CUDA(cudaMemcpyAsync(dPk.p, Pk.data(), 4 * nc, cudaMemcpyHostToDevice, st));
    CBFM_CUDA(cudaMemcpyAsync(dprow.p, prow.data(), 4 * nc, cudaMemcpyHostToDevice, st));
    CBFM_CUDA(cudaMemcpyAsync(dkk0.p, kk0.data(), 4 * nc, cudaMemcpyHostToDevice, st));
    CBFM_CUDA(cudaMemcpyAsync(dcell_off.p, m.h.cell_off.data(), 4 * (nc + 1), cudaMemcpyHostToDevice, st));
    CBFM_CUDA(cudaMemcpyAsync(dboff.p, c.boff.data(), 8 * (nc + 1), cudaMemcpyHostToDevice, st));
    CBFM_CUDA(cudaMemcpyAsync(dcoff.p, c.coff.data(), 8 * (nc + 1), cudaMemcpyHostToDevice, st));
    DevBuf<float> &Bp = pp.Bp;
    Bp.alloc((size_t)2 * brows * ldb);
    {
        dim3 g(64, nc);
        k_build_bpanel<<<g, 256, 0, st>>>(nc, dcell_off.p, dboff.p, dLs.p, dPk.p, dprow.p, dkk0.p, ldb, brows, c.CM.p,
                                          c.CJ.p, Bp.p);
        launched("k_build_bpanel");
    }

    // --- GEMM2 A panels (tiles of 128 CBF rows, K span of their cells)
    const int ntile = (int)((nh + TC_M - 1) / TC_M);
    std::vector<int32_t> cell_of_cbf(std::max<int64_t>(nh, 1)), ks(ntile), ke(ntile);
    for (int k = 0; k < nc; ++k)
        for (int64_t j = c.coff[k]; j < c.coff[k + 1]; ++j) cell_of_cbf[j] = k;
    int64_t ldc = TC_KB;
    for (int ti = 0; ti < ntile; ++ti) {
        const int64_t r0 = (int64_t)ti * TC_M, r1 = std::min<int64_t>(nh, r0 + TC_M);
        const int ka = cell_of_cbf[r0], kb = cell_of_cbf[r1 - 1];
        ks[ti] = (int32_t)(2 * (int64_t)m.h.cell_off[ka] / TC_KB * TC_KB);
        ke[ti] = (int32_t)up(2 * (int64_t)m.h.cell_off[kb + 1], TC_KB);
        ldc = std::max<int64_t>(ldc, ke[ti] - ks[ti]);
    }
    DevBuf<int32_t> &dcell_of_cbf = pp.dcell_of_cbf, &dks = pp.dks;
    dcell_of_cbf.alloc(cell_of_cbf.size());
    dks.alloc(ntile);
    CBFM_CUDA(cudaMemcpyAsync(dcell_of_cbf.p, cell_of_cbf.data(), 4 * cell_of_cbf.size(), cudaMemcpyHostToDevice, st));
    CBFM_CUDA(cudaMemcpyAsync(dks.p, ks.data(), 4 * ntile, cudaMemcpyHostToDevice, st));
    DevBuf<float> &Cp = pp.Cp;
    Cp.alloc((size_t)2 * 2 * ntile * TC_M * ldc);
    {
        dim3 g(128, 2);
        k_build_cpanel<<<g, 256, 0, st>>>(nh, ntile, ldc, dcell_of_cbf.p, dcell_off.p, dcoff.p, dboff.p, dLs.p, dks.p,
                                          c.CM.p, c.CJ.p, Cp.p);
        launched("k_build_cpanel");
    }

    // --- YT planes, zero padding columns (GEMM2 may read up to the next 32-float boundary)
    DevBuf<float> &YT = pp.YT;
    YT.alloc((size_t)2 * 4 * 2 * nh * ldz);
    if (ldz > 2 * ne)
        CBFM_CUDA(cudaMemset2DAsync(YT.p + 2 * ne, ldz * 4, 0, (ldz - 2 * ne) * 4, (size_t)2 * 4 * 2 * nh, st));

    TcMaps &maps = pp.maps;
    make_map(&maps.m[MAP_Z], Zs.p, ldz, ne, 3, 2, TC_M);
    make_map(&maps.m[MAP_BP], Bp.p, ldb, brows, 1, 2, TC_BROWS);
    make_map(&maps.m[MAP_CP], Cp.p, ldc, (int64_t)ntile * TC_M, 2, 2, TC_M);
    make_map(&maps.m[MAP_YT], YT.p, ldz, 2 * nh, 4, 2, TC_BROWS);
    TcParams &P = pp.P;
    P = TcParams{};
    P.ne = ne; P.nh = nh; P.nred = nred; P.ldz = ldz; P.yt = YT.p; P.A = A; P.err = errp;

    // --- GEMM1 tasks: (op, cell, 128-row tile of RWGs, chunk of panel rows)
    const int mt = (int)((ne + TC_M - 1) / TC_M);
    double fl1 = 0.0;
    for (int op = 0; op < 3; ++op)
        for (int k = 0; k < nc; ++k) {
            if (c.L[k] == 0) continue;
            const int64_t off = m.h.cell_off[k], N = m.h.cell_off[k + 1] - off;
            // panel rows needed: Ks both sets, Ta the J set, Tb the M set
            const int r_lo = op == 1 ? Pk[k] : 0, r_hi = op == 2 ? Pk[k] : 2 * Pk[k];
            const int nk = (int)((up(2 * (off + N), TC_KB) - kk0[k]) / TC_KB);
            for (int r = r_lo; r < r_hi; r += TC_NMAX) {
                const int n = std::min(TC_NMAX, r_hi - r);
                for (int i = 0; i < mt; ++i) {
                    TcTask t{};
                    t.amap = MAP_Z; t.bmap = MAP_BP; t.a_c2 = op; t.b_c2 = 0;
                    t.a_row0 = i * TC_M; t.b_row0 = prow[k] + r; t.a_k0 = kk0[k]; t.b_k0 = 0;
                    t.nk = nk; t.n = n; t.mode = 0; t.sidx = sidx;
                    t.e[0] = op; t.e[1] = c.L[k]; t.e[2] = Pk[k]; t.e[3] = (int32_t)c.coff[k]; t.e[4] = r;
                    t1.push_back(t);
                }
                fl1 += 8.0 * ne * N * (n / 2);
            }
        }
    pp.fl1 = fl1;
    pp.by1 = (double)2 * 3 * ne * ldz * 4 + (double)2 * 4 * 2 * nh * ldz * 4;

    // --- GEMM2 tasks: (chain, 128-row tile of CBFs, 256-row chunk of YT)
    // chains: 0 C^J^H Ks C^M (rows J, cols M), 1 C^J^H Ta C^J, 2 C^M^H Tb C^M, 3 C^M^H Ks C^J
    const int half_of_rows[4] = {1, 1, 0, 0};
    const int64_t r0q[4] = {0, 0, nh, nh}, c0q[4] = {0, nh, 0, nh};
    double fl2 = 0.0;
    for (int q = 0; q < 4; ++q)
        for (int ti = 0; ti < ntile; ++ti)
            for (int64_t b = 0; b < 2 * nh; b += TC_NMAX) {
                TcTask t{};
                t.amap = MAP_CP; t.bmap = MAP_YT; t.a_c2 = half_of_rows[q]; t.b_c2 = q;
                t.a_row0 = ti * TC_M; t.b_row0 = (int32_t)b; t.a_k0 = 0; t.b_k0 = ks[ti];
                t.nk = (ke[ti] - ks[ti]) / TC_KB;
                t.n = (int)std::min<int64_t>(TC_NMAX, up(2 * nh - b, 16));
                t.mode = 1;
                t.sidx = sidx;
                t.e[0] = (int32_t)r0q[q]; t.e[1] = (int32_t)c0q[q]; t.e[2] = (int32_t)nh;
                t2.push_back(t);
                fl2 += 8.0 * TC_M * ((ke[ti] - ks[ti]) / 2) * (t.n / 2);
            }
    pp.fl2 = fl2;
    pp.by2 = (double)2 * 4 * 2 * nh * ldz * 4 + (double)nred * nred * 8;
    return true;
}

void check_err(const int *errp, cudaStream_t st) {
    int herr = 0;
    CBFM_CUDA(cudaMemcpyAsync(&herr, errp, sizeof(int), cudaMemcpyDeviceToHost, st));
    CBFM_CUDA(cudaStreamSynchronize(st));
    if (herr) throw Fail{CBFM_ETIMEOUT, "tensor-core projection: a pipeline wait expired (stage " +
                                            std::to_string(herr) + ")"};
}

}  // namespace

// A (nred x nred, c32) = the four CBF projections of Z (3 x ne x ne, c32) on
// the tensor cores.  Z is consumed (released by the caller afterwards).
void project_tc(Mesh &m, Cbf &c, const c32 *Z, c32 *A, cudaStream_t st) {
    DevBuf<int> err;
    err.alloc(1);
    CBFM_CUDA(cudaMemsetAsync(err.p, 0, sizeof(int), st));
    TcPrep pp;
    std::vector<TcTask> t1, t2;
    if (!tc_prepare(m, c, Z, A, 0, err.p, pp, t1, t2, st)) return;
    launch_tc(pp.maps, nullptr, nullptr, t1, pp.P, st, "k_tc_gemm1");
    prof_add_work("k_tc_gemm1", pp.fl1, pp.by1);
    pp.Zs.release();
    launch_tc(pp.maps, nullptr, nullptr, t2, pp.P, st, "k_tc_gemm2");
    prof_add_work("k_tc_gemm2", pp.fl2, pp.by2);
    check_err(err.p, st);
}

// The same for several scatterers: one GEMM1 launch and one GEMM2 launch over
// the tasks of all of them (tensor maps and parameters in global memory).
void project_tc_batch(const std::vector<Mesh *> &ms, const std::vector<Cbf *> &cs, const std::vector<const c32 *> &Z,
                      const std::vector<c32 *> &A, cudaStream_t st) {
    DevBuf<int> err;
    err.alloc(1);
    CBFM_CUDA(cudaMemsetAsync(err.p, 0, sizeof(int), st));
    std::vector<std::unique_ptr<TcPrep>> preps;
    std::vector<TcTask> t1, t2;
    std::vector<TcMaps> hmaps;
    std::vector<TcParams> hpar;
    double fl1 = 0, fl2 = 0, by1 = 0, by2 = 0;
    for (size_t k = 0; k < ms.size(); ++k) {
        std::unique_ptr<TcPrep> pp(new TcPrep());
        if (!tc_prepare(*ms[k], *cs[k], Z[k], A[k], (int)hmaps.size(), err.p, *pp, t1, t2, st)) continue;
        hmaps.push_back(pp->maps);
        hpar.push_back(pp->P);
        fl1 += pp->fl1;
        fl2 += pp->fl2;
        by1 += pp->by1;
        by2 += pp->by2;
        preps.push_back(std::move(pp));
    }
    if (hmaps.empty()) return;
    DevBuf<TcMaps> dmaps;
    DevBuf<TcParams> dpar;
    dmaps.alloc(hmaps.size());
    dpar.alloc(hpar.size());
    CBFM_REQUIRE(((uintptr_t)dmaps.p & 63) == 0, "tensor maps in global memory must be 64-byte aligned");
    CBFM_CUDA(cudaMemcpyAsync(dmaps.p, hmaps.data(), sizeof(TcMaps) * hmaps.size(), cudaMemcpyHostToDevice, st));
    CBFM_CUDA(cudaMemcpyAsync(dpar.p, hpar.data(), sizeof(TcParams) * hpar.size(), cudaMemcpyHostToDevice, st));
    launch_tc(hmaps[0], dmaps.p, dpar.p, t1, hpar[0], st, "k_tc_gemm1");
    prof_add_work("k_tc_gemm1", fl1, by1);
    for (auto &pp : preps) pp->Zs.release();
    launch_tc(hmaps[0], dmaps.p, dpar.p, t2, hpar[0], st, "k_tc_gemm2");
    prof_add_work("k_tc_gemm2", fl2, by2);
    check_err(err.p, st);
}

}  // namespace cbfm
