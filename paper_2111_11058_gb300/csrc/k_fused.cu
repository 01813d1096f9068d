// k_fused.cu -- Galerkin assembly fused with the projection onto the CBFs
// (paper Eq. (CBFM_outer) with Eqs. (CBF_matrix_JM), (CBF_matrix_MJ); Z from
// Eqs. (K), (T), (Z) of Sec. II-B), mixed-precision path.  No local-block or
// RWG matrix exists in device memory: each cell pair (m, n) is one work item of
// a persistent kernel that forms the four blocks of A,
//   A_mn = [[C^J_m^H Ks C^M_n, C^J_m^H Ta C^J_n], [C^M_m^H Tb C^M_n, C^M_m^H Ks C^J_n]],
// from the triangles that support the cells' RWG functions.
//
// Work item (m, n).  T_m = triangles carrying an RWG of cell m (test side),
// T_n likewise (trial side), walked in chunks of trial triangles whose cell-n
// RWGs number at most FU_KC.  Per chunk:
//   1. every thread evaluates far triangle pairs (t, s) in T_m x chunk by the
//      FP32 moment quadrature of the far-pair kernel (far_math.cuh) -- near
//      pairs take their FP64 block from the near-pair stage -- and adds the
//      entries whose test RWG is in cell m and trial RWG in cell n into an RWG
//      tile Z_op[i][j] (op = Ks, Ta, Tb; rows i = cell-m RWGs, columns j = the
//      chunk's cell-n RWGs) in shared memory (atomic FP32 adds);
//   2. the tile is split in place into TF32 hi/lo planes;
//   3. one thread issues tcgen05.mma kind::tf32 (hi*hi + hi*lo + lo*hi):
//        Y^T[w][i] += sum_j C_n[j][w] Z_op[i][j]
//      with the CBF coefficients as the A operand (M = 128 lanes: 2 per CBF,
//      real and imaginary rows of the expanded complex product) and the tile
//      as the B operand (N = cell-m RWGs); Y^T accumulates in tensor memory
//      over all chunks of the item.  Lanes [0, 2L) and [2L, 4L) of the Ks
//      accumulator hold Y for C^M and C^J; the Ta and Tb products share a
//      second accumulator (Ta on lanes [0, 2L) with C^J, Tb on [2L, 4L) with
//      C^M; each operand is zero on the other's lanes).
// After the last chunk all warps read Y^T from tensor memory and form
// A_mn = C_m^H Y on the CUDA cores (FP32, L_m x L_n x N_m per chain), writing
// the item's blocks of A directly -- every entry of A has exactly one writer.
//
// Triangle pairs whose triangles carry RWGs of several cells are evaluated once
// per cell pair they feed (about 1.15 x per side on the RCB cells used here).
// The scatter's atomic adds make the summation order of the up to four
// triangle-pair contributions to one RWG entry vary from run to run (last-bit
// differences of A).
//
// Every mbarrier wait is bounded; on expiry the kernel records an error code,
// stops at the next block-wide barrier, frees its tensor memory and returns.
#include <algorithm>
#include <cstring>
#include <mutex>
#include <numeric>
#include <vector>

#include "far_math.cuh"
#include "tc_ptx.cuh"

namespace cbfm {

namespace {

using namespace fm;
using namespace tc;

constexpr int FU_THREADS = 384;
constexpr int FU_WARPS = FU_THREADS / 32;
constexpr int FU_KC = 8;         // trial RWG columns per chunk: 16 floats, one 64-byte swizzled row
constexpr int FU_LMAX = 32;      // largest L_m (4 L lanes of the accumulator <= 128)
constexpr int FU_NMAX = 256;     // largest N_m (MMA N)
constexpr int FU_RING = 8;       // cell-pair items held in shared memory at once
constexpr uint32_t FU_NONE16 = 0xffffu, FU_NONE8 = 0xffu;

struct FusedJob {
    const float *rec;
    const double *rec64;
    const int32_t *vid;
    const float *recT;           // test-side records, field-major over the list entries (stride ntl)
    const int32_t *vidT;
    int64_t ntl;
    const int4 *tl;
    const int32_t *tl_off, *ch_off, *cell_off;
    const int2 *chunk;
    const int16_t *chunk_cols;
    const int32_t *near_row;
    const int2 *near_ent;
    const c32 *near_val;
    const float *aimg;           // per chunk: its CBF operand, 2 planes x 3 operators x 4 L_n rows x 16 floats,
    const int64_t *aimg_off;     //   swizzled as in shared memory, at float offset aimg_off[c]
    const c32 *CM32, *CJ32;      // complex64 CBF blocks (test side of the epilogue)
    const int64_t *boff, *coff;
    const int32_t *L;
    c32 *A;
    int64_t nh, n;
    MediaT<float> md;
    double alpha;
};

// One cell-pair work item and one chunk of the CTA's chunk sequence (shared memory).
struct FuItem {
    int job, m, n, t0, nT, c1, Lm, Ln, Nm, Np, seq;
};
struct FuChunk {
    int slot;          // item ring slot, -1: no more work
    int c, s0, nS, P;  // chunk of the job's table, its trial list range, pairs
    int first;         // first chunk of its item
};

__device__ __forceinline__ void fence_proxy_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// The 27 entries of triangle pair (test list entry ti = triangle t, trial
// triangle s) of job J: FP32 far-pair quadrature, or the near-pair stage's
// block (transposed when the near list holds the pair as (s, t)).  The test
// record comes from the field-major copy (consecutive lanes, consecutive
// entries), the trial record from the triangle records.  Returns false if a
// near pair is missing from the list.
__device__ __forceinline__ bool fused_pair(const FusedJob &J, int64_t ti, int t, int s, c32 *v) {
    const float *rt = J.recT + ti, *rs = J.rec + (int64_t)s * TRI_REC;
    const int64_t L = J.ntl;
    const float cen[3] = {rt[TR_CEN * L], rt[(TR_CEN + 1) * L], rt[(TR_CEN + 2) * L]};
    const float clo[3] = {rt[TR_CLO * L], rt[(TR_CLO + 1) * L], rt[(TR_CLO + 2) * L]};
    const int32_t vt[3] = {J.vidT[ti], J.vidT[ti + L], J.vidT[ti + 2 * L]};
    const int32_t vs[3] = {__ldg(J.vid + 3 * s), __ldg(J.vid + 3 * s + 1), __ldg(J.vid + 3 * s + 2)};
    if (is_near_t<float>(cen, clo, rt[TR_H * L], rs, J.rec64 + (int64_t)t * TRI_REC, J.rec64 + (int64_t)s * TRI_REC,
                         vt, vs, J.alpha)) {
        const int e0 = J.near_row[t], e1 = J.near_row[t + 1];
        int code = -1;
        for (int e = e0; e < e1; ++e) {
            const int2 en = J.near_ent[e];
            if (en.x == s) {
                code = en.y;
                break;
            }
        }
        if (code < 0) {
            for (int c = 0; c < NCOMP; ++c) v[c] = c32(0.f, 0.f);
            return false;
        }
        const c32 *b = J.near_val + (int64_t)(code >> 1) * NCOMP;
        const bool tr = code & 1;
#pragma unroll
        for (int op = 0; op < 3; ++op)
#pragma unroll
            for (int a = 0; a < 3; ++a)
#pragma unroll
                for (int bb = 0; bb < 3; ++bb) v[op * 9 + 3 * a + bb] = b[op * 9 + (tr ? 3 * bb + a : 3 * a + bb)];
        return true;
    }
    far_entries<float, true>(rt, L, rs, J.md, v);
    return true;
}

// Adds a pair's entries into an RWG tile accumulator (shared-memory address `acc`).
__device__ __forceinline__ void fused_scatter(uint32_t acc, int NP, int4 te, int4 se, const c32 *v) {
    const uint32_t rows[3] = {(uint32_t)te.y & 0xffffu, ((uint32_t)te.y >> 16) & 0xffffu, (uint32_t)te.z & 0xffffu};
    const uint32_t cols[3] = {((uint32_t)se.z >> 16) & 0xffu, ((uint32_t)se.z >> 24) & 0xffu, (uint32_t)se.w & 0xffu};
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        if (rows[a] == FU_NONE16) continue;
#pragma unroll
        for (int b = 0; b < 3; ++b) {
            if (cols[b] == FU_NONE8) continue;
#pragma unroll
            for (int op = 0; op < 3; ++op) {
                const uint32_t sa = acc + 4u * (uint32_t)(((op * FU_KC + (int)cols[b]) * 2) * NP + (int)rows[a]);
                asm volatile("red.shared.add.f32 [%0], %1;" ::"r"(sa), "f"(v[op * 9 + 3 * a + b].re) : "memory");
                asm volatile("red.shared.add.f32 [%0], %1;" ::"r"(sa + 4u * NP), "f"(v[op * 9 + 3 * a + b].im)
                             : "memory");
            }
        }
    }
}

// Shared-memory plan (bytes from the 1024-aligned base):
//   A images (the CBF operand), two buffers: hi then lo plane, 3 operators x RA rows x 64 B;
//   the RWG tile as MMA operand, one buffer: hi then lo plane, 3 operators x NP rows x 64 B;
//   the RWG tile as FP32 accumulator, two buffers: 3 operators x 8 columns x (re, im) x NP rows
//   (column-major, so the lanes of a warp -- one trial triangle, consecutive test
//   triangles -- add into scattered banks).
// laid out [A0 | A1 | Z hi | Z lo | acc0 | acc1].  An A operand is read 128 rows
// deep from its base; rows past its image land in the next region (lanes that
// are not used).
struct FuPlan {
    int RA, NP;
    uint32_t a_op, z_op, z_base, acc_base, acc_buf, total;
};

__device__ __forceinline__ uint32_t fu_a(const FuPlan &P, int b, int plane, int op) {
    return (uint32_t)(b * 6 + plane * 3 + op) * P.a_op;
}
__device__ __forceinline__ uint32_t fu_z(const FuPlan &P, int plane, int op) {
    return P.z_base + (uint32_t)(plane * 3 + op) * P.z_op;
}
// float index of (operator, RWG column, re/im, RWG row) in an accumulator buffer
__device__ __forceinline__ uint32_t fu_acc_idx(const FuPlan &P, int op, int col, int ri, int row) {
    return (uint32_t)(((op * FU_KC + col) * 2 + ri) * P.NP + row);
}

// Thread `tid` of `nthr` takes the next item of the CTA's sequence: fills ring
// slot seq % FU_RING.  Returns false when the work is exhausted.
__device__ bool fu_fetch(const FusedJob *jobs, const int4 *items, int nitems, unsigned *counter, FuItem *ring,
                         int seq) {
    const int it = (int)atomicAdd(counter, 1u);
    if (it >= nitems) return false;
    const int4 im = __ldg(items + it);
    const FusedJob &J = jobs[im.x];
    FuItem &o = ring[seq % FU_RING];
    o.job = im.x;
    o.m = im.y;
    o.n = im.z;
    o.t0 = J.tl_off[im.y];
    o.nT = J.tl_off[im.y + 1] - o.t0;
    o.c1 = J.ch_off[im.z + 1];
    o.Lm = J.L[im.y];
    o.Ln = J.L[im.z];
    o.Nm = J.cell_off[im.y + 1] - J.cell_off[im.y];
    o.Np = (o.Nm + 15) & ~15;
    o.seq = seq;
    return true;
}

// Identity of chunk c of the item in ring slot `slot`.
__device__ void fu_chunk(const FusedJob *jobs, const FuItem *ring, int slot, int c, FuChunk &out) {
    const FuItem &it = ring[slot];
    const FusedJob &J = jobs[it.job];
    const int2 ch = J.chunk[c];
    out.slot = slot;
    out.c = c;
    out.s0 = ch.x;
    out.nS = ch.y - ch.x;
    out.P = it.nT * out.nS;
    out.first = c == J.ch_off[it.n];
}

// Chunk identity following `prev` (one thread); may fetch the next item.
__device__ void fu_next(const FusedJob *jobs, const int4 *items, int nitems, unsigned *counter, FuItem *ring,
                        int *nseq, const FuChunk &prev, FuChunk &out) {
    if (prev.slot < 0) {
        out.slot = -1;
        return;
    }
    if (prev.c + 1 < ring[prev.slot].c1) {
        fu_chunk(jobs, ring, prev.slot, prev.c + 1, out);
        return;
    }
    if (!fu_fetch(jobs, items, nitems, counter, ring, *nseq)) {
        out.slot = -1;
        return;
    }
    const int slot = *nseq % FU_RING;
    ++*nseq;
    fu_chunk(jobs, ring, slot, jobs[ring[slot].job].ch_off[ring[slot].n], out);
}

// Starts the asynchronous copies of chunk ck's CBF operand into buffer b
// (one thread; completion on `bar`).
__device__ __forceinline__ void fu_load_a(const FuPlan &P, uint32_t sbase, int b, const FusedJob *jobs, const FuItem &it,
                                          const FuChunk &ck, uint64_t *bar, int *issued) {
    const FusedJob &J = jobs[it.job];
    const uint32_t seg = (uint32_t)(4 * it.Ln) * 64u;   // bytes of one operator's rows in one plane
    mbar_expect_tx(bar, 6 * seg);
    ++*issued;
    const float *src = J.aimg + J.aimg_off[ck.c];
    for (int q = 0; q < 6; ++q)
        asm volatile(
            "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                sbase + fu_a(P, b, q / 3, q % 3)),
            "l"(src + (int64_t)q * (seg / 4)), "r"(seg), "r"(smem_u32(bar))
            : "memory");
}

__device__ __forceinline__ void fu_zero_acc(const FuPlan &P, uint8_t *sm, int b, int t0, int step) {
    for (int idx = t0; idx < 3 * FU_KC * 2 * P.NP / 4; idx += step)
        *reinterpret_cast<float4 *>(sm + P.acc_base + b * P.acc_buf + idx * 16) = make_float4(0.f, 0.f, 0.f, 0.f);
}

// A_mn = C_m^H Y for the four chains of item `pi` once its last MMAs (phase
// `parity` of `bar`) are done.  Warp w reads tensor-memory lanes 32 (w mod 4)
// ... + 31; the three warps of a lane quarter split the test CBFs l in thirds.
// Lane r < 4 L_n holds, for every test RWG i of cell m (column i of its
// accumulator), the real (r even) or imaginary (r odd) part of Y[i][w] of CBF
// w = (r mod 2 L_n) / 2: C^M_n (lower lanes) and C^J_n (upper) in the Ks
// accumulator, C^J_n with Ta (lower) and C^M_n with Tb (upper) in the other.
// Returns false if the wait expired.
constexpr int FU_LPART = (FU_LMAX + 2) / 3;   // test CBFs per warp of a lane quarter
__device__ bool fu_epilogue(const FusedJob *jobs, const FuItem &pi, uint32_t tmem, uint64_t *bar, uint32_t parity,
                            int warp, int lane) {
    const bool ok = mbar_wait(bar, parity);
    tc_fence_after();
    const FusedJob &J = jobs[pi.job];
    const int Ln = pi.Ln, Lm = pi.Lm, Nm = pi.Nm, Np = pi.Np;
    const int quarter = warp & 3, third = warp >> 2;
    const int lpart = (Lm + 2) / 3, l0 = third * lpart, nl = max(0, min(lpart, Lm - l0));
    if (ok && 32 * quarter < 4 * Ln && nl > 0) {
        const int r = 32 * quarter + lane;
        const bool valid = r < 4 * Ln;
        const bool upper = r >= 2 * Ln;
        const int w = (r - (upper ? 2 * Ln : 0)) >> 1, ri = r & 1;
        // rows of A: J-tested (C^J_m) on the lower lanes, M-tested (C^M_m) on the upper
        const c32 *Cr = (upper ? J.CM32 : J.CJ32) + J.boff[pi.m] + l0;
        const int64_t row0 = (upper ? J.nh : 0) + J.coff[pi.m] + l0;
#pragma unroll 1
        for (int g = 0; g < 2; ++g) {
            // columns: Ks group: C^M_n (lower) / C^J_n (upper); Ta/Tb group: C^J_n (lower) / C^M_n (upper)
            const int64_t col0 = ((g == 0) == upper ? J.nh : 0) + J.coff[pi.n];
            float ar[FU_LPART], ai[FU_LPART];
#pragma unroll
            for (int l = 0; l < FU_LPART; ++l) ar[l] = ai[l] = 0.f;
            for (int i0 = 0; i0 < Nm; i0 += 16) {
                uint32_t y[16];
                tmem_ld16(tmem + ((uint32_t)(32 * quarter) << 16) + (uint32_t)(g * Np + i0), y);
                if (!valid) continue;
                const int qn = min(16, Nm - i0);
#pragma unroll 4
                for (int q = 0; q < qn; ++q) {
                    const float yv = __uint_as_float(y[q]);
                    const c32 *crow = Cr + (int64_t)(i0 + q) * Lm;
                    // conj(c) (y_re + j y_im): lane ri = 0 holds y_re, ri = 1 holds y_im
                    const float s1 = ri == 0 ? 1.f : 0.f, s2 = ri == 0 ? 0.f : 1.f;
#pragma unroll
                    for (int l = 0; l < FU_LPART; ++l) {
                        if (l < nl) {
                            const c32 cc = crow[l];
                            ar[l] = fmaf(s1 * cc.re + s2 * cc.im, yv, ar[l]);
                            ai[l] = fmaf(s2 * cc.re - s1 * cc.im, yv, ai[l]);
                        }
                    }
                }
            }
#pragma unroll
            for (int l = 0; l < FU_LPART; ++l) {
                ar[l] += __shfl_xor_sync(0xffffffffu, ar[l], 1);
                ai[l] += __shfl_xor_sync(0xffffffffu, ai[l], 1);
            }
            if (valid && ri == 0) {
                c32 *dst = J.A + col0 + w;
#pragma unroll
                for (int l = 0; l < FU_LPART; ++l)
                    if (l < nl) dst[(row0 + l) * J.n] = c32(ar[l], ai[l]);
            }
        }
    }
    tc_fence_before();
    return ok;
}

__global__ void __launch_bounds__(FU_THREADS, 1)
    k_fused(const FusedJob *__restrict__ jobs, const int4 *__restrict__ items, int nitems,
            unsigned int *__restrict__ counter, int *__restrict__ err, const FuPlan plan, uint32_t tmem_cols) {
    extern __shared__ uint8_t fu_raw[];
    __shared__ uint64_t mma_bar[2], ready_bar[2], aimg_bar[2], epi_bar;
    __shared__ int pair_ctr[2], done_ctr[2];
    __shared__ int a_issued[2], a_waited[2];   // operand copies started / waited for, per buffer
    __shared__ FuItem s_it[FU_RING];
    __shared__ FuChunk s_ck[2];
    __shared__ int s_nseq, s_abort;
    __shared__ uint32_t s_tmem;
    uint8_t *sm = (uint8_t *)(((uintptr_t)fu_raw + 1023) & ~(uintptr_t)1023);
    const uint32_t sbase = smem_u32(sm);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&s_tmem)),
                     "r"(tmem_cols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 32) {
        for (int b = 0; b < 2; ++b) {
            mbar_init(&mma_bar[b], 1);
            mbar_init(&ready_bar[b], 1);
            mbar_init(&aimg_bar[b], 1);
            pair_ctr[b] = done_ctr[b] = 0;
            a_issued[b] = a_waited[b] = 0;
        }
        mbar_init(&epi_bar, FU_WARPS);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        s_abort = 0;
        s_nseq = 0;
        s_ck[0].slot = -1;
        if (fu_fetch(jobs, items, nitems, counter, s_it, 0)) {
            s_nseq = 1;
            fu_chunk(jobs, s_it, 0, jobs[s_it[0].job].ch_off[s_it[0].n], s_ck[0]);
        }
        fu_next(jobs, items, nitems, counter, s_it, &s_nseq, s_ck[0], s_ck[1]);
    }
    __syncthreads();
    // chunk 0's CBF operand now; chunk k + 1's is started by the service of chunk k
    if (tid == 32 && s_ck[0].slot >= 0)
        fu_load_a(plan, sbase, 0, jobs, s_it[s_ck[0].slot], s_ck[0], &aimg_bar[0], &a_issued[0]);
    for (int b = 0; b < 2; ++b) fu_zero_acc(plan, sm, b, tid, FU_THREADS);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = s_tmem;

    int prev_slot = -1, prev_k = -1;   // item of the previous chunk (epilogue), its last chunk
    for (int k = 0;; ++k) {
        const int b = k & 1;
        if (k >= 2 && !mbar_wait(&ready_bar[b], ((k >> 1) - 1) & 1)) {
            atomicExch(err, 5);
            s_abort = 1;
        }
        if (*(volatile int *)&s_abort) break;
        const FuChunk ck = s_ck[b];
        if (ck.slot < 0) break;
        // ---- triangle pairs of the chunk, 32 at a time per warp
        {
            const FuItem &it = s_it[ck.slot];
            const FusedJob &J = jobs[it.job];
            const uint32_t acc = sbase + plan.acc_base + b * plan.acc_buf;
            const int t0 = it.t0;
            while (true) {
                int start = 0;
                if (lane == 0) start = atomicAdd(&pair_ctr[b], 32);
                start = __shfl_sync(0xffffffffu, start, 0);
                if (start >= ck.P) break;
                const int p = start + lane;
                if (p < ck.P) {
                    // consecutive lanes: consecutive test triangles, one trial triangle (mostly)
                    const int si = p / it.nT, ti = t0 + (p - si * it.nT);
                    c32 v[NCOMP];
                    if (!fused_pair(J, ti, J.tl[ti].x, J.tl[ck.s0 + si].x, v)) atomicExch(err, 7);
                    fused_scatter(acc, plan.NP, J.tl[ti], J.tl[ck.s0 + si], v);
                }
            }
        }
        // ---- epilogue of the previous item, after this warp's share of the new item's first chunk (its
        // accumulators are needed again only by that chunk's MMAs, issued after every warp is done here)
        if (ck.first && prev_slot >= 0) {
            if (!fu_epilogue(jobs, s_it[prev_slot], tmem, &mma_bar[prev_k & 1], (prev_k >> 1) & 1, warp, lane)) {
                atomicExch(err, 6);
                s_abort = 1;
            }
            __syncwarp();
            if (lane == 0) mbar_arrive(&epi_bar);
        }
        prev_slot = ck.slot;
        prev_k = k;
        __syncwarp();
        __threadfence_block();
        int last = 0;
        if (lane == 0) last = atomicAdd(&done_ctr[b], 1) == FU_WARPS - 1;
        last = __shfl_sync(0xffffffffu, last, 0);
        if (!last) continue;
        // ---- service of chunk k by the warp that finished it last
        __threadfence_block();
        {
            const FuItem &it = s_it[ck.slot];
            const int Np = it.Np;
            // the previous chunk's MMAs must be done with the operand planes and with A[b ^ 1]
            if (k >= 1 && !mbar_wait(&mma_bar[b ^ 1], ((k - 1) >> 1) & 1)) {
                atomicExch(err, 9);
                s_abort = 1;
            }
            if (lane == 0) {
                const FuChunk &nx = s_ck[b ^ 1];   // chunk k + 1 (set by the previous service)
                if (nx.slot >= 0) fu_load_a(plan, sbase, b ^ 1, jobs, s_it[nx.slot], nx, &aimg_bar[b ^ 1], &a_issued[b ^ 1]);
            }
            // accumulator -> operand planes: hi = tf32(x), lo = tf32(x - hi); the accumulator is zeroed
            {
                float *ac = reinterpret_cast<float *>(sm + plan.acc_base + b * plan.acc_buf);
#pragma unroll 1
                for (int rest = 0; rest < 3 * FU_KC * 2; ++rest) {   // rest = (op * FU_KC + col) * 2 + ri
                    const int ri = rest & 1, col = (rest >> 1) % FU_KC, op = rest / (2 * FU_KC);
                    float *acr = ac + (uint32_t)rest * plan.NP;
                    uint8_t *ph = sm + fu_z(plan, 0, op), *pl = sm + fu_z(plan, 1, op);
                    for (int row = lane; row < Np; row += 32) {
                        const float x = acr[row];
                        acr[row] = 0.f;
                        float h, l;
                        split(x, h, l);
                        const uint32_t off = swz64(row, 2 * col + ri);
                        *reinterpret_cast<float *>(ph + off) = h;
                        *reinterpret_cast<float *>(pl + off) = l;
                    }
                }
            }
            fence_proxy_async_smem();   // generic-proxy writes -> tensor-core reads
            __syncwarp();
            if (lane == 0) {
                bool ok = true;
                // the first MMA of an item overwrites the accumulators: the previous item's epilogue must be done
                if (ck.first && it.seq > 0) ok = mbar_wait(&epi_bar, (it.seq - 1) & 1);
                if (mbar_wait(&aimg_bar[b], a_waited[b] & 1)) ++a_waited[b];   // the chunk's CBF operand has landed
                else ok = false;
                if (!ok) {
                    atomicExch(err, 8);
                    s_abort = 1;
                }
                tc_fence_after();
                const uint32_t idesc = idesc_tf32(Np);
#pragma unroll 1
                for (int op = 0; op < 3; ++op) {
                    const uint32_t d = tmem + (op == 0 ? 0u : (uint32_t)Np);
                    const uint32_t a_h = sbase + fu_a(plan, b, 0, op), a_l = sbase + fu_a(plan, b, 1, op);
                    const uint32_t b_h = sbase + fu_z(plan, 0, op), b_l = sbase + fu_z(plan, 1, op);
#pragma unroll
                    for (int ks = 0; ks < 2; ++ks) {
                        const uint32_t o = ks * 32;   // 8 TF32 along K inside the 64-byte row
                        const uint32_t acc0 = (ck.first && ks == 0 && op < 2) ? 0u : 1u;
                        mma_tf32(d, sdesc64(a_h + o), sdesc64(b_h + o), idesc, acc0);
                        mma_tf32(d, sdesc64(a_h + o), sdesc64(b_l + o), idesc, 1);
                        mma_tf32(d, sdesc64(a_l + o), sdesc64(b_h + o), idesc, 1);
                    }
                }
                mma_commit(&mma_bar[b]);
            }
            if (lane == 1) {
                // buffer b (accumulator zeroed above) takes chunk k + 2 (in parallel with the MMA issue)
                fu_next(jobs, items, nitems, counter, s_it, &s_nseq, s_ck[b ^ 1], s_ck[b]);
                pair_ctr[b] = 0;
                done_ctr[b] = 0;
            }
            __threadfence_block();
            __syncwarp();
            if (lane == 0) mbar_arrive(&ready_bar[b]);
        }
    }
    // ---- epilogue of the last item
    if (prev_slot >= 0 && !*(volatile int *)&s_abort) {
        if (!fu_epilogue(jobs, s_it[prev_slot], tmem, &mma_bar[prev_k & 1], (prev_k >> 1) & 1, warp, lane))
            atomicExch(err, 6);
    }
    tc_fence_before();
    __syncthreads();
    // after an expired wait, operand copies may still be in flight: let them land (bounded) before exit
    if (tid == 32)
        for (int b = 0; b < 2; ++b)
            while (a_waited[b] < a_issued[b]) {
                if (!mbar_wait(&aimg_bar[b], a_waited[b] & 1)) atomicExch(err, 10);
                ++a_waited[b];
            }
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(tmem_cols) : "memory");
}

// ------------------------------------------------------------ host tables
uint32_t morton10(uint32_t x) {
    x &= 0x3ff;
    x = (x | (x << 16)) & 0x030000ff;
    x = (x | (x << 8)) & 0x0300f00f;
    x = (x | (x << 4)) & 0x030c30c3;
    x = (x | (x << 2)) & 0x09249249;
    return x;
}

std::mutex g_fused_mu;

// Field-major copies of the FP32 records and vertex ids of the list entries.
__global__ void k_tl_soa(int64_t ntl, const int4 *__restrict__ tl, const float *__restrict__ rec,
                         const int32_t *__restrict__ vid, float *__restrict__ recT, int32_t *__restrict__ vidT) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < ntl * TRI_REC;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t e = i % ntl, f = i / ntl;
        const int t = tl[e].x;
        recT[i] = rec[(int64_t)t * TRI_REC + f];
        if (f < 3) vidT[i] = vid[3 * (int64_t)t + f];
    }
}

}  // namespace

FusedTables &fused_tables(Mesh &m, cudaStream_t st) {
    std::lock_guard<std::mutex> lk(g_fused_mu);
    if (m.fused) return *m.fused;
    const HostMesh &h = m.h;
    const int nc = h.ncell;
    const int64_t nt = h.nt;
    std::vector<int32_t> ecell(h.ne);
    for (int c = 0; c < nc; ++c)
        for (int32_t e = h.cell_off[c]; e < h.cell_off[c + 1]; ++e) ecell[e] = c;
    // spatial order of the triangles (Morton code of the centroid in the bounding box)
    std::vector<double> cen(3 * nt);
    double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300};
    for (int64_t t = 0; t < nt; ++t)
        for (int d = 0; d < 3; ++d) {
            double x = 0;
            for (int a = 0; a < 3; ++a) x += h.verts[3 * h.tris[3 * t + a] + d];
            cen[3 * t + d] = x / 3.0;
            lo[d] = std::min(lo[d], x / 3.0);
            hi[d] = std::max(hi[d], x / 3.0);
        }
    std::vector<uint32_t> key(nt);
    for (int64_t t = 0; t < nt; ++t) {
        uint32_t q[3];
        for (int d = 0; d < 3; ++d) {
            const double span = hi[d] - lo[d];
            q[d] = span > 0 ? (uint32_t)std::min(1023.0, (cen[3 * t + d] - lo[d]) / span * 1023.0) : 0u;
        }
        key[t] = morton10(q[0]) | (morton10(q[1]) << 1) | (morton10(q[2]) << 2);
    }
    std::vector<std::vector<int32_t>> lists(nc);
    for (int64_t t = 0; t < nt; ++t) {
        int seen[3] = {-1, -1, -1};
        for (int a = 0; a < 3; ++a) {
            const int c = ecell[h.tri_edge[3 * t + a]];
            if (c != seen[0] && c != seen[1]) lists[c].push_back((int32_t)t);
            seen[a] = c;
        }
    }
    auto ft = std::make_shared<FusedTables>();
    ft->tl_off.assign(nc + 1, 0);
    ft->ch_off.assign(nc + 1, 0);
    std::vector<int4> ent;
    std::vector<int2> chunks;
    std::vector<int16_t> ccols;
    for (int c = 0; c < nc; ++c) {
        auto &L = lists[c];
        std::stable_sort(L.begin(), L.end(), [&](int32_t a, int32_t b) { return key[a] < key[b]; });
        ft->tl_off[c] = (int32_t)ent.size();
        ft->ch_off[c] = (int32_t)chunks.size();
        ft->nmax = std::max(ft->nmax, h.cell_off[c + 1] - h.cell_off[c]);
        // greedy chunks: consecutive triangles while their cell-c RWGs number <= FU_KC
        std::vector<int32_t> cur;    // cell-local RWG index of each column
        int begin = (int)ent.size();
        auto close = [&](int end) {
            if (end <= begin) return;
            chunks.push_back(make_int2(begin, end));
            for (int q = 0; q < FU_KC; ++q) ccols.push_back(q < (int)cur.size() ? (int16_t)cur[q] : (int16_t)-1);
            cur.clear();
            begin = end;
        };
        for (int32_t t : L) {
            int newc = 0;
            for (int a = 0; a < 3; ++a) {
                const int32_t e = h.tri_edge[3 * t + a];
                if (ecell[e] != c) continue;
                const int32_t loc = e - h.cell_off[c];
                bool dup = std::find(cur.begin(), cur.end(), loc) != cur.end();
                for (int b = 0; b < a; ++b) dup |= h.tri_edge[3 * t + b] == e;
                newc += dup ? 0 : 1;
            }
            if ((int)cur.size() + newc > FU_KC) close((int)ent.size());
            uint32_t rows[3], cols[3];
            for (int a = 0; a < 3; ++a) {
                const int32_t e = h.tri_edge[3 * t + a];
                rows[a] = FU_NONE16;
                cols[a] = FU_NONE8;
                if (ecell[e] != c) continue;
                const int32_t loc = e - h.cell_off[c];
                rows[a] = (uint32_t)loc;
                auto it = std::find(cur.begin(), cur.end(), loc);
                if (it == cur.end()) {
                    cur.push_back(loc);
                    it = cur.end() - 1;
                }
                cols[a] = (uint32_t)(it - cur.begin());
            }
            int4 e4;
            e4.x = t;
            e4.y = (int)(rows[0] | (rows[1] << 16));
            e4.z = (int)(rows[2] | (cols[0] << 16) | (cols[1] << 24));
            e4.w = (int)cols[2];
            ent.push_back(e4);
        }
        close((int)ent.size());
    }
    ft->tl_off[nc] = (int32_t)ent.size();
    ft->ch_off[nc] = (int32_t)chunks.size();
    // list positions of the two triangles of every RWG function (both carry it, so both are in its cell's list)
    std::vector<int2> rpos(h.ne, make_int2(-1, -1));
    for (int c = 0; c < nc; ++c)
        for (int32_t q = ft->tl_off[c]; q < ft->tl_off[c + 1]; ++q) {
            const int32_t t = ent[q].x;
            for (int a = 0; a < 3; ++a) {
                const int32_t e = h.tri_edge[3 * t + a];
                if (ecell[e] != c) continue;
                if (h.edge_tri[2 * e] == t) rpos[e].x = q - ft->tl_off[c];
                if (h.edge_tri[2 * e + 1] == t) rpos[e].y = q - ft->tl_off[c];
            }
        }
    for (int64_t e = 0; e < h.ne; ++e)
        CBFM_REQUIRE(rpos[e].x >= 0 && rpos[e].y >= 0, "triangle tables: an RWG function's triangle is missing");
    CBFM_REQUIRE(ft->nmax <= 0xfffe, "cell too large for the fused tables");
    // near list as CSR over the test triangle, both orientations
    std::vector<int32_t> np(2 * m.n_near);
    if (m.n_near)
        CBFM_CUDA(cudaMemcpyAsync(np.data(), m.near_pairs.p, np.size() * 4, cudaMemcpyDeviceToHost, st));
    CBFM_CUDA(cudaStreamSynchronize(st));
    std::vector<int32_t> rowc(nt + 1, 0);
    for (int64_t l = 0; l < m.n_near; ++l) {
        rowc[np[2 * l] + 1]++;
        if (np[2 * l] != np[2 * l + 1]) rowc[np[2 * l + 1] + 1]++;
    }
    for (int64_t t = 0; t < nt; ++t) rowc[t + 1] += rowc[t];
    std::vector<int2> ne(rowc[nt]);
    std::vector<int32_t> fill(rowc.begin(), rowc.end() - 1);
    for (int64_t l = 0; l < m.n_near; ++l) {
        const int32_t t = np[2 * l], s = np[2 * l + 1];
        ne[fill[t]++] = make_int2(s, (int)(2 * l));
        if (t != s) ne[fill[s]++] = make_int2(t, (int)(2 * l + 1));
    }
    CBFM_REQUIRE(2 * m.n_near < (1ll << 31), "near list too long for the fused tables");
    ft->n_near = m.n_near;
    auto up = [&](auto &buf, const auto &v) {
        buf.alloc(std::max<size_t>(1, v.size()));
        if (!v.empty())
            CBFM_CUDA(cudaMemcpyAsync(buf.p, v.data(), v.size() * sizeof(v[0]), cudaMemcpyHostToDevice, st));
    };
    up(ft->tl, ent);
    up(ft->dtl_off, ft->tl_off);
    up(ft->dch_off, ft->ch_off);
    up(ft->chunk, chunks);
    up(ft->chunk_cols, ccols);
    up(ft->rwg_pos, rpos);
    up(ft->near_row, rowc);
    up(ft->near_ent, ne);
    {
        const int64_t ntl = (int64_t)ent.size();
        ft->recT.alloc((size_t)std::max<int64_t>(1, ntl) * TRI_REC);
        ft->vidT.alloc((size_t)std::max<int64_t>(1, ntl) * 3);
        const unsigned g = (unsigned)std::min<int64_t>((ntl * TRI_REC + 255) / 256, 8 * (int64_t)sm_count());
        if (ntl) {
            k_tl_soa<<<g, 256, 0, st>>>(ntl, ft->tl.p, m.tri32.p, m.tri_vid.p, ft->recT.p, ft->vidT.p);
            launched("k_tl_soa");
        }
    }
    CBFM_CUDA(cudaStreamSynchronize(st));
    m.fused = ft;
    return *ft;
}

namespace {

FuPlan fu_plan(int lmax, int nmax) {
    FuPlan p;
    const int lp = (lmax + 1) & ~1;   // 4 lp rows per A image, a multiple of 8
    p.RA = std::max(8, 4 * lp);
    p.NP = std::max(16, (nmax + 15) & ~15);
    p.a_op = (uint32_t)p.RA * 64u;
    p.z_op = (uint32_t)p.NP * 64u;
    p.z_base = 12 * p.a_op;
    p.acc_base = p.z_base + 6 * p.z_op;
    p.acc_buf = 3u * FU_KC * 2u * (uint32_t)p.NP * 4u;
    // the last A image (buffer 1, lo, Tb) is read 128 rows deep: keep that inside the allocation
    p.total = std::max(p.acc_base + 2 * p.acc_buf, 11 * p.a_op + 128u * 64u);
    return p;
}

// CBF operand of every chunk of a mesh, in the shared-memory layout of the
// fused kernel: for chunk c (trial cell n, columns = its cell-local RWGs),
// plane (hi, lo) x operator (Ks, Ta, Tb) x 4 L_n rows x 16 floats, each 64-byte
// row swizzled.  Row r = 2 w + (re, im) expands CBF w of C^M_n (Ks rows [0, 2 L),
// Tb rows [2 L, 4 L)) or C^J_n (Ks rows [2 L, 4 L), Ta rows [0, 2 L)):
// (w, re) = (c_re, -c_im), (w, im) = (c_im, c_re) along the columns; the other
// half of Ta and Tb is zero.  TF32 split hi = tf32(x), lo = tf32(x - hi) of
// the FP64 coefficient.
__global__ void k_chunk_aimg(int nch, const int32_t *__restrict__ chunk_cell, const int64_t *__restrict__ off,
                             const int16_t *__restrict__ cols, const int32_t *__restrict__ L,
                             const int64_t *__restrict__ boff, const z64 *__restrict__ CM, const z64 *__restrict__ CJ,
                             float *__restrict__ img) {
    const int c = blockIdx.x;
    if (c >= nch) return;
    const int n = chunk_cell[c], Ln = L[n], rows = 4 * Ln;
    const int64_t bo = boff[n];
    float *dst = img + off[c];
    for (int idx = threadIdx.x; idx < 3 * rows * 16; idx += blockDim.x) {
        const int op = idx / (rows * 16), rem = idx - op * rows * 16;
        const int r = rem >> 4, f = rem & 15;
        const int col = f >> 1, comp = f & 1;
        const bool upper = r >= 2 * Ln;
        const int w = (r - (upper ? 2 * Ln : 0)) >> 1, ri = r & 1;
        const int jl = cols[(int64_t)c * FU_KC + col];
        const z64 *src = op == 0 ? (upper ? CJ : CM) : op == 1 ? (upper ? nullptr : CJ) : (upper ? CM : nullptr);
        double val = 0.0;
        if (src && jl >= 0) {
            const z64 q = src[bo + (int64_t)jl * Ln + w];
            val = ri == 0 ? (comp == 0 ? q.re : -q.im) : (comp == 0 ? q.im : q.re);
        }
        float hi, lo;
        split64(val, hi, lo);
        // swz64 gives the byte offset inside the operator's rows
        const uint32_t o = swz64(r, f) >> 2;
        dst[(int64_t)(0 * 3 + op) * rows * 16 + o] = hi;
        dst[(int64_t)(1 * 3 + op) * rows * 16 + o] = lo;
    }
}

}  // namespace

bool fused_fits(const Mesh &m, const Cbf &c) {
    int lmax = 0, nmax = 0;
    for (int k = 0; k < m.h.ncell; ++k) {
        lmax = std::max(lmax, c.L[k]);
        nmax = std::max(nmax, m.h.cell_off[k + 1] - m.h.cell_off[k]);
    }
    if (lmax > FU_LMAX || nmax > FU_NMAX) return false;
    return fu_plan(lmax, nmax).total + 1024 <= 227u * 1024u;
}

namespace {

// One launch of the fused kernel over the cell pairs of jobs [j0, j1) (their
// combined shared-memory plan fits).
void fused_launch(std::vector<FusedJob> &jobs, const std::vector<std::pair<double, int4>> &items_all, int j0, int j1,
                  int lmax, int nmax, cudaStream_t st) {
    std::vector<std::pair<double, int4>> items;
    for (const auto &it : items_all)
        if (it.second.x >= j0 && it.second.x < j1) items.push_back({it.first, make_int4(it.second.x - j0, it.second.y, it.second.z, 0)});
    if (items.empty()) return;
    // largest items first (the persistent CTAs take them in this order)
    std::stable_sort(items.begin(), items.end(), [](const auto &x, const auto &y) { return x.first > y.first; });
    std::vector<int4> hit(items.size());
    for (size_t i = 0; i < items.size(); ++i) hit[i] = items[i].second;
    const FuPlan plan = fu_plan(lmax, nmax);
    CBFM_REQUIRE(plan.total + 1024 <= 227u * 1024u, "fused assembly: shared-memory plan too large");
    const uint32_t tcols = 2 * plan.NP <= 256 ? 256u : 512u;
    const int nj = j1 - j0;
    DevBuf<FusedJob> djobs;
    DevBuf<int4> ditems;
    DevBuf<unsigned int> counter;
    DevBuf<int> err;
    djobs.alloc(nj);
    ditems.alloc(hit.size());
    counter.alloc(1);
    err.alloc(1);
    CBFM_CUDA(cudaMemcpyAsync(djobs.p, jobs.data() + j0, sizeof(FusedJob) * nj, cudaMemcpyHostToDevice, st));
    CBFM_CUDA(cudaMemcpyAsync(ditems.p, hit.data(), sizeof(int4) * hit.size(), cudaMemcpyHostToDevice, st));
    CBFM_CUDA(cudaMemsetAsync(counter.p, 0, sizeof(unsigned int), st));
    CBFM_CUDA(cudaMemsetAsync(err.p, 0, sizeof(int), st));
    const size_t smem = plan.total + 1024;
    CBFM_CUDA(cudaFuncSetAttribute(k_fused, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    const unsigned grid = (unsigned)std::min<int64_t>((int64_t)hit.size(), sm_count());
    {
        ProfScope ps_("k_fused", st);
        k_fused<<<grid, FU_THREADS, smem, st>>>(djobs.p, ditems.p, (int)hit.size(), counter.p, err.p, plan, tcols);
        launched("k_fused");
    }
    int herr = 0;
    CBFM_CUDA(cudaMemcpyAsync(&herr, err.p, sizeof(int), cudaMemcpyDeviceToHost, st));
    CBFM_CUDA(cudaStreamSynchronize(st));
    if (herr == 7) throw Fail{CBFM_ECUDA, "fused assembly: a near pair is missing from the near list"};
    if (herr) throw Fail{CBFM_ETIMEOUT, "fused assembly: a tensor-core wait expired (code " + std::to_string(herr) + ")"};
}

}  // namespace

double unfused_scratch_bytes(const Mesh &m, const Cbf &c) {
    const double nt = (double)m.h.nt, ne = (double)m.h.ne, nh = (double)c.nhalf;
    const double ldz = std::ceil(2.0 * ne / 32.0) * 32.0;
    return 27.0 * nt * nt * 8 + 3.0 * ne * ne * 8 + 6.0 * ne * ldz * 4 + 8.0 * 2 * nh * ldz * 4;
}

bool mixed_takes_fused(const Mesh &m, const Cbf &c) {
    if (!fused_fits(m, c)) return false;
    size_t free_b = 0, total_b = 0;
    if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) {
        cudaGetLastError();
        return true;
    }
    return unfused_scratch_bytes(m, c) > std::min(0.25 * (double)free_b, 16.0 * (1ull << 30));
}

void assemble_project_fused(const std::vector<Mesh *> &ms, const std::vector<Cbf *> &cs, const std::vector<c32 *> &A,
                            cudaStream_t st) {
    const int nj = (int)ms.size();
    if (nj == 0) return;
    // near-pair blocks (FP64 closed forms), compact, one launch for all meshes
    std::vector<DevBuf<c32>> nearv(nj);
    std::vector<c32 *> nearp(nj);
    for (int k = 0; k < nj; ++k) {
        nearv[k].alloc((size_t)std::max<int64_t>(1, ms[k]->n_near) * NCOMP);
        nearp[k] = nearv[k].p;
    }
    near_blocks_compact(ms, nearp, st);
    std::vector<FusedJob> jobs(nj);
    std::vector<std::pair<double, int4>> items;
    std::vector<DevBuf<int32_t>> dL(nj), dcoff32(nj);
    std::vector<DevBuf<int64_t>> dboff(nj), dcoff(nj);
    std::vector<DevBuf<float>> aimg(nj);
    std::vector<DevBuf<int32_t>> dcc(nj);
    std::vector<DevBuf<int64_t>> daoff(nj);
    std::vector<int> jl(nj, 0), jn(nj, 0);
    double far_flop = 0.0, bytes = 0.0;
    for (int k = 0; k < nj; ++k) {
        Mesh &m = *ms[k];
        Cbf &c = *cs[k];
        FusedTables &ft = fused_tables(m, st);
        const int nc = m.h.ncell;
        dL[k].alloc(nc);
        dboff[k].alloc(nc + 1);
        dcoff[k].alloc(nc + 1);
        dcoff32[k].alloc(nc + 1);
        CBFM_CUDA(cudaMemcpyAsync(dL[k].p, c.L.data(), 4 * nc, cudaMemcpyHostToDevice, st));
        CBFM_CUDA(cudaMemcpyAsync(dboff[k].p, c.boff.data(), 8 * (nc + 1), cudaMemcpyHostToDevice, st));
        CBFM_CUDA(cudaMemcpyAsync(dcoff[k].p, c.coff.data(), 8 * (nc + 1), cudaMemcpyHostToDevice, st));
        CBFM_CUDA(cudaMemcpyAsync(dcoff32[k].p, m.h.cell_off.data(), 4 * (nc + 1), cudaMemcpyHostToDevice, st));
        FusedJob &J = jobs[k];
        J.rec = m.tri32.p;
        J.rec64 = m.tri64.p;
        J.vid = m.tri_vid.p;
        J.recT = ft.recT.p;
        J.vidT = ft.vidT.p;
        J.ntl = ft.tl_off[nc];
        J.tl = ft.tl.p;
        J.tl_off = ft.dtl_off.p;
        J.ch_off = ft.dch_off.p;
        J.cell_off = dcoff32[k].p;
        J.chunk = ft.chunk.p;
        J.chunk_cols = ft.chunk_cols.p;
        J.near_row = ft.near_row.p;
        J.near_ent = ft.near_ent.p;
        J.near_val = nearp[k];
        {
            // CBF operand images of every chunk (float offsets 16-float aligned: 64-byte rows)
            const int nch = ft.ch_off[nc];
            std::vector<int32_t> ccell(std::max(1, nch));
            std::vector<int64_t> coffs(std::max(1, nch));
            int64_t tot = 0;
            for (int a = 0; a < nc; ++a)
                for (int q = ft.ch_off[a]; q < ft.ch_off[a + 1]; ++q) {
                    ccell[q] = a;
                    coffs[q] = tot;
                    tot += (int64_t)2 * 3 * 4 * c.L[a] * 16;
                }
            dcc[k].alloc(ccell.size());
            daoff[k].alloc(coffs.size());
            aimg[k].alloc((size_t)std::max<int64_t>(16, tot));
            CBFM_CUDA(cudaMemcpyAsync(dcc[k].p, ccell.data(), 4 * ccell.size(), cudaMemcpyHostToDevice, st));
            CBFM_CUDA(cudaMemcpyAsync(daoff[k].p, coffs.data(), 8 * coffs.size(), cudaMemcpyHostToDevice, st));
            CBFM_REQUIRE(((uintptr_t)aimg[k].p & 15) == 0, "fused assembly: operand images not 16-byte aligned");
            if (nch > 0) {
                k_chunk_aimg<<<nch, 256, 0, st>>>(nch, dcc[k].p, daoff[k].p, ft.chunk_cols.p, dL[k].p, dboff[k].p, c.CM.p,
                                                 c.CJ.p, aimg[k].p);
                launched("k_chunk_aimg");
            }
        }
        J.aimg = aimg[k].p;
        J.aimg_off = daoff[k].p;
        J.CM32 = c.CM32.p;
        J.CJ32 = c.CJ32.p;
        J.boff = dboff[k].p;
        J.coff = dcoff[k].p;
        J.L = dL[k].p;
        J.A = A[k];
        J.nh = c.nhalf;
        J.n = 2 * c.nhalf;
        J.md = media_t<float>(media_full(m.k1, m.k2, m.eta1, m.eta2));
        J.alpha = m.alpha;
        for (int a = 0; a < nc; ++a) {
            CBFM_REQUIRE(c.L[a] == 0 || ft.ch_off[a + 1] > ft.ch_off[a], "fused assembly: a cell with CBFs has no triangles");
            jl[k] = std::max(jl[k], c.L[a]);
            jn[k] = std::max(jn[k], m.h.cell_off[a + 1] - m.h.cell_off[a]);
            if (c.L[a] == 0) continue;
            const double ta = ft.tl_off[a + 1] - ft.tl_off[a];
            for (int b = 0; b < nc; ++b) {
                if (c.L[b] == 0) continue;
                const double tb = ft.tl_off[b + 1] - ft.tl_off[b];
                items.push_back({ta * tb, make_int4(k, a, b, 0)});
            }
        }
        CBFM_REQUIRE(jl[k] <= FU_LMAX && jn[k] <= FU_NMAX, "fused assembly: cell beyond the tile limits");
        const double ntd = (double)m.h.nt;
        far_flop += (ntd * ntd - (2.0 * m.n_near - ntd)) * 49.0 * FAR_FLOP_PER_POINT_PAIR;
        bytes += ntd * TRI_REC * 4 + (double)m.n_near * NCOMP * 8 + 2.0 * c.boff[nc] * 24 + (double)J.n * J.n * 8;
    }
    // launches over consecutive jobs whose combined shared-memory plan fits
    int j0 = 0;
    while (j0 < nj) {
        int j1 = j0 + 1, lmax = jl[j0], nmax = jn[j0];
        while (j1 < nj && fu_plan(std::max(lmax, jl[j1]), std::max(nmax, jn[j1])).total + 1024 <= 227u * 1024u) {
            lmax = std::max(lmax, jl[j1]);
            nmax = std::max(nmax, jn[j1]);
            ++j1;
        }
        fused_launch(jobs, items, j0, j1, lmax, nmax, st);
        j0 = j1;
    }
    prof_add_work("k_fused", far_flop, bytes);
}

}  // namespace cbfm
