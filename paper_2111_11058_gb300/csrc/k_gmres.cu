// k_gmres.cu -- batched right-preconditioned restarted GMRES on the reduced
// CBFM system A (G^CBF)^{-1} y = b (paper Eq. (CBFM_outer)); x = (G^CBF)^{-1} y
// (Eq. (CBFM_inner)).
//
// Every right-hand side runs its own GMRES (x0 = 0, Givens rotations, stop
// when ||b - A P y|| / ||b|| <= tol); the kernels process all of them at once
// and skip the ones that have converged.  The operator B = A P is formed once
// (cbfm_cmp_setup) so an iteration needs one product B v, done in FP64
// (CBFM_FP64) or with B in complex64 and FP32 accumulation (CBFM_MIXED).
// Arnoldi orthogonalisation, Hessenberg matrix and residual are FP64 in both:
// classical Gram-Schmidt with a second pass only where the first one
// cancelled strongly (||w_after|| < ||w_before|| / sqrt 2, the Daniel-Gragg-
// Kaufman-Stewart criterion).
#include <algorithm>
#include <vector>

#include "internal.cuh"

namespace cbfm {

namespace {

constexpr int JB = 8;          // basis vectors per block in k_dots
constexpr double DGKS_ETA = 0.70710678118654752;

__device__ __forceinline__ double block_sum(double v, double *sh) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
    __syncthreads();
    double s = 0;
    if (threadIdx.x == 0)
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) s += sh[i];
    return s;   // valid in thread 0
}

// h[r][j] = sum_i conj(V[j][r][i]) w[r][i], j = j0 + warp, for the columns with
// mask[r] != 0: one warp per basis vector (JB warps per block), four partial
// sums per lane to keep the FP64 pipe busy, warp-shuffle reduction only.  The
// x == 0 blocks also store ||w||^2 when nrm2 != NULL.
__global__ void __launch_bounds__(32 * JB) k_dots(int64_t n, int nrhs, int k, const z64 *__restrict__ V,
                                                  const z64 *__restrict__ w, z64 *__restrict__ h, int hld,
                                                  const int *__restrict__ mask, double *__restrict__ nrm2) {
    const int r = blockIdx.y;
    if (!mask[r]) return;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int j = blockIdx.x * JB + warp;
    const z64 *x = w + (int64_t)r * n;
    if (j <= k) {
        const z64 *v = V + ((int64_t)j * nrhs + r) * n;
        double re[4] = {0, 0, 0, 0}, im[4] = {0, 0, 0, 0};
        int64_t i = lane;
        for (; i + 96 < n; i += 128) {
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                z64 a = v[i + 32 * u], b = x[i + 32 * u];
                re[u] += a.re * b.re + a.im * b.im;
                im[u] += a.re * b.im - a.im * b.re;
            }
        }
        for (; i < n; i += 32) {
            z64 a = v[i], b = x[i];
            re[0] += a.re * b.re + a.im * b.im;
            im[0] += a.re * b.im - a.im * b.re;
        }
        double sr = (re[0] + re[1]) + (re[2] + re[3]), si = (im[0] + im[1]) + (im[2] + im[3]);
        for (int o = 16; o > 0; o >>= 1) {
            sr += __shfl_xor_sync(0xffffffffu, sr, o);
            si += __shfl_xor_sync(0xffffffffu, si, o);
        }
        if (lane == 0) h[(int64_t)r * hld + j] = z64(sr, si);
    }
    if (nrm2 && blockIdx.x == 0 && warp == JB - 1) {
        double s0 = 0, s1 = 0;
        int64_t i = lane;
        for (; i + 32 < n; i += 64) {
            s0 += norm2(x[i]);
            s1 += norm2(x[i + 32]);
        }
        for (; i < n; i += 32) s0 += norm2(x[i]);
        double s = s0 + s1;
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (lane == 0) nrm2[r] = s;
    }
}

// w[r][i] -= sum_{j<=k} V[j][r][i] h[r][j] for masked columns (four
// independent accumulator pairs per thread)
__global__ void __launch_bounds__(256) k_orth_update(int64_t n, int nrhs, int k, const z64 *__restrict__ V,
                                                     const z64 *__restrict__ h, int hld, const int *__restrict__ mask,
                                                     z64 *__restrict__ w) {
    const int r = blockIdx.y;
    if (!mask[r]) return;
    __shared__ z64 hs[1024];
    for (int j = threadIdx.x; j <= k; j += blockDim.x) hs[j] = h[(int64_t)r * hld + j];
    __syncthreads();
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const z64 *v = V + (int64_t)r * n + i;
    const int64_t stride = (int64_t)nrhs * n;
    z64 acc[4] = {w[(int64_t)r * n + i], z64(0, 0), z64(0, 0), z64(0, 0)};
    int j = 0;
    for (; j + 3 <= k; j += 4) {
#pragma unroll
        for (int u = 0; u < 4; ++u) acc[u] -= v[(j + u) * stride] * hs[j + u];
    }
    for (; j <= k; ++j) acc[0] -= v[j * stride] * hs[j];
    w[(int64_t)r * n + i] = (acc[0] + acc[1]) + (acc[2] + acc[3]);
}

// After the first pass: reorthogonalise where ||w|| dropped below eta ||w_before||.
// `flag` holds the active mask on entry and the reorthogonalisation mask on exit.
// `reo_work` accumulates (k + 1) for every reorthogonalised column (work of the second pass).
__global__ void k_reorth_flag(int64_t n, int nrhs, int k, const z64 *__restrict__ w,
                              const double *__restrict__ nrm2_before, int *__restrict__ flag,
                              unsigned long long *__restrict__ reo_work) {
    const int r = blockIdx.x;
    if (!flag[r]) return;
    double s = 0;
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) s += norm2(w[(int64_t)r * n + i]);
    __shared__ double sh[32];
    s = block_sum(s, sh);
    if (threadIdx.x == 0) {
        const int f = (sqrt(s) < DGKS_ETA * sqrt(nrm2_before[r])) ? 1 : 0;
        flag[r] = f;
        if (f) atomicAdd(reo_work, (unsigned long long)(k + 1));
    }
}

// Column k of H for every active rhs: h1 (+ h2 if reorthogonalised), ||w||;
// previous rotations, new rotation, residual, convergence; V[k+1] = w / ||w||.
// The column and the previous rotations are staged in shared memory so the
// sequential rotation sweep of thread 0 does not wait on global loads.
__global__ void __launch_bounds__(256) k_finish(int64_t n, int nrhs, int k, int m, int last,
                                                const z64 *__restrict__ h1, const z64 *__restrict__ h2,
                                                const int *__restrict__ flag, int hld, z64 *__restrict__ H,
                                                double *__restrict__ cs, z64 *__restrict__ sn, z64 *__restrict__ g,
                                                const double *__restrict__ bnorm, double tol, int *__restrict__ done,
                                                int *__restrict__ kconv, double *__restrict__ resid,
                                                int *__restrict__ n_active, const z64 *__restrict__ w,
                                                z64 *__restrict__ V) {
    const int r = blockIdx.x;
    if (done[r]) return;
    __shared__ z64 col[1024];
    __shared__ z64 ssn[1024];
    __shared__ double scs[1024];
    const bool re = flag[r] != 0;
    for (int j = threadIdx.x; j <= k; j += blockDim.x) {
        z64 v = h1[(int64_t)r * hld + j];
        if (re) v += h2[(int64_t)r * hld + j];
        col[j] = v;
        if (j < k) {
            scs[j] = cs[(int64_t)r * m + j];
            ssn[j] = sn[(int64_t)r * m + j];
        }
    }
    const z64 *x = w + (int64_t)r * n;
    double s = 0;
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) s += norm2(x[i]);
    __shared__ double sh[32];
    __shared__ double nrm;
    s = block_sum(s, sh);   // contains __syncthreads: col/scs/ssn are visible afterwards
    if (threadIdx.x == 0) {
        nrm = sqrt(s);
        z64 *gr = g + (int64_t)r * (m + 1);
        z64 a = col[0];
        for (int j = 0; j < k; ++j) {
            z64 b = col[j + 1];
            col[j] = scs[j] * a + ssn[j] * b;
            a = -(conj(ssn[j]) * a) + scs[j] * b;
        }
        // new rotation zeroing (a, nrm)
        double na = sqrt(norm2(a)), nb = nrm;
        double cc;
        z64 ss;
        if (nb == 0.0) { cc = 1.0; ss = z64(0, 0); }
        else if (na == 0.0) { cc = 0.0; ss = z64(1, 0); }
        else {
            double t = sqrt(na * na + nb * nb);
            cc = na / t;
            ss = a * (nb / (na * t));            // (a/|a|) nb / t, nb real
        }
        cs[(int64_t)r * m + k] = cc;
        sn[(int64_t)r * m + k] = ss;
        col[k] = cc * a + ss * nb;
        z64 gk = gr[k];
        gr[k] = cc * gk;
        gr[k + 1] = -(conj(ss) * gk);
        double res = sqrt(norm2(gr[k + 1])) / bnorm[r];
        resid[r] = res;
        if (res <= tol || nb == 0.0) {
            kconv[r] = k + 1;
            done[r] = 1;
        } else if (last) {
            kconv[r] = k + 1;
            done[r] = 2;
        } else {
            atomicAdd(n_active + k, 1);
        }
    }
    __syncthreads();
    {
        z64 *Hr = H + (int64_t)r * (m + 1) * m;
        for (int j = threadIdx.x; j <= k; j += blockDim.x) Hr[(int64_t)j * m + k] = col[j];
    }
    const double inv = (nrm > 0.0) ? 1.0 / nrm : 0.0;
    z64 *vn = V + ((int64_t)(k + 1) * nrhs + r) * n;
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) vn[i] = x[i] * inv;
}

// out[r] = M in[r] for the rows r with mask[r] != 0 (M n x n row-major; T is its
// storage and arithmetic type).  Tiles: 32 right-hand sides x 16 output rows,
// K steps of 32; 128 threads with 2 x 2 outputs each.
template <typename T>
__global__ void __launch_bounds__(128) k_matvec(int64_t n, int nrhs, const cx<T> *__restrict__ M,
                                                const z64 *__restrict__ in, z64 *__restrict__ out,
                                                const int *__restrict__ mask) {
    constexpr int BM = 32, BN = 16, BK = 32;
    __shared__ cx<T> Xs[BK][BM + 1];
    __shared__ cx<T> Ms[BK][BN + 1];
    const int tx = threadIdx.x % 8, ty = threadIdx.x / 8;   // ty 0..15, tx 0..7
    const int64_t r0 = (int64_t)blockIdx.y * BM, c0 = (int64_t)blockIdx.x * BN;
    cx<T> acc[2][2];
    for (int a = 0; a < 2; ++a)
        for (int b = 0; b < 2; ++b) acc[a][b] = cx<T>(0, 0);
    for (int64_t k0 = 0; k0 < n; k0 += BK) {
        for (int idx = threadIdx.x; idx < BM * BK; idx += 128) {
            int rr = idx / BK, kk = idx % BK;
            int64_t r = r0 + rr, kx = k0 + kk;
            cx<T> v(0, 0);
            if (r < nrhs && kx < n && mask[r]) {
                z64 e = in[r * n + kx];
                v = cx<T>((T)e.re, (T)e.im);
            }
            Xs[kk][rr] = v;
        }
        for (int idx = threadIdx.x; idx < BN * BK; idx += 128) {
            int cc = idx / BK, kk = idx % BK;
            int64_t c = c0 + cc, kx = k0 + kk;
            Ms[kk][cc] = (c < n && kx < n) ? M[c * n + kx] : cx<T>(0, 0);
        }
        __syncthreads();
#pragma unroll 8
        for (int kk = 0; kk < BK; ++kk) {
            cx<T> xa[2] = {Xs[kk][ty], Xs[kk][ty + 16]};
            cx<T> mb[2] = {Ms[kk][tx], Ms[kk][tx + 8]};
            for (int a = 0; a < 2; ++a)
                for (int b = 0; b < 2; ++b) cfma(acc[a][b], xa[a], mb[b]);
        }
        __syncthreads();
    }
    for (int a = 0; a < 2; ++a) {
        int64_t r = r0 + ty + 16 * a;
        if (r >= nrhs || !mask[r]) continue;
        for (int b = 0; b < 2; ++b) {
            int64_t c = c0 + tx + 8 * b;
            if (c < n) out[r * n + c] = z64((double)acc[a][b].re, (double)acc[a][b].im);
        }
    }
}

// Back-substitution H(0:kc,0:kc) z = g(0:kc), one block per rhs (column oriented).
__global__ void k_backsolve(int nrhs, int m, const z64 *__restrict__ H, z64 *__restrict__ g,
                            const int *__restrict__ kconv, const int *__restrict__ active, z64 *__restrict__ z) {
    const int r = blockIdx.x;
    if (!active[r]) return;
    const int kc = kconv[r];
    const z64 *Hr = H + (int64_t)r * (m + 1) * m;
    z64 *gr = g + (int64_t)r * (m + 1);
    z64 *zr = z + (int64_t)r * m;
    __shared__ z64 zj;
    for (int j = kc - 1; j >= 0; --j) {
        if (threadIdx.x == 0) {
            z64 d = Hr[(int64_t)j * m + j];
            zj = (norm2(d) > 0.0) ? cdiv(gr[j], d) : z64(0, 0);
            zr[j] = zj;
        }
        __syncthreads();
        for (int i = threadIdx.x; i < j; i += blockDim.x) gr[i] -= Hr[(int64_t)i * m + j] * zj;
        __syncthreads();
    }
}

// y[rhs] += sum_{j < kc} z_j V[j][rhs]
__global__ void k_update_y(int64_t n, int nrhs, int m, const z64 *__restrict__ V, const z64 *__restrict__ z,
                           const int *__restrict__ kconv, const int *__restrict__ active, z64 *__restrict__ y) {
    const int r = blockIdx.y;
    if (!active[r]) return;
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    z64 acc = y[(int64_t)r * n + i];
    for (int j = 0; j < kconv[r]; ++j) acc += V[((int64_t)j * nrhs + r) * n + i] * z[(int64_t)r * m + j];
    y[(int64_t)r * n + i] = acc;
}

// start of a cycle: r = b - w (w = B y, or 0), beta = ||r||, V[0] = r / beta, g = beta e1
__global__ void k_start(int64_t n, int nrhs, int m, const z64 *__restrict__ b, const z64 *__restrict__ w, int have_w,
                        z64 *__restrict__ V, z64 *__restrict__ g, const double *__restrict__ bnorm,
                        double *__restrict__ resid, int *__restrict__ done, double tol) {
    const int r = blockIdx.x;
    double s = 0;
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
        z64 v = b[(int64_t)r * n + i];
        if (have_w) v -= w[(int64_t)r * n + i];
        s += norm2(v);
    }
    __shared__ double sh[32];
    __shared__ double beta;
    s = block_sum(s, sh);
    if (threadIdx.x == 0) {
        beta = sqrt(s);
        z64 *gr = g + (int64_t)r * (m + 1);
        for (int j = 0; j <= m; ++j) gr[j] = z64(0, 0);
        gr[0] = z64(beta, 0);
        double res = (bnorm[r] > 0.0) ? beta / bnorm[r] : 0.0;
        resid[r] = res;
        if (done[r] != 1) done[r] = (res <= tol || beta == 0.0) ? 1 : 0;
    }
    __syncthreads();
    const double inv = (beta > 0.0) ? 1.0 / beta : 0.0;
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
        z64 v = b[(int64_t)r * n + i];
        if (have_w) v -= w[(int64_t)r * n + i];
        V[(int64_t)r * n + i] = v * inv;
    }
}

__global__ void k_norms(int64_t n, int nrhs, const z64 *__restrict__ b, double *__restrict__ out) {
    const int r = blockIdx.x;
    double s = 0;
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) s += norm2(b[(int64_t)r * n + i]);
    __shared__ double sh[32];
    s = block_sum(s, sh);
    if (threadIdx.x == 0) out[r] = sqrt(s);
}

// mask of the columns still iterating: done == 0
__global__ void k_active(int nrhs, const int *__restrict__ done, int *__restrict__ act) {
    int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r < nrhs) act[r] = done[r] == 0 ? 1 : 0;
}

__global__ void k_fill_ones(int nrhs, int *__restrict__ a) {
    int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r < nrhs) a[r] = 1;
}

}  // namespace

// out[r] = M in[r] for the rows with mask[r] != 0, in the precision of the reduced system
void apply_rows(const Red &rd, const z64 *M64, const c32 *M32, const z64 *in, z64 *out, int nrhs, const int *mask,
                cudaStream_t st) {
    const int64_t n = rd.n;
    dim3 grid((unsigned)((n + 15) / 16), (unsigned)((nrhs + 31) / 32));
    ProfScope ps_("k_matvec", st);
    if (M32) k_matvec<float><<<grid, 128, 0, st>>>(n, nrhs, M32, in, out, mask);
    else k_matvec<double><<<grid, 128, 0, st>>>(n, nrhs, M64, in, out, mask);
    launched("k_matvec");
}

// out[r] = mask[r] ? in[r] : 0 (rows of length n)
__global__ void k_mask_rows(int64_t n, int nrhs, const int *__restrict__ mask, const z64 *__restrict__ in,
                            z64 *__restrict__ out) {
    for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < n * nrhs;
         idx += (int64_t)gridDim.x * blockDim.x)
        out[idx] = mask[idx / n] ? in[idx] : z64(0, 0);
}

static void apply_B(Red &rd, int pc, const z64 *in, z64 *out, int nrhs, const int *mask, cudaStream_t st) {
    DevBuf<z64> v, z;
    if (pc == CBFM_PC_CMP_INEXACT) {   // A (G^CBF)^{-1} in: the inner GMRES, then the product with A
        // rows the mask leaves out may hold stale basis vectors: they enter the inner solve as zero
        v.alloc((size_t)nrhs * rd.n);
        z.alloc((size_t)nrhs * rd.n);
        const int64_t work = rd.n * nrhs;
        k_mask_rows<<<(unsigned)std::min<int64_t>((work + 255) / 256, 65535), 256, 0, st>>>(rd.n, nrhs, mask, in, v.p);
        launched("k_mask_rows");
        cmp_inner_apply(rd, v.p, z.p, nrhs, st);
        in = z.p;
    }
    if (rd.prec != CBFM_FP64) apply_rows(rd, nullptr, pc_op32(rd, pc), in, out, nrhs, mask, st);
    else apply_rows(rd, pc_op64(rd, pc), nullptr, in, out, nrhs, mask, st);
}

GmresOut gmres_solve(Red &rd, const z64 *d_b, int nrhs, double tol, int maxit, int restart, int pc, z64 *d_x,
                     cudaStream_t st) {
    const int64_t n = rd.n;
    CBFM_REQUIRE(nrhs <= 65535, "nrhs must be <= 65535");
    const int m = std::max(1, std::min<int>(std::min(restart, 1023),
                                            (int)std::min<int64_t>(maxit, std::max<int64_t>(n, 1))));
    DevBuf<z64> V, H, sn, g, y, w, hb1, hb2, zs;
    DevBuf<double> cs, bnorm, resid, nrm0;
    DevBuf<int> done, kconv, active, nact, flag, ones;
    DevBuf<unsigned long long> reo;
    reo.alloc(1);
    V.alloc((size_t)(m + 1) * nrhs * n);
    H.alloc((size_t)nrhs * (m + 1) * m);
    sn.alloc((size_t)nrhs * m);
    cs.alloc((size_t)nrhs * m);
    g.alloc((size_t)nrhs * (m + 1));
    y.alloc((size_t)nrhs * n);
    w.alloc((size_t)nrhs * n);
    hb1.alloc((size_t)nrhs * (m + 1));
    hb2.alloc((size_t)nrhs * (m + 1));
    zs.alloc((size_t)nrhs * m);
    bnorm.alloc(nrhs);
    resid.alloc(nrhs);
    nrm0.alloc(nrhs);
    done.alloc(nrhs);
    kconv.alloc(nrhs);
    active.alloc(nrhs);
    flag.alloc(nrhs);
    ones.alloc(nrhs);
    nact.alloc(m + 1);
    // the polled active count lands in a pinned word kept per host thread (one API call at a
    // time per thread), so a solve -- and every inner solve of the inexact CMP -- does no
    // host allocation and no cudaFreeHost
    struct PinnedWord {
        int *p = nullptr;
        ~PinnedWord() {
            if (p) cudaFreeHost(p);
        }
    };
    static thread_local PinnedWord t_nact;
    if (t_nact.p == nullptr) CBFM_CUDA(cudaMallocHost((void **)&t_nact.p, sizeof(int)));
    int *h_nact = t_nact.p;
    CBFM_CUDA(cudaMemsetAsync(y.p, 0, sizeof(z64) * nrhs * n, st));
    CBFM_CUDA(cudaMemsetAsync(H.p, 0, sizeof(z64) * nrhs * (m + 1) * m, st));
    CBFM_CUDA(cudaMemsetAsync(done.p, 0, sizeof(int) * nrhs, st));
    CBFM_CUDA(cudaMemsetAsync(reo.p, 0, sizeof(unsigned long long), st));
    double pass1 = 0.0, nmatvec = 0.0;   // algorithmic work counters (profiling)
    {
        ProfScope ps_("k_norms", st);
        k_norms<<<nrhs, 256, 0, st>>>(n, nrhs, d_b, bnorm.p);
        launched("k_norms");
    }
    {
        k_fill_ones<<<(nrhs + 127) / 128, 128, 0, st>>>(nrhs, ones.p);
        launched("k_fill_ones");
    }

    const int hld = m + 1;
    const int CHECK = 4;   // iterations between convergence polls
    std::vector<int> h_iters(nrhs, 0), h_done(nrhs, 0), h_kc(nrhs, 0), h_act(nrhs, 0);
    int total = 0;
    bool first = true;
    while (total < maxit) {
        if (!first) apply_B(rd, pc, y.p, w.p, nrhs, ones.p, st);
        {
            ProfScope ps_("k_start", st);
            k_start<<<nrhs, 256, 0, st>>>(n, nrhs, m, d_b, w.p, first ? 0 : 1, V.p, g.p, bnorm.p, resid.p, done.p,
                                          tol);
            launched("k_start");
        }
        first = false;
        CBFM_CUDA(cudaMemcpyAsync(h_done.data(), done.p, sizeof(int) * nrhs, cudaMemcpyDeviceToHost, st));
        CBFM_CUDA(cudaStreamSynchronize(st));
        int nrun = 0;
        for (int r = 0; r < nrhs; ++r) {
            h_act[r] = h_done[r] == 1 ? 0 : 1;
            nrun += h_act[r];
        }
        if (nrun == 0) break;
        CBFM_CUDA(cudaMemcpyAsync(active.p, h_act.data(), sizeof(int) * nrhs, cudaMemcpyHostToDevice, st));
        CBFM_CUDA(cudaMemsetAsync(kconv.p, 0, sizeof(int) * nrhs, st));
        CBFM_CUDA(cudaMemsetAsync(nact.p, 0, sizeof(int) * (m + 1), st));
        const int mc = std::min(m, maxit - total);
        int k = 0;
        for (; k < mc; ++k) {
            const z64 *vk = V.p + (int64_t)k * nrhs * n;
            {
                k_active<<<(nrhs + 127) / 128, 128, 0, st>>>(nrhs, done.p, flag.p);
                launched("k_active");
            }
            apply_B(rd, pc, vk, w.p, nrhs, flag.p, st);
            dim3 gd((unsigned)((k + 1 + JB - 1) / JB), nrhs), gu((unsigned)((n + 255) / 256), nrhs);
            {
                ProfScope ps_("k_dots", st);
                k_dots<<<gd, 32 * JB, 0, st>>>(n, nrhs, k, V.p, w.p, hb1.p, hld, flag.p, nrm0.p);
                launched("k_dots");
            }
            {
                ProfScope ps_("k_orth_update", st);
                k_orth_update<<<gu, 256, 0, st>>>(n, nrhs, k, V.p, hb1.p, hld, flag.p, w.p);
                launched("k_orth_update");
            }
            {
                ProfScope ps_("k_reorth_flag", st);
                k_reorth_flag<<<nrhs, 256, 0, st>>>(n, nrhs, k, w.p, nrm0.p, flag.p, reo.p);
                launched("k_reorth_flag");
            }
            {
                ProfScope ps_("k_dots", st);
                k_dots<<<gd, 32 * JB, 0, st>>>(n, nrhs, k, V.p, w.p, hb2.p, hld, flag.p, nullptr);
                launched("k_dots");
            }
            {
                ProfScope ps_("k_orth_update", st);
                k_orth_update<<<gu, 256, 0, st>>>(n, nrhs, k, V.p, hb2.p, hld, flag.p, w.p);
                launched("k_orth_update");
            }
            const int last = (k + 1 == mc) ? 1 : 0;
            {
                ProfScope ps_("k_finish", st);
                k_finish<<<nrhs, 256, 0, st>>>(n, nrhs, k, m, last, hb1.p, hb2.p, flag.p, hld, H.p, cs.p, sn.p, g.p,
                                               bnorm.p, tol, done.p, kconv.p, resid.p, nact.p, w.p, V.p);
                launched("k_finish");
            }
            if ((k + 1) % CHECK == 0 || last) {
                CBFM_CUDA(cudaMemcpyAsync(h_nact, nact.p + k, sizeof(int), cudaMemcpyDeviceToHost, st));
                CBFM_CUDA(cudaStreamSynchronize(st));
                if (*h_nact == 0) {
                    ++k;
                    break;
                }
            }
        }
        total += k;
        CBFM_CUDA(cudaMemcpyAsync(h_kc.data(), kconv.p, sizeof(int) * nrhs, cudaMemcpyDeviceToHost, st));
        CBFM_CUDA(cudaMemcpyAsync(h_done.data(), done.p, sizeof(int) * nrhs, cudaMemcpyDeviceToHost, st));
        CBFM_CUDA(cudaStreamSynchronize(st));
        for (int r = 0; r < nrhs; ++r)
            if (h_act[r]) {
                h_iters[r] += h_kc[r];
                pass1 += 0.5 * (double)h_kc[r] * (h_kc[r] + 1);
                nmatvec += h_kc[r] + 1;
            }
        {
            ProfScope ps_("k_backsolve", st);
            k_backsolve<<<nrhs, 128, 0, st>>>(nrhs, m, H.p, g.p, kconv.p, active.p, zs.p);
            launched("k_backsolve");
        }
        {
            dim3 gu((unsigned)((n + 255) / 256), nrhs);
            ProfScope ps_("k_update_y", st);
            k_update_y<<<gu, 256, 0, st>>>(n, nrhs, m, V.p, zs.p, kconv.p, active.p, y.p);
            launched("k_update_y");
        }
        bool all = true;
        for (int r = 0; r < nrhs; ++r) all &= (h_done[r] == 1);
        if (all) break;
        for (int r = 0; r < nrhs; ++r)
            if (h_done[r] == 2) h_done[r] = 0;
        CBFM_CUDA(cudaMemcpyAsync(done.p, h_done.data(), sizeof(int) * nrhs, cudaMemcpyHostToDevice, st));
        CBFM_CUDA(cudaMemsetAsync(H.p, 0, sizeof(z64) * nrhs * (m + 1) * m, st));
    }
    // x = P y
    if (pc == CBFM_PC_CMP) apply_rows(rd, rd.Ginv.p, nullptr, y.p, d_x, nrhs, ones.p, st);
    else if (pc == CBFM_PC_TDIAG) tdiag_recover(rd, y.p, d_x, nrhs, st);
    else if (pc == CBFM_PC_CMP_INEXACT) cmp_inner_apply(rd, y.p, d_x, nrhs, st);
    else CBFM_CUDA(cudaMemcpyAsync(d_x, y.p, sizeof(z64) * nrhs * n, cudaMemcpyDeviceToDevice, st));
    GmresOut out;
    out.iters = h_iters;
    out.resid.resize(nrhs);
    CBFM_CUDA(cudaMemcpyAsync(out.resid.data(), resid.p, sizeof(double) * nrhs, cudaMemcpyDeviceToHost, st));
    CBFM_CUDA(cudaMemcpyAsync(h_done.data(), done.p, sizeof(int) * nrhs, cudaMemcpyDeviceToHost, st));
    CBFM_CUDA(cudaStreamSynchronize(st));
    for (int r = 0; r < nrhs; ++r)
        if (h_done[r] != 1) out.iters[r] = -std::abs(out.iters[r]) - 1;   // marks non-convergence
    if (g_prof.load()) {
        unsigned long long p2 = 0;
        CBFM_CUDA(cudaMemcpy(&p2, reo.p, sizeof(p2), cudaMemcpyDeviceToHost));
        const double cb = sizeof(z64);
        // dot products and updates: 8 flops per complex multiply-add, one basis element read each
        prof_add_work("k_dots", 8.0 * n * (pass1 + p2), cb * n * (pass1 + p2));
        prof_add_work("k_orth_update", 8.0 * n * (pass1 + p2), cb * n * (pass1 + p2));
        const double eb = rd.prec != CBFM_FP64 ? sizeof(c32) : sizeof(z64);
        prof_add_work("k_matvec", 8.0 * n * n * (nmatvec + (pc == CBFM_PC_CMP ? nrhs : 0)), eb * n * n * (nmatvec + 1.0));
    }
    return out;
}

}  // namespace cbfm
