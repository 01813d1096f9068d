// k_gmres.cu -- batched right-preconditioned restarted GMRES on the reduced
// CBFM system A (G^CBF)^{-1} y = b (paper Eq. (CBFM_outer)); x = (G^CBF)^{-1} y
// (Eq. (CBFM_inner)).  Every right-hand side runs its own GMRES: x0 = 0,
// classical Gram-Schmidt with one reorthogonalisation (CGS2) in FP64, Givens
// rotations, stop when ||b - A P y|| / ||b|| <= tol.  The operator product
// A P v runs in FP64 (CBFM_FP64) or complex64 with FP32 accumulation
// (CBFM_MIXED); Arnoldi, Hessenberg and residual stay FP64 in both.
#include <algorithm>
#include <vector>

#include "internal.cuh"

namespace cbfm {

namespace {

// h[rhs][j] = sum_i conj(V[j][rhs][i]) w[rhs][i], j = 0..k
__global__ void k_dots(int64_t n, int nrhs, const z64 *__restrict__ V, const z64 *__restrict__ w,
                       z64 *__restrict__ h, int hld) {
    const int j = blockIdx.x, r = blockIdx.y;
    const z64 *v = V + ((int64_t)j * nrhs + r) * n;
    const z64 *x = w + (int64_t)r * n;
    double re = 0, im = 0;
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
        z64 a = v[i], b = x[i];
        re += a.re * b.re + a.im * b.im;
        im += a.re * b.im - a.im * b.re;
    }
    __shared__ double sre[32], sim[32];
    for (int o = 16; o > 0; o >>= 1) {
        re += __shfl_down_sync(0xffffffffu, re, o);
        im += __shfl_down_sync(0xffffffffu, im, o);
    }
    if ((threadIdx.x & 31) == 0) { sre[threadIdx.x >> 5] = re; sim[threadIdx.x >> 5] = im; }
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0, b = 0;
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) { a += sre[i]; b += sim[i]; }
        h[(int64_t)r * hld + j] = z64(a, b);
    }
}

// w[rhs][i] -= sum_{j<=k} V[j][rhs][i] h[rhs][j]
__global__ void k_orth_update(int64_t n, int nrhs, int k, const z64 *__restrict__ V, const z64 *__restrict__ h,
                              int hld, z64 *__restrict__ w) {
    const int r = blockIdx.y;
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    z64 acc = w[(int64_t)r * n + i];
    for (int j = 0; j <= k; ++j) acc -= V[((int64_t)j * nrhs + r) * n + i] * h[(int64_t)r * hld + j];
    w[(int64_t)r * n + i] = acc;
}

// H[rhs][j][k] += h1 + h2 for j <= k; then ||w|| -> H[k+1][k], V[k+1] = w/||w||
__global__ void k_norm_next(int64_t n, int nrhs, int k, int m, const z64 *__restrict__ h1, const z64 *__restrict__ h2,
                            int hld, z64 *__restrict__ H, const z64 *__restrict__ w, z64 *__restrict__ V) {
    const int r = blockIdx.x;
    const z64 *x = w + (int64_t)r * n;
    double s = 0;
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) s += norm2(x[i]);
    __shared__ double red[32];
    __shared__ double nrm;
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0;
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) a += red[i];
        nrm = sqrt(a);
        z64 *Hr = H + (int64_t)r * (m + 1) * m;
        for (int j = 0; j <= k; ++j) Hr[(int64_t)j * m + k] = h1[(int64_t)r * hld + j] + h2[(int64_t)r * hld + j];
        Hr[(int64_t)(k + 1) * m + k] = z64(nrm, 0);
    }
    __syncthreads();
    const double inv = (nrm > 0.0) ? 1.0 / nrm : 0.0;
    z64 *vn = V + ((int64_t)(k + 1) * nrhs + r) * n;
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) vn[i] = x[i] * inv;
}

// Givens update of column k for every active rhs; marks convergence.
__global__ void k_givens(int nrhs, int k, int m, int last, z64 *__restrict__ H, double *__restrict__ cs, z64 *__restrict__ sn,
                         z64 *__restrict__ g, const double *__restrict__ bnorm, double tol, int *__restrict__ done,
                         int *__restrict__ kconv, double *__restrict__ resid, int *__restrict__ n_active) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= nrhs) return;
    if (done[r]) return;
    z64 *Hr = H + (int64_t)r * (m + 1) * m;
    double *c = cs + (int64_t)r * m;
    z64 *s = sn + (int64_t)r * m;
    z64 *gr = g + (int64_t)r * (m + 1);
    for (int j = 0; j < k; ++j) {
        z64 a = Hr[(int64_t)j * m + k], b = Hr[(int64_t)(j + 1) * m + k];
        Hr[(int64_t)j * m + k] = c[j] * a + s[j] * b;
        Hr[(int64_t)(j + 1) * m + k] = -(conj(s[j]) * a) + c[j] * b;
    }
    z64 a = Hr[(int64_t)k * m + k], b = Hr[(int64_t)(k + 1) * m + k];
    double na = sqrt(norm2(a)), nb = sqrt(norm2(b));
    double cc;
    z64 ss;
    if (nb == 0.0) { cc = 1.0; ss = z64(0, 0); }
    else if (na == 0.0) { cc = 0.0; ss = cdiv(conj(b), z64(nb, 0)); }
    else {
        double t = sqrt(na * na + nb * nb);
        cc = na / t;
        z64 ph = a * (1.0 / na);                  // a / |a|
        ss = ph * conj(b) * (1.0 / t);
    }
    c[k] = cc;
    s[k] = ss;
    Hr[(int64_t)k * m + k] = cc * a + ss * b;
    Hr[(int64_t)(k + 1) * m + k] = z64(0, 0);
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
        done[r] = 2;   // end of cycle without convergence
    }
    if (done[r] == 0) atomicAdd(n_active, 1);
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
    for (int j = kc - 1; j >= 0; --j) {
        __shared__ z64 zj;
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

// start of a cycle: r = b - w (w = A P y, or 0), beta = ||r||, V[0] = r / beta, g = beta e1
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
    __shared__ double red[32];
    __shared__ double beta;
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0;
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) a += red[i];
        beta = sqrt(a);
        z64 *gr = g + (int64_t)r * (m + 1);
        for (int j = 0; j <= m; ++j) gr[j] = z64(0, 0);
        gr[0] = z64(beta, 0);
        double res = (bnorm[r] > 0.0) ? beta / bnorm[r] : 0.0;
        resid[r] = res;
        // a column that already converged stays done
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
    __shared__ double red[32];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0;
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) a += red[i];
        out[r] = sqrt(a);
    }
}

}  // namespace

// out (nrhs x n) = in (nrhs x n) * M^T, i.e. out[r] = M in[r], in FP64 or FP32.
static void apply_rows(const Red &r, bool mixed, const z64 *Mat64, const c32 *Mat32, const z64 *in, z64 *out, int nrhs,
                       DevBuf<c32> &t_in, DevBuf<c32> &t_out, cudaStream_t st) {
    const int64_t n = r.n;
    std::vector<GemmDesc> g{GemmDesc{nrhs, n, n, 0, n, 0, n, 0, n}};
    if (!mixed) {
        gemm_grouped<double>(g, 0, 1, in, Mat64, out, false, st);
    } else {
        launch_z64_to_c32(in, t_in.p, n * nrhs, st);
        gemm_grouped<float>(g, 0, 1, t_in.p, Mat32, t_out.p, false, st);
        launch_c32_to_z64(t_out.p, out, n * nrhs, st);
    }
}

GmresOut gmres_solve(Red &rd, const z64 *d_b, int nrhs, double tol, int maxit, int restart, bool use_cmp, z64 *d_x,
                     cudaStream_t st) {
    const int64_t n = rd.n;
    const int m = std::max(1, std::min<int>(restart, (int)std::min<int64_t>(maxit, std::max<int64_t>(n, 1))));
    const bool mixed = rd.prec == CBFM_MIXED;
    DevBuf<z64> V, H, sn, g, y, w, z, hb1, hb2, zs;
    DevBuf<double> cs, bnorm, resid;
    DevBuf<int> done, kconv, active, nact;
    DevBuf<c32> t_in, t_out;
    V.alloc((size_t)(m + 1) * nrhs * n);
    H.alloc((size_t)nrhs * (m + 1) * m);
    sn.alloc((size_t)nrhs * m);
    cs.alloc((size_t)nrhs * m);
    g.alloc((size_t)nrhs * (m + 1));
    y.alloc((size_t)nrhs * n);
    w.alloc((size_t)nrhs * n);
    z.alloc((size_t)nrhs * n);
    hb1.alloc((size_t)nrhs * (m + 1));
    hb2.alloc((size_t)nrhs * (m + 1));
    zs.alloc((size_t)nrhs * m);
    bnorm.alloc(nrhs);
    resid.alloc(nrhs);
    done.alloc(nrhs);
    kconv.alloc(nrhs);
    active.alloc(nrhs);
    nact.alloc(1);
    if (mixed) {
        t_in.alloc((size_t)nrhs * n);
        t_out.alloc((size_t)nrhs * n);
    }
    CBFM_CUDA(cudaMemsetAsync(y.p, 0, sizeof(z64) * nrhs * n, st));
    CBFM_CUDA(cudaMemsetAsync(H.p, 0, sizeof(z64) * nrhs * (m + 1) * m, st));
    CBFM_CUDA(cudaMemsetAsync(done.p, 0, sizeof(int) * nrhs, st));
    {
        ProfScope ps_("k_norms", st);
        k_norms<<<nrhs, 256, 0, st>>>(n, nrhs, d_b, bnorm.p);
        launched("k_norms");
    }

    const int hld = m + 1;
    std::vector<int> h_iters(nrhs, 0), h_done(nrhs, 0), h_kc(nrhs, 0), h_act(nrhs, 0);
    int total = 0;
    bool first = true;
    while (total < maxit) {
        // residual of the current iterate
        if (!first) {
            if (use_cmp) {
                apply_rows(rd, mixed, rd.Ginv.p, rd.Ginv32.p, y.p, z.p, nrhs, t_in, t_out, st);
                apply_rows(rd, mixed, rd.A64.p, rd.A32.p, z.p, w.p, nrhs, t_in, t_out, st);
            } else {
                apply_rows(rd, mixed, rd.A64.p, rd.A32.p, y.p, w.p, nrhs, t_in, t_out, st);
            }
        }
        {
            ProfScope ps_("k_start", st);
            k_start<<<nrhs, 256, 0, st>>>(n, nrhs, m, d_b, w.p, first ? 0 : 1, V.p, g.p, bnorm.p, resid.p, done.p, tol);
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
        const int mc = std::min(m, maxit - total);
        int k = 0;
        for (; k < mc; ++k) {
            const z64 *vk = V.p + (int64_t)k * nrhs * n;
            if (use_cmp) {
                apply_rows(rd, mixed, rd.Ginv.p, rd.Ginv32.p, vk, z.p, nrhs, t_in, t_out, st);
                apply_rows(rd, mixed, rd.A64.p, rd.A32.p, z.p, w.p, nrhs, t_in, t_out, st);
            } else {
                apply_rows(rd, mixed, rd.A64.p, rd.A32.p, vk, w.p, nrhs, t_in, t_out, st);
            }
            dim3 gd(k + 1, nrhs), gu((unsigned)((n + 255) / 256), nrhs);
            {
                ProfScope ps_("k_dots", st);
                k_dots<<<gd, 256, 0, st>>>(n, nrhs, V.p, w.p, hb1.p, hld);
                launched("k_dots");
            }
            {
                ProfScope ps_("k_orth_update", st);
                k_orth_update<<<gu, 256, 0, st>>>(n, nrhs, k, V.p, hb1.p, hld, w.p);
                launched("k_orth_update");
            }
            {
                ProfScope ps_("k_dots", st);
                k_dots<<<gd, 256, 0, st>>>(n, nrhs, V.p, w.p, hb2.p, hld);
                launched("k_dots");
            }
            {
                ProfScope ps_("k_orth_update", st);
                k_orth_update<<<gu, 256, 0, st>>>(n, nrhs, k, V.p, hb2.p, hld, w.p);
                launched("k_orth_update");
            }
            {
                ProfScope ps_("k_norm_next", st);
                k_norm_next<<<nrhs, 256, 0, st>>>(n, nrhs, k, m, hb1.p, hb2.p, hld, H.p, w.p, V.p);
                launched("k_norm_next");
            }
            CBFM_CUDA(cudaMemsetAsync(nact.p, 0, sizeof(int), st));
            // the last step of a cycle closes every active column
            const int last = (k + 1 == mc) ? 1 : 0;
            {
                ProfScope ps_("k_givens", st);
                k_givens<<<(nrhs + 127) / 128, 128, 0, st>>>(nrhs, k, m, last, H.p, cs.p, sn.p, g.p, bnorm.p, tol, done.p,
                                                              kconv.p, resid.p, nact.p);
                launched("k_givens");
            }
            int na = 0;
            CBFM_CUDA(cudaMemcpyAsync(&na, nact.p, sizeof(int), cudaMemcpyDeviceToHost, st));
            CBFM_CUDA(cudaStreamSynchronize(st));
            if (na == 0) { ++k; break; }
        }
        total += k;
        CBFM_CUDA(cudaMemcpyAsync(h_kc.data(), kconv.p, sizeof(int) * nrhs, cudaMemcpyDeviceToHost, st));
        CBFM_CUDA(cudaMemcpyAsync(h_done.data(), done.p, sizeof(int) * nrhs, cudaMemcpyDeviceToHost, st));
        CBFM_CUDA(cudaStreamSynchronize(st));
        for (int r = 0; r < nrhs; ++r)
            if (h_act[r]) h_iters[r] += h_kc[r];
        {
            ProfScope ps_("k_backsolve", st);
            k_backsolve<<<nrhs, 128, 0, st>>>(nrhs, m, H.p, g.p, kconv.p, active.p, zs.p);
            launched("k_backsolve");
        }
        dim3 gu((unsigned)((n + 255) / 256), nrhs);
        {
            ProfScope ps_("k_update_y", st);
            k_update_y<<<gu, 256, 0, st>>>(n, nrhs, m, V.p, zs.p, kconv.p, active.p, y.p);
            launched("k_update_y");
        }
        bool all = true;
        for (int r = 0; r < nrhs; ++r) all &= (h_done[r] == 1);
        if (all) break;
        // columns that ended the cycle unconverged restart from their iterate
        for (int r = 0; r < nrhs; ++r)
            if (h_done[r] == 2) h_done[r] = 0;
        CBFM_CUDA(cudaMemcpyAsync(done.p, h_done.data(), sizeof(int) * nrhs, cudaMemcpyHostToDevice, st));
        CBFM_CUDA(cudaMemsetAsync(H.p, 0, sizeof(z64) * nrhs * (m + 1) * m, st));
    }
    // x = P y
    if (use_cmp) apply_rows(rd, mixed, rd.Ginv.p, rd.Ginv32.p, y.p, d_x, nrhs, t_in, t_out, st);
    else CBFM_CUDA(cudaMemcpyAsync(d_x, y.p, sizeof(z64) * nrhs * n, cudaMemcpyDeviceToDevice, st));
    GmresOut out;
    out.iters = h_iters;
    out.resid.resize(nrhs);
    CBFM_CUDA(cudaMemcpyAsync(out.resid.data(), resid.p, sizeof(double) * nrhs, cudaMemcpyDeviceToHost, st));
    CBFM_CUDA(cudaMemcpyAsync(h_done.data(), done.p, sizeof(int) * nrhs, cudaMemcpyDeviceToHost, st));
    CBFM_CUDA(cudaStreamSynchronize(st));
    for (int r = 0; r < nrhs; ++r)
        if (h_done[r] != 1) out.iters[r] = -std::abs(out.iters[r]) - 1;   // marks non-convergence
    return out;
}

}  // namespace cbfm
