// T-diagonal arrangement and the conventional MoM matrix (paper Sec. IV, Eq. (MoM_T);
// Sec. IV-A, Eq. (cbfm_Tdiag)).
//
// The K-diagonal operator A (Eq. (Z) order: columns [alpha^M; alpha^J], or the
// reduced system's [M-coefficient; J-coefficient] CBFs) has its two column halves
// swapped by P (unknowns [alpha^J; alpha^M]): the diagonal blocks of A P hold the T
// operators.  With D = diag(A P) (Jacobi) or D = I the solver iterates with
//     Bt = A P D^{-1},   Bt[i][j] = A[i][p(j)] / D_j,   D_j = A[j][p(j)],
// where p(j) = j + n/2 (mod n) is its own inverse, and recovers
//     x = P D^{-1} y,    x_k = y_{p(k)} / D_{p(k)} = y_{p(k)} tdinv[k],
//     tdinv[k] = 1 / A[p(k)][k].
// With the swap switched off (p(k) = k) the same kernels give the plain Jacobi scaling A D^{-1},
// D = diag(A), which the inexact CMP's inner GMRES on G^CBF uses (the paper's D^CBF).
// Every kernel here is a grid-stride elementwise pass, bound by HBM bandwidth.
#include <algorithm>

#include "internal.cuh"

namespace cbfm {

namespace {

inline unsigned grid_for(int64_t work) {
    int64_t b = (work + 255) / 256;
    return (unsigned)std::max<int64_t>(1, std::min<int64_t>(b, 65535));
}

// p(k): the partner of k under the half swap (swap != 0), else k itself
__device__ __forceinline__ int64_t half_swap(int64_t k, int64_t h, int swap) {
    return swap ? (k < h ? k + h : k - h) : k;
}

template <typename T>
__global__ void k_tdiag_dinv(int64_t n, const cx<T> *__restrict__ A, int jacobi, int swap, z64 *__restrict__ tdinv,
                             int *__restrict__ zero_pivot) {
    const int64_t h = n / 2;
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
        z64 d(1.0, 0.0);
        if (jacobi) {
            const cx<T> a = A[half_swap(k, h, swap) * n + k];
            const z64 a64((double)a.re, (double)a.im);
            if (a64.re == 0.0 && a64.im == 0.0) {
                atomicExch(zero_pivot, 1);
                d = z64(0.0, 0.0);
            } else {
                d = cdiv(z64(1.0, 0.0), a64);
            }
        }
        tdinv[k] = d;
    }
}

// Bt[i][j] = A[i][p(j)] tdinv[p(j)]; the product in FP64, rounded once to T
template <typename T>
__global__ void k_tdiag_operator(int64_t n, const cx<T> *__restrict__ A, const z64 *__restrict__ tdinv, int swap,
                                 cx<T> *__restrict__ Bt) {
    const int64_t h = n / 2;
    for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < n * n;
         idx += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = idx / n, pj = half_swap(idx % n, h, swap);
        const cx<T> a = A[i * n + pj];
        const z64 s = tdinv[pj];
        const double re = (double)a.re * s.re - (double)a.im * s.im;
        const double im = (double)a.re * s.im + (double)a.im * s.re;
        Bt[idx] = cx<T>((T)re, (T)im);
    }
}

__global__ void k_tdiag_recover(int64_t n, int64_t nrhs, const z64 *__restrict__ tdinv, int swap,
                                const z64 *__restrict__ y, z64 *__restrict__ x) {
    const int64_t h = n / 2;
    for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < nrhs * n;
         idx += (int64_t)gridDim.x * blockDim.x) {
        const int64_t q = idx / n, k = idx % n;
        x[idx] = y[q * n + half_swap(k, h, swap)] * tdinv[k];
    }
}

// A = [[Ks, Ta], [Tb, Ks]] from Z = (Ks, Ta, Tb), each ne x ne row-major
template <typename T>
__global__ void k_mom_place(int64_t ne, const cx<T> *__restrict__ Z, cx<T> *__restrict__ A) {
    const int64_t n = 2 * ne;
    for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < n * n;
         idx += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = idx / n, j = idx % n;
        const int hi = i >= ne, hj = j >= ne;
        const int op = hi == hj ? 0 : (hi ? 2 : 1);
        A[idx] = Z[op * ne * ne + (i - hi * ne) * ne + (j - hj * ne)];
    }
}

// out[(a ne + r)][(b ne + c)] = A[(a ne + int(r))][(b ne + int(c))] for canonical edges r, c
__global__ void k_mom_canon(int64_t ne, const int32_t *__restrict__ int_of_canon, const z64 *__restrict__ A,
                            z64 *__restrict__ out) {
    const int64_t n = 2 * ne;
    for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < n * n;
         idx += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = idx / n, j = idx % n;
        const int64_t hi = i >= ne ? ne : 0, hj = j >= ne ? ne : 0;
        out[idx] = A[(hi + int_of_canon[i - hi]) * n + hj + int_of_canon[j - hj]];
    }
}

}  // namespace

bool tdiag_build(Red &r, bool jacobi, cudaStream_t st, bool swap) {
    const int64_t n = r.n;
    CBFM_REQUIRE(n > 0 && (!swap || n % 2 == 0), "the system has no two halves to swap");
    const int sw = swap ? 1 : 0;
    DevBuf<int> flag;
    flag.alloc(1);
    CBFM_CUDA(cudaMemsetAsync(flag.p, 0, sizeof(int), st));
    r.tdiag_ready = false;
    r.tdinv.alloc((size_t)n);
    const bool f64 = r.prec == CBFM_FP64;
    {
        ProfScope ps_("k_tdiag_dinv", st);
        if (f64) k_tdiag_dinv<double><<<grid_for(n), 256, 0, st>>>(n, r.A64.p, jacobi ? 1 : 0, sw, r.tdinv.p, flag.p);
        else k_tdiag_dinv<float><<<grid_for(n), 256, 0, st>>>(n, r.A32.p, jacobi ? 1 : 0, sw, r.tdinv.p, flag.p);
        launched("k_tdiag_dinv");
    }
    {
        ProfScope ps_("k_tdiag_operator", st);
        if (f64) {
            r.Bt32.release();
            r.Bt64.alloc((size_t)n * n);
            k_tdiag_operator<double><<<grid_for(n * n), 256, 0, st>>>(n, r.A64.p, r.tdinv.p, sw, r.Bt64.p);
        } else {
            r.Bt64.release();
            r.Bt32.alloc((size_t)n * n);
            k_tdiag_operator<float><<<grid_for(n * n), 256, 0, st>>>(n, r.A32.p, r.tdinv.p, sw, r.Bt32.p);
        }
        launched("k_tdiag_operator");
    }
    int h = 0;
    CBFM_CUDA(cudaMemcpyAsync(&h, flag.p, sizeof(int), cudaMemcpyDeviceToHost, st));
    CBFM_CUDA(cudaStreamSynchronize(st));
    if (h) return false;
    r.tdiag_ready = true;
    r.tdiag_jacobi = jacobi;
    r.tdiag_swap = swap;
    return true;
}

void tdiag_recover(const Red &r, const z64 *y, z64 *x, int nrhs, cudaStream_t st) {
    ProfScope ps_("k_tdiag_recover", st);
    k_tdiag_recover<<<grid_for(r.n * nrhs), 256, 0, st>>>(r.n, nrhs, r.tdinv.p, r.tdiag_swap ? 1 : 0, y, x);
    launched("k_tdiag_recover");
}

void cmp_inner_apply(Red &r, const z64 *v, z64 *z, int nrhs, cudaStream_t st) {
    // the inner iterate is used as it stands when inner_maxit is reached (an inexact preconditioner)
    gmres_solve(*r.ginner, v, nrhs, r.inner_tol, r.inner_maxit, r.inner_restart, CBFM_PC_TDIAG, z, st);
}

template <typename T>
void mom_place(int64_t ne, const cx<T> *Z, cx<T> *A, cudaStream_t st) {
    ProfScope ps_("k_mom_place", st);
    k_mom_place<T><<<grid_for(4 * ne * ne), 256, 0, st>>>(ne, Z, A);
    launched("k_mom_place");
}
template void mom_place<double>(int64_t, const z64 *, z64 *, cudaStream_t);
template void mom_place<float>(int64_t, const c32 *, c32 *, cudaStream_t);

void mom_to_canonical(int64_t ne, const int32_t *d_int_of_canon, const z64 *A, z64 *out, cudaStream_t st) {
    ProfScope ps_("k_mom_canon", st);
    k_mom_canon<<<grid_for(4 * ne * ne), 256, 0, st>>>(ne, d_int_of_canon, A, out);
    launched("k_mom_canon");
}

}  // namespace cbfm
