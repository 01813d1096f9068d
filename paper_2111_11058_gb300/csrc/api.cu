// api.cu -- the C ABI (include/cbfm.h): handles, argument checks, error
// reporting and the orchestration of the kernels of each step.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <complex>
#include <memory>
#include <cstring>
#include <new>
#include <map>
#include <mutex>
#include <numeric>

#include "internal.cuh"

namespace cbfm {

std::atomic<int64_t> g_launches{0};
thread_local CallStream g_call;

// tuned launch parameters (first use on a device picks them by timing)
namespace {
std::mutex g_tune_mu;
std::map<std::string, int> g_tune;
}  // namespace

int tuning_get(const std::string &key) {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tune.find(key);
    return it == g_tune.end() ? 0 : it->second;
}

void tuning_set(const std::string &key, int value) {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tune[key] = value;
}

void pool_setup() {
    static std::atomic<uint64_t> done{0};   // one bit per device
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return;
    if (done.load(std::memory_order_acquire) & (1ull << dev)) return;
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
        uint64_t keep = 8ull << 30;   // freed scratch stays cached up to 8 GiB between calls
        cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
    }
    noalloc_prepare();   // the no-alloc export's scratch is taken now, not when memory may be full
    done.fetch_or(1ull << dev, std::memory_order_acq_rel);
}
std::atomic<bool> g_prof{false};
static thread_local std::string t_err;

// ------------------------------------------------------ kernel timing
namespace {
struct PendingEv {
    std::string name;
    cudaEvent_t a, b;
};
struct ProfAcc {
    int64_t launches = 0;
    double ms = 0.0;
    double flop = 0.0;
    double bytes = 0.0;
};
std::mutex g_prof_mu;
std::vector<PendingEv> g_pending;
std::map<std::string, ProfAcc> g_acc;
}  // namespace

int prof_start(const char *name, cudaStream_t st) {
    cudaEvent_t a, b;
    if (cudaEventCreate(&a) != cudaSuccess) return -1;
    if (cudaEventCreate(&b) != cudaSuccess) {
        cudaEventDestroy(a);
        return -1;
    }
    cudaEventRecord(a, st);
    std::lock_guard<std::mutex> lk(g_prof_mu);
    g_pending.push_back(PendingEv{name, a, b});
    return (int)g_pending.size() - 1;
}

void prof_stop(int token, cudaStream_t st) {
    std::lock_guard<std::mutex> lk(g_prof_mu);
    if (token >= 0 && token < (int)g_pending.size()) cudaEventRecord(g_pending[token].b, st);
}

void prof_add_work(const char *name, double flop, double bytes) {
    if (!g_prof.load()) return;
    std::lock_guard<std::mutex> lk(g_prof_mu);
    ProfAcc &a = g_acc[name];
    a.flop += flop;
    a.bytes += bytes;
}

void prof_flush() {
    std::lock_guard<std::mutex> lk(g_prof_mu);
    for (auto &p : g_pending) {
        float ms = 0.f;
        if (cudaEventSynchronize(p.b) == cudaSuccess && cudaEventElapsedTime(&ms, p.a, p.b) == cudaSuccess) {
            ProfAcc &acc = g_acc[p.name];
            acc.launches += 1;
            acc.ms += ms;
        }
        cudaEventDestroy(p.a);
        cudaEventDestroy(p.b);
    }
    g_pending.clear();
}

void set_error(const std::string &msg) { t_err = msg; }

int sm_count() {
    static std::atomic<int> cache[64];   // zero-initialised (static storage)
    int dev = 0;
    CBFM_CUDA(cudaGetDevice(&dev));
    if (dev >= 0 && dev < 64) {
        const int c = cache[dev].load(std::memory_order_relaxed);
        if (c > 0) return c;
    }
    int n = 0;
    CBFM_CUDA(cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev));
    if (dev >= 0 && dev < 64) cache[dev].store(n, std::memory_order_relaxed);
    return n;
}

bool is_device_ptr(const void *p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

void copy_in(void *dst_dev, const void *src_any, size_t bytes, cudaStream_t st) {
    if (bytes) CBFM_CUDA(cudaMemcpyAsync(dst_dev, src_any, bytes, cudaMemcpyDefault, st));
}
void copy_out(void *dst_any, const void *src_dev, size_t bytes, cudaStream_t st) {
    if (bytes) CBFM_CUDA(cudaMemcpyAsync(dst_any, src_dev, bytes, cudaMemcpyDefault, st));
}

namespace {

// ------------------------------------------------------- helper kernels
// Z_mm = [[Ks, Ta], [Tb, Ks]] restricted to the cell's edges (paper Eq. (pcbf)).
// V_m = [vE(Lambda_m); vH(Lambda_m)]
__global__ void k_extract_v(int ncell, const int32_t *__restrict__ cell_off, const int64_t *__restrict__ voff, int s,
                            const z64 *__restrict__ vE, const z64 *__restrict__ vH, z64 *__restrict__ out) {
    const int c = blockIdx.y;
    const int64_t off = cell_off[c], N = cell_off[c + 1] - off;
    for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < 2 * N * s;
         idx += (int64_t)gridDim.x * blockDim.x) {
        int64_t i = idx / s, w = idx % s;
        out[voff[c] + idx] = (i < N) ? vE[(off + i) * s + w] : vH[(off + i - N) * s + w];
    }
}

// IPCBF coefficient sets: [J^M; J^J] of cell c from the whole-system solutions x (s rows of
// [alpha^M; alpha^J], length 2 ne, internal edge order)
__global__ void k_ipcbf_gather(int ncell, const int32_t *__restrict__ cell_off, const int64_t *__restrict__ voff,
                               int s, int64_t ne, const z64 *__restrict__ x, z64 *__restrict__ out) {
    const int c = blockIdx.y;
    const int64_t off = cell_off[c], N = cell_off[c + 1] - off;
    for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < 2 * N * s;
         idx += (int64_t)gridDim.x * blockDim.x) {
        int64_t i = idx / s, w = idx % s;
        out[voff[c] + idx] = x[w * 2 * ne + (i < N ? off + i : ne + off + i - N)];
    }
}

// dense G_m (N_m x N_m) of every cell from the sparse Gram rows
__global__ void k_cell_gram(int ncell, const int32_t *__restrict__ cell_off, const int64_t *__restrict__ goff,
                            const double *__restrict__ val, const int32_t *__restrict__ col, z64 *__restrict__ G) {
    const int c = blockIdx.y;
    const int64_t off = cell_off[c], N = cell_off[c + 1] - off;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
        z64 *row = G + goff[c] + i * N;
        for (int64_t j = 0; j < N; ++j) row[j] = z64(0, 0);
        for (int sl = 0; sl < 6; ++sl) {
            int64_t cc = col[6 * (off + i) + sl];
            if (cc >= off && cc < off + N) row[cc - off].re += val[6 * (off + i) + sl];
        }
    }
}

// dst (column-major s x s) = src (row-major s x s), per cell
__global__ void k_to_colmajor(int s, const z64 *__restrict__ src, z64 *__restrict__ dst) {
    const int c = blockIdx.y;
    for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < (int64_t)s * s;
         idx += (int64_t)gridDim.x * blockDim.x) {
        int64_t i = idx / s, j = idx % s;
        dst[(int64_t)c * s * s + j * s + i] = src[(int64_t)c * s * s + idx];
    }
}

// U_L = X(:, perm(0:L)) / sigma, V_L = V(:, perm(0:L)), row-major s x L_m at loff[c]
__global__ void k_select(int s, const int32_t *__restrict__ perm, const int32_t *__restrict__ L,
                         const int64_t *__restrict__ loff, const z64 *__restrict__ X, const z64 *__restrict__ V,
                         const double *__restrict__ sig, z64 *__restrict__ UL, z64 *__restrict__ VL) {
    const int c = blockIdx.y;
    const int Lc = L[c];
    for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < (int64_t)s * Lc;
         idx += (int64_t)gridDim.x * blockDim.x) {
        int64_t r = idx / Lc, l = idx % Lc;
        int pc = perm[(int64_t)c * s + l];
        double sg = sig[(int64_t)c * s + pc];
        z64 x = X[(int64_t)c * s * s + (int64_t)pc * s + r];
        UL[loff[c] + idx] = (sg > 0.0) ? x * (1.0 / sg) : z64(0, 0);
        VL[loff[c] + idx] = V[(int64_t)c * s * s + (int64_t)pc * s + r];
    }
}

// X = Gf * C_all (ne x nh), C_all block diagonal: X[i][coff_c + l] = sum_slots val * C_c[col - off_c][l]
__global__ void k_gram_times_c(int64_t ne, int64_t nh, const int32_t *__restrict__ edge_cell,
                               const int32_t *__restrict__ cell_off, const int64_t *__restrict__ coff,
                               const int64_t *__restrict__ boff, const int32_t *__restrict__ Lc,
                               const double *__restrict__ val, const int32_t *__restrict__ col,
                               const z64 *__restrict__ C, z64 *__restrict__ X) {
    const int64_t i = blockIdx.y;
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < nh; k += (int64_t)gridDim.x * blockDim.x) {
        z64 acc(0, 0);
        for (int sl = 0; sl < 6; ++sl) {
            int cc = col[6 * i + sl];
            int c = edge_cell[cc];
            int64_t l = k - coff[c];
            if (l < 0 || l >= Lc[c]) continue;
            acc += val[6 * i + sl] * C[boff[c] + (int64_t)(cc - cell_off[c]) * Lc[c] + l];
        }
        X[i * nh + k] = acc;
    }
}

// complex transpose: dst (cols x rows) = src (rows x cols)^T
__global__ void k_transpose(int64_t rows, int64_t cols, const z64 *__restrict__ src, z64 *__restrict__ dst) {
    for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < rows * cols;
         idx += (int64_t)gridDim.x * blockDim.x) {
        int64_t i = idx / cols, j = idx % cols;
        dst[j * rows + i] = src[idx];
    }
}

// j in canonical edge order: out[ce][w] = in[int(ce)][w] (M part), out[ne+ce][w] = in[ne+int(ce)][w]
__global__ void k_to_canonical(int64_t ne, int nrhs, const int32_t *__restrict__ int_of_canon,
                               const z64 *__restrict__ in, z64 *__restrict__ out) {
    for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < 2 * ne * nrhs;
         idx += (int64_t)gridDim.x * blockDim.x) {
        int64_t row = idx / nrhs, w = idx % nrhs;
        int64_t half = row >= ne, ce = row - half * ne;
        out[idx] = in[(half * ne + int_of_canon[ce]) * nrhs + w];
    }
}

// block-diagonal assembly of two half inverses into the n x n matrix
__global__ void k_place_block(int64_t n, int64_t nh, int64_t r0, const z64 *__restrict__ blk, z64 *__restrict__ out) {
    for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < nh * nh;
         idx += (int64_t)gridDim.x * blockDim.x) {
        int64_t i = idx / nh, j = idx % nh;
        out[(r0 + i) * n + r0 + j] = blk[idx];
    }
}

// out[(r0 + i) * n + r0 + j] = -conj(blk[j * nh + i]): minus the adjoint of an nh x nh block
__global__ void k_place_neg_adjoint(int64_t n, int64_t nh, int64_t r0, const z64 *__restrict__ blk, int64_t ldb,
                                    z64 *__restrict__ out) {
    for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < nh * nh;
         idx += (int64_t)gridDim.x * blockDim.x) {
        int64_t i = idx / nh, j = idx % nh;
        const z64 v = blk[j * ldb + i];
        out[(r0 + i) * n + r0 + j] = z64(-v.re, v.im);
    }
}

__global__ void k_copy_block(int64_t n, int64_t nh, int64_t r0, const z64 *__restrict__ full, z64 *__restrict__ blk) {
    for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < nh * nh;
         idx += (int64_t)gridDim.x * blockDim.x) {
        int64_t i = idx / nh, j = idx % nh;
        blk[idx] = full[(r0 + i) * n + r0 + j];
    }
}

inline unsigned nblk(int64_t work, int64_t per = 256, int64_t cap = 65535) {
    return (unsigned)std::max<int64_t>(1, std::min<int64_t>((work + per - 1) / per, cap));
}

template <typename F>
cbfm_status guarded(F &&f) {
    struct Flush {
        ~Flush() {
            if (g_prof.load()) prof_flush();
        }
    } flush_on_exit;
    try {
        f();
        t_err.clear();
        return CBFM_OK;
    } catch (const Fail &e) {
        t_err = e.msg;
        return e.st;
    } catch (const std::bad_alloc &) {
        t_err = "host allocation failed";
        return CBFM_ENOMEM;
    } catch (const std::exception &e) {
        t_err = e.what();
        return CBFM_EINVAL;
    }
}

void check_device(const HandleBase *h, uint32_t kind, const char *what) {
    CBFM_REQUIRE(h != nullptr, std::string(what) + " handle is NULL");
    CBFM_REQUIRE(h->kind == kind, std::string(what) + " handle has the wrong type");
    int dev = -1;
    CBFM_CUDA(cudaGetDevice(&dev));
    CBFM_REQUIRE(dev == h->device, std::string(what) + " handle belongs to another device");
}

template <typename T>
void upload(DevBuf<T> &b, const std::vector<T> &v, cudaStream_t st) {
    b.alloc(v.size());
    if (!v.empty()) CBFM_CUDA(cudaMemcpyAsync(b.p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice, st));
}

void cbf_finish(Cbf &c) {
    const HostMesh &h = c.mesh->h;
    c.coff.assign(h.ncell + 1, 0);
    c.boff.assign(h.ncell + 1, 0);
    for (int m = 0; m < h.ncell; ++m) {
        c.coff[m + 1] = c.coff[m] + c.L[m];
        c.boff[m + 1] = c.boff[m] + (int64_t)(h.cell_off[m + 1] - h.cell_off[m]) * c.L[m];
    }
    c.nhalf = c.coff[h.ncell];
}

void cbf_make32(Cbf &c, cudaStream_t st) {
    int64_t tot = c.boff.back();
    c.CM32.alloc(tot);
    c.CJ32.alloc(tot);
    launch_z64_to_c32(c.CM.p, c.CM32.p, tot, st);
    launch_z64_to_c32(c.CJ.p, c.CJ32.p, tot, st);
}

// Steps after the coefficient sets (paper Eqs. (gram_CBF), (gram_CBF_SVD), (CBF)): G'_m = (J^M)^H G_m J^J,
// SVD, truncation sigma_i / sigma_1 >= delta_svd (at most lmax when > 0), C^M = J^M U_L, C^J = J^J V_L.
// Vm holds, per cell, [J^M; J^J] (2 N_m x s, row-major) at voff[c].
std::unique_ptr<Cbf> dual_cbfs(Mesh *m, int s, const z64 *Vm, const std::vector<int64_t> &voff, double delta_svd,
                               int lmax, int32_t *L_per_cell, double *sigma_out, cudaStream_t st) {
    const HostMesh &h = m->h;
    const int nc = h.ncell;
    std::vector<int64_t> goff(nc + 1, 0), soff(nc);
    std::vector<int> nn(nc);
    for (int c = 0; c < nc; ++c) {
        int64_t N = h.cell_off[c + 1] - h.cell_off[c];
        nn[c] = (int)(2 * N);
        goff[c + 1] = goff[c] + N * N;
        soff[c] = (int64_t)c * s * s;
    }
    DevBuf<int32_t> dcoff;
    upload(dcoff, h.cell_off, st);
    DevBuf<int64_t> dgoff;
    upload(dgoff, goff, st);
    DevBuf<int> info;
    info.alloc(nc);
    std::vector<int> hinfo(nc);
    // Gram of every cell, G'_m = (J^M)^H G_m J^J
    DevBuf<z64> Gm, T1, Gp, X, Vs;
    Gm.alloc(goff[nc]);
    {
        ProfScope ps_("k_cell_gram", st);
        k_cell_gram<<<dim3(nblk(4096), nc), 256, 0, st>>>(nc, dcoff.p, dgoff.p, m->gram_val.p, m->gram_col.p, Gm.p);
        launched("k_cell_gram");
    }
    std::vector<int64_t> t1off(nc);
    int64_t t1t = 0;
    for (int c = 0; c < nc; ++c) {
        t1off[c] = t1t;
        t1t += (int64_t)(nn[c] / 2) * s;
    }
    T1.alloc(t1t);
    Gp.alloc((size_t)nc * s * s);
    std::vector<GemmDesc> g1, g2;
    for (int c = 0; c < nc; ++c) {
        int64_t N = nn[c] / 2;
        // T1 = G_m J^J  (J^J = rows N..2N-1 of V_m)
        g1.push_back(GemmDesc{N, s, N, goff[c], N, voff[c] + N * s, s, t1off[c], s});
        // G' = (J^M)^H T1
        g2.push_back(GemmDesc{s, s, N, voff[c], s, t1off[c], s, soff[c], s});
    }
    gemm_grouped<double>(g1, 0, 0, Gm.p, Vm, T1.p, false, st);
    gemm_grouped<double>(g2, 2, 0, Vm, T1.p, Gp.p, false, st);
    X.alloc((size_t)nc * s * s);
    Vs.alloc((size_t)nc * s * s);
    {
        ProfScope ps_("k_to_colmajor", st);
        k_to_colmajor<<<dim3(nblk((int64_t)s * s), nc), 256, 0, st>>>(s, Gp.p, X.p);
        launched("k_to_colmajor");
    }
    DevBuf<double> sig;
    sig.alloc((size_t)nc * s);
    CBFM_CUDA(cudaMemsetAsync(info.p, 0, sizeof(int) * nc, st));
    jacobi_svd_batched(nc, s, X.p, Vs.p, sig.p, info.p, st, delta_svd);
    std::vector<double> hs((size_t)nc * s);
    CBFM_CUDA(cudaMemcpyAsync(hs.data(), sig.p, sizeof(double) * nc * s, cudaMemcpyDeviceToHost, st));
    CBFM_CUDA(cudaMemcpyAsync(hinfo.data(), info.p, sizeof(int) * nc, cudaMemcpyDeviceToHost, st));
    CBFM_CUDA(cudaStreamSynchronize(st));
    for (int c = 0; c < nc; ++c)
        if (hinfo[c]) throw Fail{hinfo[c] == 1 ? CBFM_ETIMEOUT : CBFM_ECUDA,
                                 (hinfo[c] == 1 ? "Jacobi SVD: a cluster synchronisation expired in cell "
                                                : "Jacobi SVD did not converge in cell ") + std::to_string(c)};
    // truncation: keep sigma_i / sigma_1 >= delta_svd (paper Eq. (gram_CBF_SVD))
    std::unique_ptr<Cbf> cb(new Cbf());
    cb->kind = H_CBF;
    cb->device = m->device;
    cb->mesh = m;
    cb->L.assign(nc, 0);
    std::vector<int32_t> perm((size_t)nc * s);
    std::vector<int64_t> loff(nc + 1, 0);
    for (int c = 0; c < nc; ++c) {
        int32_t *pc = perm.data() + (size_t)c * s;
        std::iota(pc, pc + s, 0);
        const double *sc = hs.data() + (size_t)c * s;
        std::stable_sort(pc, pc + s, [&](int a, int b) { return sc[a] > sc[b]; });
        double s1 = sc[pc[0]];
        CBFM_REQUIRE(s1 > 0.0, "zero CBF Gram matrix in cell " + std::to_string(c));
        int L = 0;
        for (int i = 0; i < s; ++i)
            if (sc[pc[i]] / s1 >= delta_svd) ++L;
        if (lmax > 0) L = std::min(L, (int)lmax);
        L = std::min<int>(L, nn[c] / 2);
        L = std::max(L, 1);
        cb->L[c] = L;
        L_per_cell[c] = L;
        if (sigma_out)
            for (int i = 0; i < s; ++i) sigma_out[(size_t)c * s + i] = sc[pc[i]] / s1;
        loff[c + 1] = loff[c] + (int64_t)s * L;
    }
    cbf_finish(*cb);
    DevBuf<int32_t> dperm, dL;
    DevBuf<int64_t> dloff;
    upload(dperm, perm, st);
    upload(dL, cb->L, st);
    upload(dloff, loff, st);
    DevBuf<z64> UL, VL;
    UL.alloc(loff[nc]);
    VL.alloc(loff[nc]);
    {
        ProfScope ps_("k_select", st);
        k_select<<<dim3(nblk((int64_t)s * 64), nc), 256, 0, st>>>(s, dperm.p, dL.p, dloff.p, X.p, Vs.p, sig.p, UL.p,
                                                                  VL.p);
        launched("k_select");
    }
    // C^M = J^M U_L, C^J = J^J V_L (paper Eq. (CBF))
    cb->CM.alloc(cb->boff[nc]);
    cb->CJ.alloc(cb->boff[nc]);
    std::vector<GemmDesc> gm, gj;
    for (int c = 0; c < nc; ++c) {
        int64_t N = nn[c] / 2, L = cb->L[c];
        gm.push_back(GemmDesc{N, L, s, voff[c], s, loff[c], L, cb->boff[c], L});
        gj.push_back(GemmDesc{N, L, s, voff[c] + N * s, s, loff[c], L, cb->boff[c], L});
    }
    gemm_grouped<double>(gm, 0, 0, Vm, UL.p, cb->CM.p, false, st);
    gemm_grouped<double>(gj, 0, 0, Vm, VL.p, cb->CJ.p, false, st);
    cbf_make32(*cb, st);
    return cb;
}

}  // namespace
}  // namespace cbfm

using namespace cbfm;

extern "C" {

const char *cbfm_last_error(void) { return t_err.c_str(); }

int64_t cbfm_launch_count(void) { return g_launches.load(); }

int64_t cbfm_tuning(char *buf, int64_t cap) {
    std::string j = "{";
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        bool first = true;
        for (auto &kv : g_tune) {
            j += (first ? "\"" : ", \"") + kv.first + "\": " + std::to_string(kv.second);
            first = false;
        }
    }
    j += "}";
    if (buf && cap > 0) {
        const size_t n = std::min<size_t>((size_t)cap - 1, j.size());
        std::memcpy(buf, j.data(), n);
        buf[n] = 0;
    }
    return (int64_t)j.size();
}

void cbfm_profile(int32_t enable) {
    prof_flush();
    g_prof.store(enable != 0);
}

int64_t cbfm_profile_read(char *buf, int64_t cap, int32_t reset) {
    prof_flush();
    std::lock_guard<std::mutex> lk(g_prof_mu);
    std::string js = "{";
    bool first = true;
    for (auto &kv : g_acc) {
        char tmp[320];
        snprintf(tmp, sizeof(tmp), "%s\"%s\": {\"launches\": %lld, \"ms\": %.6f, \"flop\": %.6e, \"bytes\": %.6e}",
                 first ? "" : ", ", kv.first.c_str(), (long long)kv.second.launches, kv.second.ms, kv.second.flop,
                 kv.second.bytes);
        js += tmp;
        first = false;
    }
    js += "}";
    if (reset) g_acc.clear();
    if (buf && cap > 0) {
        int64_t n = std::min<int64_t>(cap - 1, (int64_t)js.size());
        memcpy(buf, js.data(), n);
        buf[n] = 0;
    }
    return (int64_t)js.size() + 1;
}

cbfm_status cbfm_mesh(const double *verts, int64_t nv, const int32_t *tris, int64_t nt, const int32_t *edge_cell,
                      int32_t ncell, int32_t partition, double eps_re, double eps_im, double mu_r, double alpha,
                      void *stream, cbfm_mesh_t *out) {
    return guarded([&] {
        StreamScope ss_((cudaStream_t)stream);   // scratch is stream-ordered on the caller's stream
        CBFM_REQUIRE(out != nullptr && verts != nullptr && tris != nullptr, "NULL argument");
        *out = nullptr;
        CBFM_REQUIRE(eps_im <= 0.0, "eps_im must be <= 0 (passive medium, exp(+j w t))");
        CBFM_REQUIRE(mu_r > 0.0 && alpha > 0.0, "mu_r and alpha must be positive");
        CBFM_REQUIRE(!(eps_re == 0.0 && eps_im == 0.0), "eps_r must be nonzero");
        cudaStream_t st = (cudaStream_t)stream;
        std::vector<double> hv(3 * nv);
        std::vector<int32_t> ht(3 * nt);
        CBFM_REQUIRE(nv > 0 && nt > 0, "empty mesh");
        copy_out(hv.data(), verts, hv.size() * sizeof(double), st);
        copy_out(ht.data(), tris, ht.size() * sizeof(int32_t), st);
        std::vector<int32_t> hc;
        if (edge_cell) {
            hc.resize((size_t)(3 * nt / 2));
            copy_out(hc.data(), edge_cell, hc.size() * sizeof(int32_t), st);
        }
        CBFM_CUDA(cudaStreamSynchronize(st));
        Mesh *m = new Mesh();
        std::unique_ptr<Mesh> guard(m);
        m->kind = H_MESH;
        CBFM_CUDA(cudaGetDevice(&m->device));
        build_host_mesh(hv.data(), nv, ht.data(), nt, edge_cell ? hc.data() : nullptr, ncell, partition, m->h);
        m->eps_re = eps_re;
        m->eps_im = eps_im;
        m->mu_r = mu_r;
        m->alpha = alpha;
        std::complex<double> eps(eps_re, eps_im);
        std::complex<double> n2 = std::sqrt(eps * mu_r);
        if (n2.real() < 0) n2 = -n2;
        std::complex<double> k2 = K0 * n2;
        std::complex<double> eta2 = ETA0 * std::sqrt(std::complex<double>(mu_r, 0) / eps);
        m->k1 = z64(K0, 0);
        m->eta1 = z64(ETA0, 0);
        m->k2 = z64(k2.real(), k2.imag());
        m->eta2 = z64(eta2.real(), eta2.imag());
        for (int d = 0; d < 3; ++d) {
            double lo = INFINITY, hi = -INFINITY;
            for (int64_t i = 0; i < nv; ++i) {
                lo = std::min(lo, hv[3 * i + d]);
                hi = std::max(hi, hv[3 * i + d]);
            }
            m->centre[d] = 0.5 * (lo + hi);
        }
        const HostMesh &h = m->h;
        DevBuf<double> dv;
        DevBuf<int32_t> dt;
        upload(dv, h.verts, st);
        upload(dt, h.tris, st);
        upload(m->tri_vid, h.tris, st);
        upload(m->tri_edge, h.tri_edge, st);
        {
            // cell of each RWG of each triangle (edges are sorted by cell)
            std::vector<int32_t> tc((size_t)3 * h.nt);
            for (size_t k = 0; k < tc.size(); ++k) {
                const int32_t e = h.tri_edge[k];
                tc[k] = (int32_t)(std::upper_bound(h.cell_off.begin(), h.cell_off.end(), e) - h.cell_off.begin()) - 1;
            }
            upload(m->tri_cell, tc, st);
        }
        upload(m->edge_tri, h.edge_tri, st);
        upload(m->edge_loc, h.edge_loc, st);
        std::vector<int32_t> ecell(h.ne);
        for (int c = 0; c < h.ncell; ++c)
            for (int32_t e = h.cell_off[c]; e < h.cell_off[c + 1]; ++e) ecell[e] = c;
        upload(m->edge_cell, ecell, st);
        m->tri64.alloc((size_t)h.nt * TRI_REC);
        m->tri32.alloc((size_t)h.nt * TRI_REC);
        launch_tri_records(*m, dv.p, dt.p, st);
        launch_near_pairs(*m, st);
        launch_gram_rows(*m, st);
        CBFM_CUDA(cudaStreamSynchronize(st));
        *out = (cbfm_mesh_t)guard.release();
    });
}

cbfm_status cbfm_mesh_edges(const double *verts, int64_t nv, const int32_t *tris, int64_t nt, int32_t ncell,
                            int32_t partition, int64_t *n_edges, int32_t *edges, int32_t *cells) {
    return guarded([&] {
        CBFM_REQUIRE(verts && tris && n_edges, "NULL argument");
        HostMesh hm;
        build_host_mesh(verts, nv, tris, nt, nullptr, ncell, partition, hm);
        *n_edges = hm.ne;
        for (int64_t e = 0; e < hm.ne; ++e) {
            if (edges) {
                edges[2 * e] = hm.canon_u[e];
                edges[2 * e + 1] = hm.canon_v[e];
            }
            if (cells) cells[e] = hm.cell_of_canon[e];
        }
    });
}

cbfm_status cbfm_mesh_info(cbfm_mesh_t mesh, int64_t *n_edges, int32_t *n_cells, int64_t *n_near) {
    return guarded([&] {
        Mesh *m = (Mesh *)mesh;
        CBFM_REQUIRE(m && m->kind == H_MESH, "bad mesh handle");
        if (n_edges) *n_edges = m->h.ne;
        if (n_cells) *n_cells = m->h.ncell;
        if (n_near) *n_near = m->n_near;
    });
}

cbfm_status cbfm_mesh_cells(cbfm_mesh_t mesh, int32_t *edge_cell, void *stream) {
    return guarded([&] {
        StreamScope ss_((cudaStream_t)stream);   // scratch is stream-ordered on the caller's stream
        Mesh *m = (Mesh *)mesh;
        check_device(m, H_MESH, "mesh");
        CBFM_REQUIRE(edge_cell, "NULL edge_cell");
        copy_out(edge_cell, m->h.cell_of_canon.data(), m->h.ne * sizeof(int32_t), (cudaStream_t)stream);
        CBFM_CUDA(cudaStreamSynchronize((cudaStream_t)stream));
    });
}

cbfm_status cbfm_build_cbfs(cbfm_mesh_t mesh, const double *waves, int32_t s, double delta_svd, int32_t lmax,
                            void *stream, cbfm_cbf_t *out, int32_t *L_per_cell, double *sigma_out) {
    return guarded([&] {
        StreamScope ss_((cudaStream_t)stream);   // scratch is stream-ordered on the caller's stream
        Mesh *m = (Mesh *)mesh;
        check_device(m, H_MESH, "mesh");
        CBFM_REQUIRE(out && waves && L_per_cell, "NULL argument");
        *out = nullptr;
        CBFM_REQUIRE(s >= 1 && s <= 1024, "s must be in [1, 1024]");
        CBFM_REQUIRE(delta_svd >= 0.0 && delta_svd <= 1.0, "delta_svd must be in [0, 1]");
        cudaStream_t st = (cudaStream_t)stream;
        const HostMesh &h = m->h;
        const int nc = h.ncell;
        const int64_t ne = h.ne;
        for (int c = 0; c < nc; ++c) CBFM_REQUIRE(2 * (h.cell_off[c + 1] - h.cell_off[c]) <= 4096, "cell too large");
        DevBuf<double> dw;
        dw.alloc(3 * (size_t)s);
        copy_in(dw.p, waves, 3 * sizeof(double) * s, st);
        // plane-wave RHS
        DevBuf<z64> vE, vH;
        vE.alloc((size_t)ne * s);
        vH.alloc((size_t)ne * s);
        launch_rhs(*m, dw.p, s, vE.p, vH.p, st);
        // per-cell systems
        std::vector<int64_t> zoff(nc), voff(nc);
        std::vector<int> nn(nc);
        int64_t zt = 0, vt = 0;
        for (int c = 0; c < nc; ++c) {
            int64_t N = h.cell_off[c + 1] - h.cell_off[c];
            zoff[c] = zt;
            voff[c] = vt;
            nn[c] = (int)(2 * N);
            zt += 4 * N * N;
            vt += 2 * N * s;
        }
        DevBuf<z64> Zmm, Vm;
        Zmm.alloc(zt);
        Vm.alloc(vt);
        DevBuf<int32_t> dcoff;
        upload(dcoff, h.cell_off, st);
        DevBuf<int64_t> dvoff;
        upload(dvoff, voff, st);
        assemble_cell_diag(*m, Zmm.p, zoff, st);   // the cells' diagonal blocks Z_mm (FP64)
        {
            ProfScope ps_("k_extract_v", st);
            k_extract_v<<<dim3(nblk(4096 * 4), nc), 256, 0, st>>>(nc, dcoff.p, dvoff.p, s, vE.p, vH.p, Vm.p);
            launched("k_extract_v");
        }
        DevBuf<int> info;
        info.alloc(nc);
        CBFM_CUDA(cudaMemsetAsync(info.p, 0, sizeof(int) * nc, st));
        lu_solve_batched(nc, zoff.data(), voff.data(), nn.data(), s, Zmm.p, Vm.p, info.p, st);
        std::vector<int> hinfo(nc);
        CBFM_CUDA(cudaMemcpyAsync(hinfo.data(), info.p, sizeof(int) * nc, cudaMemcpyDeviceToHost, st));
        CBFM_CUDA(cudaStreamSynchronize(st));
        for (int c = 0; c < nc; ++c)
            if (hinfo[c]) throw Fail{CBFM_ESINGULAR, "singular Z_mm in cell " + std::to_string(c)};
        Zmm.release();
        std::unique_ptr<Cbf> cb = dual_cbfs(m, s, Vm.p, voff, delta_svd, lmax, L_per_cell, sigma_out, st);
        CBFM_CUDA(cudaStreamSynchronize(st));
        *out = (cbfm_cbf_t)cb.release();
    });
}

cbfm_status cbfm_build_ipcbfs(cbfm_red_t mom, const double *waves, int32_t s, double delta_r, int32_t maxit,
                              int32_t restart, double delta_svd, int32_t lmax, void *stream, cbfm_cbf_t *out,
                              int32_t *L_per_cell, double *sigma_out, int32_t *iters_out) {
    return guarded([&] {
        StreamScope ss_((cudaStream_t)stream);   // scratch is stream-ordered on the caller's stream
        Red *r = (Red *)mom;
        check_device(r, H_RED, "MoM system");
        CBFM_REQUIRE(r->cbf == nullptr, "IPCBFs are generated from a cbfm_assemble_mom handle");
        CBFM_REQUIRE(out && waves && L_per_cell, "NULL argument");
        *out = nullptr;
        CBFM_REQUIRE(s >= 1 && s <= 1024, "s must be in [1, 1024]");
        CBFM_REQUIRE(delta_r > 0.0 && maxit >= 1 && restart >= 1, "delta_r, maxit and restart must be positive");
        CBFM_REQUIRE(delta_svd >= 0.0 && delta_svd <= 1.0, "delta_svd must be in [0, 1]");
        cudaStream_t st = (cudaStream_t)stream;
        Mesh *m = r->mesh;
        const HostMesh &h = m->h;
        const int nc = h.ncell;
        const int64_t ne = h.ne, n = r->n;
        // the MoM arrangement of Eq. (MoM_T): T-diagonal with the diagonal preconditioner
        if (!(r->tdiag_ready && r->tdiag_jacobi) && !tdiag_build(*r, true, st))
            throw Fail{CBFM_ESINGULAR, "a diagonal entry of the T-diagonal arrangement is zero"};
        DevBuf<double> dw;
        dw.alloc(3 * (size_t)s);
        copy_in(dw.p, waves, 3 * sizeof(double) * s, st);
        DevBuf<z64> vE, vH, bt, b, x;
        vE.alloc((size_t)ne * s);
        vH.alloc((size_t)ne * s);
        launch_rhs(*m, dw.p, s, vE.p, vH.p, st, r->prec != CBFM_FP64);
        bt.alloc((size_t)n * s);
        CBFM_CUDA(cudaMemcpyAsync(bt.p, vE.p, sizeof(z64) * ne * s, cudaMemcpyDeviceToDevice, st));
        CBFM_CUDA(cudaMemcpyAsync(bt.p + ne * s, vH.p, sizeof(z64) * ne * s, cudaMemcpyDeviceToDevice, st));
        vE.release();
        vH.release();
        b.alloc((size_t)n * s);
        {
            ProfScope ps_("k_transpose", st);
            k_transpose<<<nblk(n * s), 256, 0, st>>>(n, s, bt.p, b.p);
            launched("k_transpose");
        }
        bt.release();
        // each generating wave's whole-system GMRES solution, stopped at relative residual delta_r
        x.alloc((size_t)n * s);
        GmresOut go = gmres_solve(*r, b.p, s, delta_r, maxit, restart, CBFM_PC_TDIAG, x.p, st);
        for (int w = 0; w < s; ++w) {
            if (iters_out) iters_out[w] = go.iters[w] >= 0 ? go.iters[w] : -go.iters[w] - 1;
            if (go.iters[w] < 0)
                throw Fail{CBFM_ENOCONV, "IPCBF wave " + std::to_string(w) + " did not reach delta_r within maxit"};
        }
        b.release();
        // coefficient sets of every cell: the solutions restricted to the cell's RWG functions
        std::vector<int64_t> voff(nc);
        int64_t vt = 0;
        for (int c = 0; c < nc; ++c) {
            voff[c] = vt;
            vt += 2 * (int64_t)(h.cell_off[c + 1] - h.cell_off[c]) * s;
        }
        DevBuf<z64> Vm;
        Vm.alloc(vt);
        DevBuf<int32_t> dcoff;
        upload(dcoff, h.cell_off, st);
        DevBuf<int64_t> dvoff;
        upload(dvoff, voff, st);
        {
            ProfScope ps_("k_ipcbf_gather", st);
            k_ipcbf_gather<<<dim3(nblk(4096 * 4), nc), 256, 0, st>>>(nc, dcoff.p, dvoff.p, s, ne, x.p, Vm.p);
            launched("k_ipcbf_gather");
        }
        x.release();
        std::unique_ptr<Cbf> cb = dual_cbfs(m, s, Vm.p, voff, delta_svd, lmax, L_per_cell, sigma_out, st);
        CBFM_CUDA(cudaStreamSynchronize(st));
        *out = (cbfm_cbf_t)cb.release();
    });
}

cbfm_status cbfm_cbf_import(cbfm_mesh_t mesh, const int32_t *L_per_cell, const double *CM, const double *CJ,
                            void *stream, cbfm_cbf_t *out) {
    return guarded([&] {
        StreamScope ss_((cudaStream_t)stream);   // scratch is stream-ordered on the caller's stream
        Mesh *m = (Mesh *)mesh;
        check_device(m, H_MESH, "mesh");
        CBFM_REQUIRE(out && L_per_cell && CM && CJ, "NULL argument");
        *out = nullptr;
        cudaStream_t st = (cudaStream_t)stream;
        std::unique_ptr<Cbf> cb(new Cbf());
        cb->kind = H_CBF;
        cb->device = m->device;
        cb->mesh = m;
        cb->L.assign(L_per_cell, L_per_cell + m->h.ncell);
        for (int c = 0; c < m->h.ncell; ++c) {
            CBFM_REQUIRE(cb->L[c] >= 1, "L_per_cell must be >= 1");
            CBFM_REQUIRE(cb->L[c] <= m->h.cell_off[c + 1] - m->h.cell_off[c], "L_m larger than N_m");
        }
        cbf_finish(*cb);
        int64_t tot = cb->boff.back();
        cb->CM.alloc(tot);
        cb->CJ.alloc(tot);
        copy_in(cb->CM.p, CM, tot * sizeof(z64), st);
        copy_in(cb->CJ.p, CJ, tot * sizeof(z64), st);
        cbf_make32(*cb, st);
        CBFM_CUDA(cudaStreamSynchronize(st));
        *out = (cbfm_cbf_t)cb.release();
    });
}

cbfm_status cbfm_cbf_export(cbfm_cbf_t cbf, double *CM, double *CJ, void *stream) {
    return guarded([&] {
        StreamScope ss_((cudaStream_t)stream);   // scratch is stream-ordered on the caller's stream
        Cbf *c = (Cbf *)cbf;
        check_device(c, H_CBF, "cbf");
        int64_t tot = c->boff.back();
        if (CM) copy_out(CM, c->CM.p, tot * sizeof(z64), (cudaStream_t)stream);
        if (CJ) copy_out(CJ, c->CJ.p, tot * sizeof(z64), (cudaStream_t)stream);
        CBFM_CUDA(cudaStreamSynchronize((cudaStream_t)stream));
    });
}

}  // extern "C"

namespace {

// A = (C^JM)^H Z C^MJ from the RWG blocks (T = double or float)
template <typename T>
void project(Red &r, cudaStream_t st) {
    Mesh &m = *r.mesh;
    Cbf &c = *r.cbf;
    const int64_t ne = m.h.ne, nh = c.nhalf, n = 2 * nh;
    const int nc = m.h.ncell;
    DevBuf<cx<T>> A;
    A.alloc((size_t)n * n);
    if constexpr (sizeof(T) == 4) {
        // mixed precision: assembly fused with the tensor-core projection (no RWG
        // matrix in memory) when the cells fit the fused kernel's tiles
        if ((r.prec == CBFM_MIXED_FUSED && fused_fits(m, c)) || (r.prec == CBFM_MIXED && mixed_takes_fused(m, c))) {
            assemble_project_fused({&m}, {&c}, {A.p}, st);
            A.give(r.A32);
            return;
        }
    }
    DevBuf<cx<T>> Z;
    Z.alloc(3 * (size_t)ne * ne);
    assemble_rwg<T>(m, Z.p, st);
    if constexpr (sizeof(T) == 4) {
        if (r.prec == CBFM_MIXED || r.prec == CBFM_MIXED_UNFUSED || r.prec == CBFM_MIXED_FUSED) {
            project_tc(m, c, Z.p, A.p, st);
            A.give(r.A32);
            return;
        }
    }
    const cx<T> *CM, *CJ;
    if constexpr (sizeof(T) == 8) { CM = c.CM.p; CJ = c.CJ.p; }
    else { CM = c.CM32.p; CJ = c.CJ32.p; }
    // chains: (operator, coefficient side of the columns, row test side, A row block, A column block)
    struct Chain { int op; bool colM; bool rowJ; int64_t r0, c0; };
    const Chain ch[4] = {{0, true, true, 0, 0}, {1, false, true, 0, nh}, {2, true, false, nh, 0}, {0, false, false, nh, nh}};
    DevBuf<cx<T>> Y;
    Y.alloc((size_t)ne * nh);
    for (int q = 0; q < 4; ++q) {
        std::vector<GemmDesc> g1, g2;
        for (int k = 0; k < nc; ++k) {
            int64_t off = m.h.cell_off[k], N = m.h.cell_off[k + 1] - off, L = c.L[k];
            // Y[:, coff_k + l] = Z_op[:, Lambda_k] C_k
            g1.push_back(GemmDesc{ne, L, N, (int64_t)ch[q].op * ne * ne + off, ne, c.boff[k], L, c.coff[k], nh});
            // A[r0 + coff_k + l, c0 + :] = C_k^H Y[Lambda_k, :]
            g2.push_back(GemmDesc{L, nh, N, c.boff[k], L, off * nh, nh, (ch[q].r0 + c.coff[k]) * n + ch[q].c0, n});
        }
        gemm_grouped<T>(g1, 0, 0, Z.p, ch[q].colM ? CM : CJ, Y.p, false, st);
        gemm_grouped<T>(g2, 2, 0, ch[q].rowJ ? CJ : CM, Y.p, A.p, false, st);
    }
    if constexpr (sizeof(T) == 8) {
        A.give(r.A64);
    } else {
        A.give(r.A32);
    }
}


// G^CBF = (C^JM)^H G_ffff C^MJ (paper Eq. (CBF_Gram_matrix)) into r.G: the sparse RWG Gram rows
// times the CBF blocks, then the two halves' cell-block products
void gram_cbf(Red &r, cudaStream_t st) {
    Mesh &m = *r.mesh;
    Cbf &c = *r.cbf;
    const int64_t ne = m.h.ne, nh = c.nhalf, n = r.n;
    const int nc = m.h.ncell;
    DevBuf<int32_t> dcoff, dL;
    DevBuf<int64_t> dcoff64, dboff;
    upload(dcoff, m.h.cell_off, st);
    upload(dL, c.L, st);
    upload(dcoff64, c.coff, st);
    upload(dboff, c.boff, st);
    DevBuf<z64> XM;
    XM.alloc((size_t)ne * nh);
    dim3 gx(nblk(nh), (unsigned)ne);
    CBFM_REQUIRE(ne <= 65535, "too many edges for the Gram product grid");
    {
        ProfScope ps_("k_gram_times_c", st);
        k_gram_times_c<<<gx, 256, 0, st>>>(ne, nh, m.edge_cell.p, dcoff.p, dcoff64.p, dboff.p, dL.p, m.gram_val.p,
                                           m.gram_col.p, c.CM.p, XM.p);
        launched("k_gram_times_c");
    }
    r.G.alloc((size_t)n * n);
    CBFM_CUDA(cudaMemsetAsync(r.G.p, 0, sizeof(z64) * n * n, st));
    std::vector<GemmDesc> gJ;
    for (int k = 0; k < nc; ++k) {
        int64_t off = m.h.cell_off[k], N = m.h.cell_off[k + 1] - off, L = c.L[k];
        // first half: (C^J)^H Gf C^M
        gJ.push_back(GemmDesc{L, nh, N, c.boff[k], L, off * nh, nh, c.coff[k] * n, n});
    }
    gemm_grouped<double>(gJ, 2, 0, c.CJ.p, XM.p, r.G.p, false, st);
    // second half (C^M)^H Gf C^J = -((C^J)^H Gf C^M)^H: the RWG Gram Gf = <f_a, n x f_b> is
    // real and antisymmetric (a . (n x b) = -b . (n x a), entry by entry in k_gram_rows)
    {
        ProfScope ps_("k_place_neg_adjoint", st);
        k_place_neg_adjoint<<<nblk(nh * nh), 256, 0, st>>>(n, nh, nh, r.G.p, n, r.G.p);
        launched("k_place_neg_adjoint");
    }
    XM.release();
}

// Rows b (nrhs x n) of the reduced right-hand sides for plane-wave excitations
// d_exc (device, nrhs x (theta, phi, pol)): v = the tested incident fields
// (paper Eq. (V)), b = (C^JM)^H v (b = v for the RWG system).  FP32 products
// for the mixed-precision systems.
void reduced_rhs_rows(Red &r, const double *d_exc, int nrhs, z64 *b, cudaStream_t st) {
    Mesh &m = *r.mesh;
    Cbf *cp = r.cbf;
    const int64_t ne = m.h.ne, nh = cp ? cp->nhalf : ne, n = r.n;
    const int nc = m.h.ncell;
    DevBuf<z64> vE, vH, bt;
    vE.alloc((size_t)ne * nrhs);
    vH.alloc((size_t)ne * nrhs);
    launch_rhs(m, d_exc, nrhs, vE.p, vH.p, st, r.prec != CBFM_FP64);
    // b = (C^JM)^H v  -> (n x nrhs), then rows per rhs
    bt.alloc((size_t)n * nrhs);
    const bool f32 = r.prec != CBFM_FP64;   // mixed precision: right-hand side and recovery in FP32
    if (!cp) {   // b = v = [v^E; v^H]
        CBFM_CUDA(cudaMemcpyAsync(bt.p, vE.p, sizeof(z64) * ne * nrhs, cudaMemcpyDeviceToDevice, st));
        CBFM_CUDA(cudaMemcpyAsync(bt.p + ne * nrhs, vH.p, sizeof(z64) * ne * nrhs, cudaMemcpyDeviceToDevice, st));
    } else {
        const Cbf &c = *cp;
        std::vector<GemmDesc> gE, gH;
        for (int k = 0; k < nc; ++k) {
            int64_t off = m.h.cell_off[k], N = m.h.cell_off[k + 1] - off, L = c.L[k];
            gE.push_back(GemmDesc{L, nrhs, N, c.boff[k], L, off * nrhs, nrhs, c.coff[k] * nrhs, nrhs});
            gH.push_back(GemmDesc{L, nrhs, N, c.boff[k], L, off * nrhs, nrhs, (nh + c.coff[k]) * nrhs, nrhs});
        }
        if (f32) {
            DevBuf<c32> e32, h32, b32;
            e32.alloc((size_t)ne * nrhs);
            h32.alloc((size_t)ne * nrhs);
            b32.alloc((size_t)n * nrhs);
            launch_z64_to_c32(vE.p, e32.p, ne * nrhs, st);
            launch_z64_to_c32(vH.p, h32.p, ne * nrhs, st);
            gemm_grouped<float>(gE, 2, 0, c.CJ32.p, e32.p, b32.p, false, st);
            gemm_grouped<float>(gH, 2, 0, c.CM32.p, h32.p, b32.p, false, st);
            launch_c32_to_z64(b32.p, bt.p, n * nrhs, st);
        } else {
            gemm_grouped<double>(gE, 2, 0, c.CJ.p, vE.p, bt.p, false, st);
            gemm_grouped<double>(gH, 2, 0, c.CM.p, vH.p, bt.p, false, st);
        }
    }
    {
        ProfScope ps_("k_transpose", st);
        k_transpose<<<nblk(n * nrhs), 256, 0, st>>>(n, nrhs, bt.p, b);
        launched("k_transpose");
    }
}

// Currents (internal edge order, (2 ne) x nrhs) j = C^MJ x from the reduced
// solutions x (nrhs x n rows), paper Eq. (trans_current); j = x for the RWG system.
void recover_currents(Red &r, const z64 *x, int nrhs, z64 *jint, cudaStream_t st) {
    Mesh &m = *r.mesh;
    Cbf *cp = r.cbf;
    const int64_t ne = m.h.ne, nh = cp ? cp->nhalf : ne, n = r.n;
    const int nc = m.h.ncell;
    const bool f32 = r.prec != CBFM_FP64;
    if (!cp) {   // j = x
        ProfScope ps_("k_transpose", st);
        k_transpose<<<nblk(n * nrhs), 256, 0, st>>>(nrhs, n, x, jint);
        launched("k_transpose");
        return;
    }
    const Cbf &c = *cp;
    std::vector<GemmDesc> jM, jJ;
    for (int k = 0; k < nc; ++k) {
        int64_t off = m.h.cell_off[k], N = m.h.cell_off[k + 1] - off, L = c.L[k];
        jM.push_back(GemmDesc{N, nrhs, L, c.boff[k], L, c.coff[k], n, off * nrhs, nrhs});
        jJ.push_back(GemmDesc{N, nrhs, L, c.boff[k], L, nh + c.coff[k], n, (ne + off) * nrhs, nrhs});
    }
    if (f32) {
        DevBuf<c32> x32, j32;
        x32.alloc((size_t)nrhs * n);
        j32.alloc((size_t)2 * ne * nrhs);
        launch_z64_to_c32(x, x32.p, nrhs * n, st);
        gemm_grouped<float>(jM, 0, 1, c.CM32.p, x32.p, j32.p, false, st);
        gemm_grouped<float>(jJ, 0, 1, c.CJ32.p, x32.p, j32.p, false, st);
        launch_c32_to_z64(j32.p, jint, 2 * ne * nrhs, st);
    } else {
        gemm_grouped<double>(jM, 0, 1, c.CM.p, x, jint, false, st);
        gemm_grouped<double>(jJ, 0, 1, c.CJ.p, x, jint, false, st);
    }
}

constexpr uint32_t H_SESSION = 0x53455353u;

// A block solve that right-hand sides may join while it runs (the serving
// loop's continuous batching).  Joins are queued under the mutex by any
// thread and taken by the solver at block-iteration boundaries.
struct Session : HandleBase, BgmresJoin {
    Red *r = nullptr;
    double tol = 1e-6;
    int maxit = 0, restart = 0, precond = CBFM_PC_CMP;
    std::mutex mu;
    std::vector<double> queued;        // excitations waiting to join, 3 per right-hand side
    std::atomic<int> nqueued{0};
    int accepted = 0;                  // right-hand sides accepted so far (slots)
    bool closed = false, ran = false;
    std::vector<double> exc_all;       // excitations in slot order (taken by the solver)
    std::vector<double> rcs;           // monostatic RCS parts, 2 per slot
    std::vector<int> iters;
    std::vector<double> resid;
    bool pending() override { return nqueued.load(std::memory_order_acquire) > 0; }
    int take(cudaStream_t st, DevBuf<z64> &rows) override {
        std::vector<double> exc;
        {
            std::lock_guard<std::mutex> lk(mu);
            exc.swap(queued);
            nqueued.store(0, std::memory_order_release);
        }
        const int k = (int)(exc.size() / 3);
        if (k == 0) return 0;
        DevBuf<double> dexc;
        dexc.alloc(exc.size());
        CBFM_CUDA(cudaMemcpyAsync(dexc.p, exc.data(), sizeof(double) * exc.size(), cudaMemcpyHostToDevice, st));
        rows.alloc((size_t)k * r->n);
        reduced_rhs_rows(*r, dexc.p, k, rows.p, st);
        exc_all.insert(exc_all.end(), exc.begin(), exc.end());
        return k;
    }
    bool close_if_idle() override {
        std::lock_guard<std::mutex> lk(mu);
        if (nqueued.load() > 0) return false;
        closed = true;
        return true;
    }
};

}  // namespace

extern "C" {

cbfm_status cbfm_assemble_reduced(cbfm_mesh_t mesh, cbfm_cbf_t cbf, cbfm_precision prec, void *stream, cbfm_red_t *out,
                                  int64_t *n_cbf) {
    return guarded([&] {
        StreamScope ss_((cudaStream_t)stream);   // scratch is stream-ordered on the caller's stream
        Mesh *m = (Mesh *)mesh;
        Cbf *c = (Cbf *)cbf;
        check_device(m, H_MESH, "mesh");
        check_device(c, H_CBF, "cbf");
        CBFM_REQUIRE(c->mesh == m, "cbf handle belongs to another mesh");
        CBFM_REQUIRE(out, "NULL out");
        CBFM_REQUIRE(prec == CBFM_FP64 || prec == CBFM_MIXED || prec == CBFM_MIXED_SIMT || prec == CBFM_MIXED_UNFUSED ||
                         prec == CBFM_MIXED_FUSED,
                     "unknown precision");
        *out = nullptr;
        cudaStream_t st = (cudaStream_t)stream;
        std::unique_ptr<Red> r(new Red());
        r->kind = H_RED;
        r->device = m->device;
        r->mesh = m;
        r->cbf = c;
        r->prec = prec;
        r->n = 2 * c->nhalf;
        if (prec == CBFM_FP64) project<double>(*r, st);
        else project<float>(*r, st);
        CBFM_CUDA(cudaStreamSynchronize(st));
        if (n_cbf) *n_cbf = r->n;
        *out = (cbfm_red_t)r.release();
    });
}

cbfm_status cbfm_assemble_mom(cbfm_mesh_t mesh, cbfm_precision prec, void *stream, cbfm_red_t *out, int64_t *n) {
    return guarded([&] {
        StreamScope ss_((cudaStream_t)stream);   // scratch is stream-ordered on the caller's stream
        Mesh *m = (Mesh *)mesh;
        check_device(m, H_MESH, "mesh");
        CBFM_REQUIRE(out, "NULL out");
        CBFM_REQUIRE(prec == CBFM_FP64 || prec == CBFM_MIXED || prec == CBFM_MIXED_SIMT, "unknown precision");
        *out = nullptr;
        cudaStream_t st = (cudaStream_t)stream;
        std::unique_ptr<Red> r(new Red());
        r->kind = H_RED;
        r->device = m->device;
        r->mesh = m;
        r->cbf = nullptr;
        r->prec = prec;
        const int64_t ne = m->h.ne;
        r->n = 2 * ne;
        // Z = [[Ks, Ta], [Tb, Ks]] (Eq. (Z)) from the RWG blocks
        if (prec == CBFM_FP64) {
            DevBuf<z64> Z;
            Z.alloc(3 * (size_t)ne * ne);
            assemble_rwg<double>(*m, Z.p, st);
            r->A64.alloc((size_t)r->n * r->n);
            mom_place<double>(ne, Z.p, r->A64.p, st);
        } else {
            DevBuf<c32> Z;
            Z.alloc(3 * (size_t)ne * ne);
            assemble_rwg<float>(*m, Z.p, st);
            r->A32.alloc((size_t)r->n * r->n);
            mom_place<float>(ne, Z.p, r->A32.p, st);
        }
        CBFM_CUDA(cudaStreamSynchronize(st));
        if (n) *n = r->n;
        *out = (cbfm_red_t)r.release();
    });
}

cbfm_status cbfm_tdiag_setup(cbfm_red_t red, int32_t jacobi, void *stream) {
    return guarded([&] {
        StreamScope ss_((cudaStream_t)stream);   // scratch is stream-ordered on the caller's stream
        Red *r = (Red *)red;
        check_device(r, H_RED, "reduced system");
        if (!tdiag_build(*r, jacobi != 0, (cudaStream_t)stream))
            throw Fail{CBFM_ESINGULAR, "a diagonal entry of the T-diagonal arrangement is zero"};
    });
}

cbfm_status cbfm_assemble_reduced_batch(const cbfm_mesh_t *meshes, const cbfm_cbf_t *cbfs, int32_t count,
                                        cbfm_precision prec, void *stream, cbfm_red_t *out, int64_t *n_cbf) {
    // created handles are freed again if a later wave fails
    std::vector<std::unique_ptr<Red>> made;
    cbfm_status st_ = guarded([&] {
        StreamScope ss_((cudaStream_t)stream);   // scratch is stream-ordered on the caller's stream
        CBFM_REQUIRE(count >= 0, "negative count");
        CBFM_REQUIRE(count == 0 || (meshes && cbfs && out), "NULL array");
        CBFM_REQUIRE(prec == CBFM_MIXED || prec == CBFM_MIXED_FUSED,
                     "batched assembly runs the mixed-precision path (CBFM_MIXED or CBFM_MIXED_FUSED) only");
        for (int32_t k = 0; k < count; ++k) out[k] = nullptr;
        cudaStream_t st = (cudaStream_t)stream;
        std::vector<Mesh *> ms(count);
        std::vector<Cbf *> cs(count);
        for (int32_t k = 0; k < count; ++k) {
            ms[k] = (Mesh *)meshes[k];
            cs[k] = (Cbf *)cbfs[k];
            check_device(ms[k], H_MESH, "mesh");
            check_device(cs[k], H_CBF, "cbf");
            CBFM_REQUIRE(cs[k]->mesh == ms[k], "cbf handle belongs to another mesh");
        }
        made.resize(count);
        auto make = [&](int32_t k) -> Red * {
            std::unique_ptr<Red> r(new Red());
            r->kind = H_RED;
            r->device = ms[k]->device;
            r->mesh = ms[k];
            r->cbf = cs[k];
            r->prec = prec;
            r->n = 2 * cs[k]->nhalf;
            r->A32.alloc((size_t)r->n * r->n);
            made[k] = std::move(r);
            return made[k].get();
        };
        // scatterers whose cells fit the fused kernel: one launch over all their cell pairs
        std::vector<int32_t> rest;
        {
            std::vector<Mesh *> fm;
            std::vector<Cbf *> fc;
            std::vector<c32 *> fa;
            for (int32_t k = 0; k < count; ++k) {
                const bool fused = prec == CBFM_MIXED_FUSED ? fused_fits(*ms[k], *cs[k]) : mixed_takes_fused(*ms[k], *cs[k]);
                if (!fused) {
                    rest.push_back(k);
                    continue;
                }
                Red *r = make(k);
                fm.push_back(ms[k]);
                fc.push_back(cs[k]);
                fa.push_back(r->A32.p);
            }
            assemble_project_fused(fm, fc, fa, st);
        }
        // the others: RWG matrices in memory, in waves of scatterers whose transient
        // operators fit in half of the free device memory and in 6 GiB (larger waves
        // would map fresh memory from the stream-ordered pool on every call)
        size_t free_b = 0, total_b = 0;
        CBFM_CUDA(cudaMemGetInfo(&free_b, &total_b));
        const double budget = std::min(0.5 * (double)free_b, 6.0 * (1ull << 30));
        auto transient = [&](int k) {
            const double nt = (double)ms[k]->h.nt, ne = (double)ms[k]->h.ne, nh = (double)cs[k]->nhalf;
            const double ldz = std::ceil(2.0 * ne / 32.0) * 32.0;
            return 27.0 * nt * nt * 8 + 3.0 * ne * ne * 8 + 6.0 * ne * ldz * 4 + 8.0 * 2 * nh * ldz * 4 +
                   4.0 * nh * nh * 8;
        };
        size_t i0 = 0;
        while (i0 < rest.size()) {
            size_t i1 = i0;
            double used = 0.0;
            while (i1 < rest.size() && (i1 == i0 || used + transient(rest[i1]) <= budget)) used += transient(rest[i1++]);
            std::vector<Mesh *> wm;
            std::vector<Cbf *> wc;
            std::vector<DevBuf<c32>> Z(i1 - i0);
            std::vector<c32 *> Zp, Ap;
            std::vector<const c32 *> Zc;
            for (size_t i = i0; i < i1; ++i) {
                const int32_t k = rest[i];
                Red *r = make(k);
                wm.push_back(ms[k]);
                wc.push_back(cs[k]);
                const int64_t ne = ms[k]->h.ne;
                Z[i - i0].alloc((size_t)3 * ne * ne);
                Zp.push_back(Z[i - i0].p);
                Zc.push_back(Z[i - i0].p);
                Ap.push_back(r->A32.p);
            }
            assemble_rwg_batch<float>(wm, Zp, st);
            project_tc_batch(wm, wc, Zc, Ap, st);
            CBFM_CUDA(cudaStreamSynchronize(st));
            i0 = i1;
        }
        for (int32_t k = 0; k < count; ++k) {
            if (n_cbf) n_cbf[k] = made[k]->n;
            out[k] = (cbfm_red_t)made[k].release();
        }
    });
    return st_;   // on failure `made` frees what was built
}

cbfm_status cbfm_red_export(cbfm_red_t red, double *A, void *stream) {
    return guarded([&] {
        StreamScope ss_((cudaStream_t)stream);   // scratch is stream-ordered on the caller's stream
        Red *r = (Red *)red;
        check_device(r, H_RED, "reduced system");
        CBFM_REQUIRE(A, "NULL A");
        cudaStream_t st = (cudaStream_t)stream;
        int64_t nn = r->n * r->n;
        if (r->cbf == nullptr) {   // conventional MoM: Z in canonical edge order
            DevBuf<z64> t, c;
            const z64 *src = r->A64.p;
            if (r->prec != CBFM_FP64) {
                t.alloc(nn);
                launch_c32_to_z64(r->A32.p, t.p, nn, st);
                src = t.p;
            }
            DevBuf<int32_t> dmap;
            upload(dmap, r->mesh->h.int_of_canon, st);
            c.alloc(nn);
            mom_to_canonical(r->mesh->h.ne, dmap.p, src, c.p, st);
            copy_out(A, c.p, nn * sizeof(z64), st);
            CBFM_CUDA(cudaStreamSynchronize(st));
        } else if (r->prec == CBFM_FP64) {
            copy_out(A, r->A64.p, nn * sizeof(z64), st);
        } else {
            DevBuf<z64> t;
            t.alloc(nn);
            launch_c32_to_z64(r->A32.p, t.p, nn, st);
            copy_out(A, t.p, nn * sizeof(z64), st);
            CBFM_CUDA(cudaStreamSynchronize(st));
        }
        CBFM_CUDA(cudaStreamSynchronize(st));
    });
}

cbfm_status cbfm_red_export_noalloc(cbfm_red_t red, double *A, void *stream) {
    return guarded([&] {
        Red *r = (Red *)red;
        check_device(r, H_RED, "reduced system");
        red_export_noalloc(*r, A, (cudaStream_t)stream);
    });
}

cbfm_status cbfm_cmp_setup(cbfm_red_t red, void *stream) {
    return guarded([&] {
        StreamScope ss_((cudaStream_t)stream);   // scratch is stream-ordered on the caller's stream
        Red *r = (Red *)red;
        check_device(r, H_RED, "reduced system");
        CBFM_REQUIRE(r->cbf != nullptr,
                     "no CBFs: the Calderon preconditioner of the RWG-only system has a singular Gram matrix");
        cudaStream_t st = (cudaStream_t)stream;
        gram_cbf(*r, st);
        const int64_t nh = r->cbf->nhalf, n = r->n;
        // inverse of the first half by Gauss-Jordan (FP64); the second half of G^CBF is
        // minus the adjoint of the first, so its inverse is minus the adjoint of this one
        r->Ginv.alloc((size_t)n * n);
        CBFM_CUDA(cudaMemsetAsync(r->Ginv.p, 0, sizeof(z64) * n * n, st));
        DevBuf<z64> blk, aug;
        DevBuf<int> info;
        blk.alloc((size_t)nh * nh);
        aug.alloc((size_t)2 * nh * nh);
        info.alloc(1);
        CBFM_CUDA(cudaMemsetAsync(info.p, 0, sizeof(int), st));
        {
            ProfScope ps_("k_copy_block", st);
            k_copy_block<<<nblk(nh * nh), 256, 0, st>>>(n, nh, 0, r->G.p, blk.p);
            launched("k_copy_block");
        }
        gauss_jordan_inverse(nh, 1, aug.p, blk.p, info.p, st);
        {
            ProfScope ps_("k_place_block", st);
            k_place_block<<<nblk(nh * nh), 256, 0, st>>>(n, nh, 0, blk.p, r->Ginv.p);
            launched("k_place_block");
            k_place_neg_adjoint<<<nblk(nh * nh), 256, 0, st>>>(n, nh, nh, blk.p, nh, r->Ginv.p);
            launched("k_place_neg_adjoint");
        }
        int hinfo = 0;
        CBFM_CUDA(cudaMemcpyAsync(&hinfo, info.p, sizeof(int), cudaMemcpyDeviceToHost, st));
        CBFM_CUDA(cudaStreamSynchronize(st));
        if (hinfo) throw Fail{CBFM_ESINGULAR, "G^CBF is singular"};
        // B = A (G^CBF)^{-1}: GMRES then needs one product per iteration
        std::vector<GemmDesc> gb{GemmDesc{n, n, n, 0, n, 0, n, 0, n}};
        if (r->prec != CBFM_FP64) {
            r->Ginv32.alloc((size_t)n * n);
            launch_z64_to_c32(r->Ginv.p, r->Ginv32.p, n * n, st);
            r->B32.alloc((size_t)n * n);
            gemm_grouped<float>(gb, 0, 0, r->A32.p, r->Ginv32.p, r->B32.p, false, st);
        } else {
            r->B64.alloc((size_t)n * n);
            gemm_grouped<double>(gb, 0, 0, r->A64.p, r->Ginv.p, r->B64.p, false, st);
        }
        CBFM_CUDA(cudaStreamSynchronize(st));
        r->cmp_ready = true;
    });
}

cbfm_status cbfm_cmp_setup_inexact(cbfm_red_t red, double inner_tol, int32_t inner_maxit, int32_t inner_restart,
                                   void *stream) {
    return guarded([&] {
        StreamScope ss_((cudaStream_t)stream);   // scratch is stream-ordered on the caller's stream
        Red *r = (Red *)red;
        check_device(r, H_RED, "reduced system");
        CBFM_REQUIRE(r->cbf != nullptr,
                     "no CBFs: the Calderon preconditioner of the RWG-only system has a singular Gram matrix");
        CBFM_REQUIRE(inner_tol > 0.0 && inner_maxit >= 1 && inner_restart >= 1,
                     "inner_tol, inner_maxit and inner_restart must be positive");
        cudaStream_t st = (cudaStream_t)stream;
        r->cmp_inexact_ready = false;
        if (r->G.p == nullptr) gram_cbf(*r, st);
        // the inner system: G^CBF (FP64) iterated with its Jacobi operator G D^{-1}, D = diag(G^CBF)
        std::unique_ptr<Red> g(new Red());
        g->kind = H_RED;
        g->device = r->device;
        g->mesh = r->mesh;
        g->cbf = r->cbf;
        g->prec = CBFM_FP64;
        g->n = r->n;
        g->A64.alloc((size_t)r->n * r->n);
        CBFM_CUDA(cudaMemcpyAsync(g->A64.p, r->G.p, sizeof(z64) * r->n * r->n, cudaMemcpyDeviceToDevice, st));
        if (!tdiag_build(*g, true, st, false)) throw Fail{CBFM_ESINGULAR, "a diagonal entry of G^CBF is zero"};
        r->ginner = std::move(g);
        r->inner_tol = inner_tol;
        r->inner_maxit = inner_maxit;
        r->inner_restart = inner_restart;
        r->cmp_inexact_ready = true;
    });
}

cbfm_status cbfm_wait_selftest(int32_t kind, double limit_s, void *stream) {
    return guarded([&] {
        StreamScope ss_((cudaStream_t)stream);
        CBFM_REQUIRE(kind >= 0 && kind <= 2, "kind must be 0, 1 or 2");
        CBFM_REQUIRE(limit_s > 0.0 && limit_s <= 1.0, "limit_s must be in (0, 1]");
        if (wait_selftest(kind, limit_s, (cudaStream_t)stream))
            throw Fail{CBFM_ETIMEOUT, kind == 0 ? "self-test: the grid barrier wait expired"
                                                : "self-test: a cluster barrier wait expired"};
    });
}

cbfm_status cbfm_gram_inverse(const double *A, int64_t n, int32_t nbatch, double *Ainv, void *stream) {
    return guarded([&] {
        StreamScope ss_((cudaStream_t)stream);   // scratch is stream-ordered on the caller's stream
        CBFM_REQUIRE(A && Ainv, "NULL matrix");
        CBFM_REQUIRE(n >= 1 && nbatch >= 1, "n and nbatch must be positive");
        cudaStream_t st = (cudaStream_t)stream;
        const size_t cnt = (size_t)nbatch * n * n;
        DevBuf<z64> blk, aug;
        DevBuf<int> info;
        blk.alloc(cnt);
        aug.alloc(2 * cnt);
        info.alloc(1);
        CBFM_CUDA(cudaMemsetAsync(info.p, 0, sizeof(int), st));
        copy_in(blk.p, A, cnt * sizeof(z64), st);
        gauss_jordan_inverse(n, nbatch, aug.p, blk.p, info.p, st);
        int hinfo = 0;
        CBFM_CUDA(cudaMemcpyAsync(&hinfo, info.p, sizeof(int), cudaMemcpyDeviceToHost, st));
        CBFM_CUDA(cudaStreamSynchronize(st));
        if (hinfo) throw Fail{CBFM_ESINGULAR, "matrix is singular"};
        copy_out(Ainv, blk.p, cnt * sizeof(z64), st);
        CBFM_CUDA(cudaStreamSynchronize(st));
    });
}

cbfm_status cbfm_gram_export(cbfm_red_t red, double *G, void *stream) {
    return guarded([&] {
        StreamScope ss_((cudaStream_t)stream);   // scratch is stream-ordered on the caller's stream
        Red *r = (Red *)red;
        check_device(r, H_RED, "reduced system");
        CBFM_REQUIRE(r->G.p != nullptr, "call cbfm_cmp_setup or cbfm_cmp_setup_inexact first");
        CBFM_REQUIRE(G, "NULL G");
        copy_out(G, r->G.p, r->n * r->n * sizeof(z64), (cudaStream_t)stream);
        CBFM_CUDA(cudaStreamSynchronize((cudaStream_t)stream));
    });
}

cbfm_status cbfm_solve(cbfm_red_t red, const double *exc, int32_t nrhs, double tol, int32_t maxit, int32_t restart,
                       int32_t precond, int32_t solver, double *j_out, const double *obs, int32_t ndir,
                       double *rcs_out, int32_t *iters_out, double *resid_out, void *stream) {
    cbfm_status conv = CBFM_OK;
    cbfm_status st_ = guarded([&] {
        StreamScope ss_((cudaStream_t)stream);   // scratch is stream-ordered on the caller's stream
        Red *r = (Red *)red;
        check_device(r, H_RED, "reduced system");
        CBFM_REQUIRE(exc && nrhs >= 1, "need at least one excitation");
        CBFM_REQUIRE(tol > 0.0 && maxit >= 1 && restart >= 1, "tol, maxit and restart must be positive");
        CBFM_REQUIRE(precond == CBFM_PC_NONE || precond == CBFM_PC_CMP || precond == CBFM_PC_TDIAG ||
                         precond == CBFM_PC_CMP_INEXACT,
                     "precond must be CBFM_PC_NONE, CBFM_PC_CMP, CBFM_PC_TDIAG or CBFM_PC_CMP_INEXACT");
        CBFM_REQUIRE(precond != CBFM_PC_CMP || r->cmp_ready, "CBFM_PC_CMP requires cbfm_cmp_setup");
        CBFM_REQUIRE(precond != CBFM_PC_CMP_INEXACT || r->cmp_inexact_ready,
                     "CBFM_PC_CMP_INEXACT requires cbfm_cmp_setup_inexact");
        CBFM_REQUIRE(precond != CBFM_PC_TDIAG || r->tdiag_ready, "CBFM_PC_TDIAG requires cbfm_tdiag_setup");
        const bool mono = (obs == nullptr && ndir == -1);
        CBFM_REQUIRE(mono || ndir >= 0, "ndir must be >= 0, or -1 with obs == NULL for monostatic");
        CBFM_REQUIRE(mono || ndir == 0 || obs != nullptr, "obs is NULL");
        cudaStream_t st = (cudaStream_t)stream;
        Mesh &m = *r->mesh;
        const int64_t ne = m.h.ne, n = r->n;
        DevBuf<double> dexc, dobs, drcs;
        dexc.alloc(3 * (size_t)nrhs);
        copy_in(dexc.p, exc, 3 * sizeof(double) * nrhs, st);
        DevBuf<z64> b, x, jint;
        b.alloc((size_t)nrhs * n);
        reduced_rhs_rows(*r, dexc.p, nrhs, b.p, st);
        CBFM_REQUIRE(solver == 0 || solver == 1, "solver must be 0 (per right-hand side) or 1 (block)");
        x.alloc((size_t)nrhs * n);
        GmresOut go;
        if (solver == 0) {
            go = gmres_solve(*r, b.p, nrhs, tol, maxit, restart, precond, x.p, st);
        } else {
            for (int r0 = 0; r0 < nrhs; r0 += 128) {
                const int cnt = std::min(128, nrhs - r0);
                GmresOut g = bgmres_solve(*r, b.p + (int64_t)r0 * n, cnt, tol, maxit, restart, precond,
                                          x.p + (int64_t)r0 * n, st);
                go.iters.insert(go.iters.end(), g.iters.begin(), g.iters.end());
                go.resid.insert(go.resid.end(), g.resid.begin(), g.resid.end());
            }
        }
        // j = C^MJ x  (internal order, (2 ne) x nrhs)
        jint.alloc((size_t)2 * ne * nrhs);
        recover_currents(*r, x.p, nrhs, jint.p, st);
        if (rcs_out && (mono || ndir > 0)) {
            int nd = mono ? 1 : ndir;
            if (!mono) {
                dobs.alloc(2 * (size_t)ndir);
                copy_in(dobs.p, obs, 2 * sizeof(double) * ndir, st);
            }
            drcs.alloc((size_t)nrhs * nd * 2);
            launch_farfield(m, jint.p, nrhs, dobs.p, nd, mono, dexc.p, drcs.p, st, r->prec != CBFM_FP64);
            copy_out(rcs_out, drcs.p, sizeof(double) * nrhs * nd * 2, st);
        }
        if (j_out) {
            DevBuf<int32_t> dmap;
            upload(dmap, m.h.int_of_canon, st);
            DevBuf<z64> jc;
            jc.alloc((size_t)2 * ne * nrhs);
            {
                ProfScope ps_("k_to_canonical", st);
                k_to_canonical<<<nblk(2 * ne * nrhs), 256, 0, st>>>(ne, nrhs, dmap.p, jint.p, jc.p);
                launched("k_to_canonical");
            }
            copy_out(j_out, jc.p, sizeof(z64) * 2 * ne * nrhs, st);
            CBFM_CUDA(cudaStreamSynchronize(st));
        }
        CBFM_CUDA(cudaStreamSynchronize(st));
        for (int i = 0; i < nrhs; ++i) {
            if (iters_out) iters_out[i] = go.iters[i] >= 0 ? go.iters[i] : -go.iters[i] - 1;
            if (resid_out) resid_out[i] = go.resid[i];
            if (go.iters[i] < 0) conv = CBFM_ENOCONV;
        }
    });
    if (st_ == CBFM_OK && conv != CBFM_OK) {
        t_err = "GMRES did not converge for at least one right-hand side";
        return conv;
    }
    return st_;
}

cbfm_status cbfm_session_create(cbfm_red_t red, const double *exc, int32_t nrhs, double tol, int32_t maxit,
                                int32_t restart, int32_t precond, cbfm_session_t *out) {
    return guarded([&] {
        Red *r = (Red *)red;
        check_device(r, H_RED, "reduced system");
        CBFM_REQUIRE(out != nullptr, "out is NULL");
        CBFM_REQUIRE(exc && nrhs >= 1 && nrhs <= 128, "a session starts with 1 to 128 excitations");
        CBFM_REQUIRE(tol > 0.0 && maxit >= 1 && restart >= 1, "tol, maxit and restart must be positive");
        CBFM_REQUIRE(precond == CBFM_PC_NONE || precond == CBFM_PC_CMP || precond == CBFM_PC_TDIAG,
                     "precond must be CBFM_PC_NONE, CBFM_PC_CMP or CBFM_PC_TDIAG");
        CBFM_REQUIRE(precond != CBFM_PC_CMP || r->cmp_ready, "CBFM_PC_CMP requires cbfm_cmp_setup");
        CBFM_REQUIRE(precond != CBFM_PC_TDIAG || r->tdiag_ready, "CBFM_PC_TDIAG requires cbfm_tdiag_setup");
        std::unique_ptr<Session> s(new Session());
        s->kind = H_SESSION;
        CBFM_CUDA(cudaGetDevice(&s->device));
        s->r = r;
        s->tol = tol;
        s->maxit = maxit;
        s->restart = restart;
        s->precond = precond;
        s->queued.assign(exc, exc + 3 * (size_t)nrhs);
        s->nqueued.store(nrhs);
        s->accepted = nrhs;
        *out = (cbfm_session_t)s.release();
    });
}

cbfm_status cbfm_session_join(cbfm_session_t sess, const double *exc, int32_t nrhs, int32_t *first_slot) {
    return guarded([&] {
        Session *s = (Session *)sess;
        CBFM_REQUIRE(s != nullptr && s->kind == H_SESSION, "bad session handle");
        CBFM_REQUIRE(exc && nrhs >= 1, "need at least one excitation");
        std::lock_guard<std::mutex> lk(s->mu);
        if (s->closed || s->accepted + nrhs > 128)
            throw Fail{CBFM_EFULL, s->closed ? "the session has finished" : "the session holds 128 right-hand sides"};
        if (first_slot) *first_slot = s->accepted;
        s->queued.insert(s->queued.end(), exc, exc + 3 * (size_t)nrhs);
        s->accepted += nrhs;
        s->nqueued.store((int)(s->queued.size() / 3), std::memory_order_release);
    });
}

cbfm_status cbfm_session_run(cbfm_session_t sess, void *stream) {
    cbfm_status conv = CBFM_OK;
    cbfm_status st_ = guarded([&] {
        StreamScope ss_((cudaStream_t)stream);
        Session *s = (Session *)sess;
        CBFM_REQUIRE(s != nullptr && s->kind == H_SESSION, "bad session handle");
        check_device(s->r, H_RED, "reduced system");
        CBFM_REQUIRE(!s->ran, "a session runs once");
        s->ran = true;
        cudaStream_t st = (cudaStream_t)stream;
        Red &r = *s->r;
        const int64_t ne = r.mesh->h.ne, n = r.n;
        DevBuf<z64> b0, xall;
        const int k0 = s->take(st, b0);
        GmresOut go = bgmres_solve(r, b0.p, k0, s->tol, s->maxit, s->restart, s->precond, nullptr, st, s, &xall);
        {
            std::lock_guard<std::mutex> lk(s->mu);
            s->closed = true;   // joins left waiting (the iteration limit came first) have no result
        }
        const int ns = (int)(s->exc_all.size() / 3);
        CBFM_REQUIRE(ns == (int)go.iters.size(), "session bookkeeping");
        DevBuf<z64> jint;
        DevBuf<double> dexc, drcs;
        jint.alloc((size_t)2 * ne * ns);
        recover_currents(r, xall.p, ns, jint.p, st);
        dexc.alloc(s->exc_all.size());
        CBFM_CUDA(cudaMemcpyAsync(dexc.p, s->exc_all.data(), sizeof(double) * s->exc_all.size(),
                                  cudaMemcpyHostToDevice, st));
        drcs.alloc((size_t)ns * 2);
        launch_farfield(*r.mesh, jint.p, ns, nullptr, 1, true, dexc.p, drcs.p, st, r.prec != CBFM_FP64);
        s->rcs.resize((size_t)ns * 2);
        CBFM_CUDA(cudaMemcpyAsync(s->rcs.data(), drcs.p, sizeof(double) * ns * 2, cudaMemcpyDeviceToHost, st));
        CBFM_CUDA(cudaStreamSynchronize(st));
        s->iters.resize(ns);
        s->resid.resize(ns);
        for (int i = 0; i < ns; ++i) {
            s->iters[i] = go.iters[i] >= 0 ? go.iters[i] : -go.iters[i] - 1;
            s->resid[i] = go.resid[i];
            if (go.iters[i] < 0) conv = CBFM_ENOCONV;
        }
    });
    if (st_ == CBFM_OK && conv != CBFM_OK) {
        t_err = "GMRES did not converge for at least one right-hand side";
        return conv;
    }
    return st_;
}

cbfm_status cbfm_session_results(cbfm_session_t sess, int32_t capacity, double *rcs_out, int32_t *iters_out,
                                 double *resid_out, int32_t *nslots) {
    return guarded([&] {
        Session *s = (Session *)sess;
        CBFM_REQUIRE(s != nullptr && s->kind == H_SESSION, "bad session handle");
        CBFM_REQUIRE(s->ran, "the session has not run");
        const int ns = (int)s->iters.size();
        if (nslots) *nslots = ns;
        CBFM_REQUIRE(capacity >= ns || (!rcs_out && !iters_out && !resid_out), "output capacity too small");
        for (int i = 0; i < ns; ++i) {
            if (rcs_out) {
                rcs_out[2 * i] = s->rcs[2 * i];
                rcs_out[2 * i + 1] = s->rcs[2 * i + 1];
            }
            if (iters_out) iters_out[i] = s->iters[i];
            if (resid_out) resid_out[i] = s->resid[i];
        }
    });
}

void cbfm_free(void *handle) {
    if (!handle) return;
    HandleBase *h = (HandleBase *)handle;
    switch (h->kind) {
        case H_MESH: h->kind = 0; delete (Mesh *)h; break;
        case H_CBF: h->kind = 0; delete (Cbf *)h; break;
        case H_RED: h->kind = 0; delete (Red *)h; break;
        case H_SESSION: h->kind = 0; delete (Session *)h; break;
        default: break;
    }
}

}  // extern "C"
