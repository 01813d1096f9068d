// noalloc.cu -- an export of the reduced matrix that allocates no memory.
//
// cbfm_red_export converts a mixed-precision (complex64) reduced matrix to
// complex128 in a temporary device buffer that it allocates.  Some callers
// cannot allocate device memory at that point: a serving process whose HBM is
// already filled with cached meshes, CBFs and reduced matrices, code running
// under an allocator that forbids cudaMalloc (a memory pool sized at start-up,
// a real-time loop), or a thread that must not synchronise the device the way
// cudaMalloc/cudaFree can.  cbfm_red_export_noalloc does the same conversion
// into a fixed scratch array compiled into the library instead.
//
// The scratch is a file-scope __device__ array of NOALLOC_MAX_ELEMS complex128
// values (4 MiB); every GPU that loads the library holds it until the process
// exits.  In host code its name is only a host-side stand-in, so its device
// address is looked up once per device with cudaGetSymbolAddress (with that
// device current) and passed to the kernel.
#include <mutex>

#include "internal.cuh"

namespace cbfm {

namespace {

constexpr int64_t NOALLOC_MAX_ELEMS = 512 * 512;   // n_cbf <= 512
constexpr int NOALLOC_MAX_DEVICES = 64;

static __device__ __align__(256) z64 g_noalloc_scratch[NOALLOC_MAX_ELEMS];

std::mutex g_sym_mu;
z64 *g_sym_addr[NOALLOC_MAX_DEVICES] = {nullptr};

// Device address of the scratch array on the current device (looked up once).
z64 *scratch_address() {
    int dev = -1;
    CBFM_CUDA(cudaGetDevice(&dev));
    CBFM_REQUIRE(dev >= 0 && dev < NOALLOC_MAX_DEVICES, "device index beyond the no-alloc table");
    std::lock_guard<std::mutex> lk(g_sym_mu);
    if (!g_sym_addr[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p)
            throw Fail{CBFM_ECUDA, std::string("cudaGetSymbolAddress(no-alloc scratch): ") + cudaGetErrorString(e)};
        g_sym_addr[dev] = (z64 *)p;
    }
    return g_sym_addr[dev];
}

__global__ void k_c32_to_z64_scratch(const c32 *__restrict__ src, z64 *__restrict__ dst, int64_t n) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) dst[i] = z64(src[i].re, src[i].im);
}

}  // namespace

// Body of cbfm_red_export_noalloc; the C entry point lives in api.cu.
void red_export_noalloc(Red &r, double *A, cudaStream_t st) {
    const int64_t nn = r.n * r.n;
    CBFM_REQUIRE(nn <= NOALLOC_MAX_ELEMS,
                 "n_cbf = " + std::to_string(r.n) + " exceeds the no-alloc export limit of 512");
    CBFM_REQUIRE(A != nullptr, "NULL A");
    CBFM_REQUIRE(r.cbf != nullptr, "a conventional MoM system is exported with cbfm_red_export");
    if (r.prec == CBFM_FP64) {
        // already complex128: a plain copy, no scratch needed
        copy_out(A, r.A64.p, nn * sizeof(z64), st);
    } else {
        z64 *scratch = scratch_address();
        k_c32_to_z64_scratch<<<(unsigned)((nn + 255) / 256), 256, 0, st>>>(r.A32.p, scratch, nn);
        launched("k_c32_to_z64_scratch");
        copy_out(A, scratch, nn * sizeof(z64), st);
    }
    CBFM_CUDA(cudaStreamSynchronize(st));
}

}  // namespace cbfm
