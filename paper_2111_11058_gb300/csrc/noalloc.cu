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
// values (4 MiB).  CUDA loads a module (and with it this array) on a device
// lazily, the first time something in it is used, so the library looks the
// array up during the first API call on each device (noalloc_prepare, called
// from pool_setup) -- that first call is where the 4 MiB is taken, before the
// caller can have filled device memory.  In host code the array's name is only
// a host-side stand-in; its device address comes from cudaGetSymbolAddress
// with the device current, on every call (no cached address survives a
// context reset).
#include "internal.cuh"

namespace cbfm {

namespace {

constexpr int64_t NOALLOC_MAX_ELEMS = 512 * 512;   // n_cbf <= 512

static __device__ __align__(256) z64 g_noalloc_scratch[NOALLOC_MAX_ELEMS];

// Device address of the scratch array on the current device.
z64 *scratch_address() {
    void *p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p)
        throw Fail{CBFM_ECUDA, std::string("cudaGetSymbolAddress(no-alloc scratch): ") + cudaGetErrorString(e)};
    return (z64 *)p;
}

__global__ void k_c32_to_z64_scratch(const c32 *__restrict__ src, z64 *__restrict__ dst, int64_t n) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) dst[i] = z64(src[i].re, src[i].im);
}

}  // namespace

// Loads this file's module (and its scratch array) on the current device; run
// once per device by the library's first API call there.  Errors are left to
// the export itself to report.
void noalloc_prepare() {
    void *p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess) cudaGetLastError();
}

// Body of cbfm_red_export_noalloc; the C entry point lives in api.cu.
void red_export_noalloc(Red &r, double *A, cudaStream_t st) {
    CBFM_REQUIRE(A != nullptr, "NULL A");
    CBFM_REQUIRE(r.cbf != nullptr, "a conventional MoM system is exported with cbfm_red_export");
    const int64_t nn = r.n * r.n;
    CBFM_REQUIRE(nn <= NOALLOC_MAX_ELEMS,
                 "n_cbf = " + std::to_string(r.n) + " exceeds the no-alloc export limit of 512");
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
