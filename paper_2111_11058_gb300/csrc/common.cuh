// common.cuh -- shared device/host helpers of the CBFM library (sm_103a).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>
#include <string>

#include "../../include/cbfm.h"

namespace cbfm {

// ------------------------------------------------------------------ errors
void set_error(const std::string &msg);
extern std::atomic<int64_t> g_launches;

struct Fail {
    cbfm_status st;
    std::string msg;
};

#define CBFM_CUDA(call)                                                                    \
    do {                                                                                   \
        cudaError_t e_ = (call);                                                           \
        if (e_ != cudaSuccess)                                                             \
            throw ::cbfm::Fail{CBFM_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_)}; \
    } while (0)

#define CBFM_REQUIRE(cond, msg)                                                            \
    do {                                                                                   \
        if (!(cond)) throw ::cbfm::Fail{CBFM_EINVAL, std::string(msg)};                     \
    } while (0)

// Optional per-kernel timing with CUDA events on the launching stream
// (cbfm_profile): a scope records an event pair around one launch; pairs are
// resolved and accumulated per kernel name when an API call finishes.
extern std::atomic<bool> g_prof;
int prof_start(const char *name, cudaStream_t st);
void prof_stop(int token, cudaStream_t st);
void prof_flush();
// algorithmic work attributed to a kernel name (FP operations, bytes), reported by cbfm_profile_read
void prof_add_work(const char *name, double flop, double bytes);
struct ProfScope {
    int tok;
    cudaStream_t st;
    ProfScope(const char *name, cudaStream_t s) : tok(g_prof.load(std::memory_order_relaxed) ? prof_start(name, s) : -1), st(s) {}
    ~ProfScope() {
        if (tok >= 0) prof_stop(tok, st);
    }
};

// Checks the last launch and counts it.
inline void launched(const char *name) {
    cudaError_t e = cudaGetLastError();
    g_launches.fetch_add(1, std::memory_order_relaxed);
    if (e != cudaSuccess) throw Fail{CBFM_ECUDA, std::string("launch ") + name + ": " + cudaGetErrorString(e)};
}

// ------------------------------------------------------------ complex type
template <typename T>
struct cx {
    T re, im;
    cx() = default;
    __host__ __device__ cx(T r, T i = 0) : re(r), im(i) {}
};
typedef cx<double> z64;   // complex128
typedef cx<float> c32;    // complex64

template <typename T> __host__ __device__ inline cx<T> operator+(cx<T> a, cx<T> b) { return cx<T>(a.re + b.re, a.im + b.im); }
template <typename T> __host__ __device__ inline cx<T> operator-(cx<T> a, cx<T> b) { return cx<T>(a.re - b.re, a.im - b.im); }
template <typename T> __host__ __device__ inline cx<T> operator-(cx<T> a) { return cx<T>(-a.re, -a.im); }
template <typename T> __host__ __device__ inline cx<T> operator*(cx<T> a, cx<T> b) {
    return cx<T>(a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re);
}
template <typename T> __host__ __device__ inline cx<T> operator*(T s, cx<T> a) { return cx<T>(s * a.re, s * a.im); }
template <typename T> __host__ __device__ inline cx<T> operator*(cx<T> a, T s) { return cx<T>(s * a.re, s * a.im); }
template <typename T> __host__ __device__ inline cx<T> &operator+=(cx<T> &a, cx<T> b) { a.re += b.re; a.im += b.im; return a; }
template <typename T> __host__ __device__ inline cx<T> &operator-=(cx<T> &a, cx<T> b) { a.re -= b.re; a.im -= b.im; return a; }
template <typename T> __host__ __device__ inline cx<T> conj(cx<T> a) { return cx<T>(a.re, -a.im); }
template <typename T> __host__ __device__ inline T norm2(cx<T> a) { return a.re * a.re + a.im * a.im; }
template <typename T> __host__ __device__ inline cx<T> cdiv(cx<T> a, cx<T> b) {
    T d = b.re * b.re + b.im * b.im;
    return cx<T>((a.re * b.re + a.im * b.im) / d, (a.im * b.re - a.re * b.im) / d);
}
// a += b * c
template <typename T> __host__ __device__ inline void cfma(cx<T> &a, cx<T> b, cx<T> c) {
    a.re = a.re + b.re * c.re - b.im * c.im;
    a.im = a.im + b.re * c.im + b.im * c.re;
}
// a += conj(b) * c
template <typename T> __host__ __device__ inline void cfmaconj(cx<T> &a, cx<T> b, cx<T> c) {
    a.re = a.re + b.re * c.re + b.im * c.im;
    a.im = a.im + b.re * c.im - b.im * c.re;
}

// ------------------------------------------------------------ FP32 trig
// sin/cos of x (|x| < 2^22 * 2 pi) with a two-constant Cody-Waite reduction
// by 2 pi (round to nearest multiple with the 1.5*2^23 shifter) and the
// hardware approximation on [-pi, pi].
__device__ __forceinline__ void sincos_red(float x, float *s, float *c) {
    const float INV2PI = 0.159154943091895335768883763372514362f;
    const float TWOPI_HI = 6.28318548202514648437500f;      // float(2 pi)
    const float TWOPI_LO = -1.7484555314695172e-7f;         // 2 pi - TWOPI_HI
    const float SHIFT = 12582912.0f;                        // 1.5 * 2^23
    float n = __fadd_rn(__fmaf_rn(x, INV2PI, SHIFT), -SHIFT);
    float r = __fmaf_rn(-n, TWOPI_HI, x);
    r = __fmaf_rn(-n, TWOPI_LO, r);
    __sincosf(r, s, c);
}
__device__ __forceinline__ void sincos_red(double x, double *s, double *c) { sincos(x, s, c); }
// ------------------------------------------------------------ constants
constexpr double PI = 3.14159265358979323846;
constexpr double ETA0 = 376.730313668;   // mu0 c (CODATA 2018)
constexpr double K0 = 2.0 * PI;          // lengths in free-space wavelengths

// ------------------------------------------------- triangle record layout
// Per-triangle record (FP64 master and FP32 copy share the layout):
//   [0,21)  7 quadrature points (x,y,z)      [21,28) weights * area
//   [28,37) vertices p_0..p_2 (x,y,z)        [37,40) c_a = sign_a l_a / (2 A)
//   [40,43) centroid                         [43]    longest edge
//   [44,47) FP32 copy only: low parts of the centroid (centroid = hi + lo)
//   [47]    padding
constexpr int TRI_REC = 48;
constexpr int TR_Q = 0, TR_W = 21, TR_P = 28, TR_C = 37, TR_CEN = 40, TR_H = 43, TR_CLO = 44;

// ---------------------------------------------------------- device memory
// The stream of the API call that runs on this thread.  Scratch buffers
// allocated during a call come from the stream-ordered pool on that stream and
// go back to it on the same stream, so concurrent calls on different streams
// do not synchronise the device through cudaMalloc / cudaFree.
struct CallStream {
    cudaStream_t st = nullptr;
    bool valid = false;
};
extern thread_local CallStream g_call;
void pool_setup();   // once per device: keep freed pool memory cached for the next call

struct StreamScope {
    CallStream saved;
    explicit StreamScope(cudaStream_t s) : saved(g_call) {
        pool_setup();
        g_call.st = s;
        g_call.valid = true;
    }
    ~StreamScope() { g_call = saved; }
    StreamScope(const StreamScope &) = delete;
    StreamScope &operator=(const StreamScope &) = delete;
};

// Device buffer.  Inside an API call it is stream-ordered on the call's
// stream; a buffer that outlives the call (owned by a handle, or released
// from another call or stream) is returned with cudaFree, which also accepts
// pool memory.
template <typename T>
struct DevBuf {
    T *p = nullptr;
    size_t n = 0;
    cudaStream_t st = nullptr;
    bool pooled = false;
    DevBuf() = default;
    DevBuf(const DevBuf &) = delete;
    DevBuf &operator=(const DevBuf &) = delete;
    ~DevBuf() { release(); }
    void release() {
        if (p) {
            if (pooled && g_call.valid && g_call.st == st) cudaFreeAsync(p, st);
            else cudaFree(p);
        }
        p = nullptr;
        n = 0;
        pooled = false;
    }
    void alloc(size_t count) {
        release();
        if (count == 0) return;
        cudaError_t e;
        if (g_call.valid) {
            e = cudaMallocAsync((void **)&p, count * sizeof(T), g_call.st);
            pooled = e == cudaSuccess;
            st = g_call.st;
        } else {
            e = cudaMalloc((void **)&p, count * sizeof(T));
        }
        if (e != cudaSuccess) {
            p = nullptr;
            pooled = false;
            throw Fail{CBFM_ENOMEM, std::string("device allocation of ") + std::to_string(count * sizeof(T)) +
                                        " bytes: " + cudaGetErrorString(e)};
        }
        n = count;
    }
    // hand the allocation to another buffer (it will be returned with cudaFree)
    void give(DevBuf &dst) {
        dst.release();
        dst.p = p;
        dst.n = n;
        p = nullptr;
        n = 0;
        pooled = false;
    }
};

// streaming multiprocessors of the current device (queried once per device)
int sm_count();

// copies that accept host or device sources/destinations
void copy_in(void *dst_dev, const void *src_any, size_t bytes, cudaStream_t st);
void copy_out(void *dst_any, const void *src_dev, size_t bytes, cudaStream_t st);
bool is_device_ptr(const void *p);

}  // namespace cbfm
