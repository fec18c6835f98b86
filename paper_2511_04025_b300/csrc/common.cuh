// common.cuh -- shared definitions of libshl (context, errors, workspaces,
// reductions).  Everything in csrc/ is compiled as one translation unit
// (shl.cu) for sm_103a.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <cmath>
#include <cstdarg>
#include <cstddef>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/shl.h"

namespace shl {

constexpr int kBlk = 256;

// Last error text is per context; calls made without a context (argument
// errors before creation) write to a process-wide buffer.
struct ErrState {
    std::string msg;
};

inline ErrState &global_err() {
    static ErrState e;
    return e;
}

}  // namespace shl

// Device workspace cache: named slots of device memory reused across calls
// (re-allocated only when a call needs more bytes than the slot holds).
struct shl_workspace {
    std::map<std::string, std::pair<void *, size_t>> slots;
};

struct shl_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    shl_opts opts{};
    std::string err;
    shl_workspace ws;
    std::recursive_mutex mu;  // serialises public calls on one context
    void *serve = nullptr;    // serving scheduler state (serve.cuh)
    unsigned long long launches = 0;  // kernels launched (telemetry)
    // serving slots: every call runs on `stream`, so workspaces are allocated
    // and freed stream-ordered there (no device-wide synchronisation, which
    // would disturb other slots' CUDA-graph captures)
    bool stream_ordered_alloc = false;
    void *pinned = nullptr;  // host staging of the multigrid setup (page-locked, allocated once)
    // instantiated PCG-iteration graphs by solve shape, refreshed per solve with
    // cudaGraphExecUpdate (an instantiation costs far more than an update)
    std::map<std::string, cudaGraphExec_t> graphs;
    // side streams for independent setup chains (the per-level power
    // iterations of the multigrid setup), forked from and joined back into
    // the calling stream by events; created on first use
    static constexpr int kAux = 4;
    cudaStream_t aux[kAux] = {};
    cudaEvent_t aux_ev[kAux + 1] = {};
};

namespace shl {

inline int set_err(shl_ctx *ctx, int code, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    if (ctx)
        ctx->err = buf;
    else
        global_err().msg = buf;
    return code;
}

#define SHL_CUDA(ctx, call)                                                                            \
    do {                                                                                               \
        cudaError_t e_ = (call);                                                                       \
        if (e_ != cudaSuccess)                                                                         \
            return shl::set_err((ctx), SHL_ECUDA, "%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_), \
                                __FILE__, __LINE__);                                                   \
    } while (0)

#define SHL_TRY(x)                   \
    do {                             \
        int s_ = (x);                \
        if (s_ != SHL_OK) return s_; \
    } while (0)

// Get (allocating or growing) a named device workspace slot.  Fresh slots are
// zero-filled (reduction tickets rely on it).
inline int ws_get(shl_ctx *ctx, const std::string &name, size_t bytes, void **out) {
    auto &slot = ctx->ws.slots[name];
    if (slot.second < bytes) {
        const bool so = ctx->stream_ordered_alloc;
        if (slot.first) {
            if (so) {
                cudaFreeAsync(slot.first, ctx->stream);
            } else {
                // the old buffer may still be in use on the caller's stream
                cudaDeviceSynchronize();
                cudaFree(slot.first);
            }
        }
        slot.first = nullptr;
        slot.second = 0;
        size_t sz = bytes < 256 ? 256 : bytes;
        cudaError_t e = so ? cudaMallocAsync(&slot.first, sz, ctx->stream) : cudaMalloc(&slot.first, sz);
        if (e != cudaSuccess) {
            cudaGetLastError();
            slot.first = nullptr;
            return set_err(ctx, SHL_ENOMEM, "device allocation of %zu bytes for workspace '%s' failed: %s", sz,
                           name.c_str(), cudaGetErrorString(e));
        }
        slot.second = sz;
        // zero-fill ordered before any later use on any stream: the context's
        // stream is synchronised (a legacy-stream memset would not be ordered
        // with the non-blocking streams the work runs on)
        e = cudaMemsetAsync(slot.first, 0, sz, ctx->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
        if (e != cudaSuccess) return set_err(ctx, SHL_ECUDA, "workspace zero-fill: %s", cudaGetErrorString(e));
    }
    *out = slot.first;
    return SHL_OK;
}

template <typename T>
inline int ws_get_t(shl_ctx *ctx, const std::string &name, size_t count, T **out) {
    void *p = nullptr;
    int s = ws_get(ctx, name, count * sizeof(T), &p);
    *out = static_cast<T *>(p);
    return s;
}

inline void ws_free_all(shl_ctx *ctx) {
    for (auto &kv : ctx->graphs)
        if (kv.second) cudaGraphExecDestroy(kv.second);
    ctx->graphs.clear();
    for (auto &kv : ctx->ws.slots)
        if (kv.second.first) {
            if (ctx->stream_ordered_alloc)
                cudaFreeAsync(kv.second.first, ctx->stream);
            else
                cudaFree(kv.second.first);
        }
    if (ctx->stream_ordered_alloc) cudaStreamSynchronize(ctx->stream);
    ctx->ws.slots.clear();
    if (ctx->pinned) {
        cudaFreeHost(ctx->pinned);
        ctx->pinned = nullptr;
    }
}

inline cudaStream_t pick_stream(shl_ctx *ctx, void *s) { return s ? static_cast<cudaStream_t>(s) : ctx->stream; }

// The context's side streams and their fork/join events (created once).
inline int aux_streams(shl_ctx *ctx) {
    if (ctx->aux[0]) return SHL_OK;
    for (int i = 0; i < shl_ctx::kAux; ++i)
        SHL_CUDA(ctx, cudaStreamCreateWithFlags(&ctx->aux[i], cudaStreamNonBlocking));
    for (int i = 0; i <= shl_ctx::kAux; ++i)
        SHL_CUDA(ctx, cudaEventCreateWithFlags(&ctx->aux_ev[i], cudaEventDisableTiming));
    return SHL_OK;
}

// Releases the side streams (after the context's work has finished).
inline void aux_release(shl_ctx *ctx) {
    for (int i = 0; i < shl_ctx::kAux; ++i)
        if (ctx->aux[i]) {
            cudaStreamSynchronize(ctx->aux[i]);
            cudaStreamDestroy(ctx->aux[i]);
            ctx->aux[i] = nullptr;
        }
    for (int i = 0; i <= shl_ctx::kAux; ++i)
        if (ctx->aux_ev[i]) {
            cudaEventDestroy(ctx->aux_ev[i]);
            ctx->aux_ev[i] = nullptr;
        }
}

__host__ __device__ inline int wrapi(int v, int r) {
    v %= r;
    return v < 0 ? v + r : v;
}

// ---------------------------------------------------------------------------
// Programmatic dependent launch.  Kernels of the PCG iteration start with
// pdl_wait() (nothing of the preceding kernel is read or overwritten before
// it has completed and its memory is visible) and then pdl_trigger() (the
// next kernel may be launched once every CTA of this one has started), so the
// next launch overlaps this kernel's tail instead of following it.  Both are
// no-ops for an ordinary launch.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;\n" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;\n" ::: "memory"); }
__device__ __forceinline__ void pdl_enter() {
    pdl_wait();
    pdl_trigger();
}

// ---------------------------------------------------------------------------
// Deterministic grid reductions: every block writes its partial sums to
// partial[block*NV + v]; the last block to finish (ticket counter) combines
// the partials in a fixed order.  Bitwise reproducible for a fixed launch
// shape.  Blocks must be a multiple of 32 threads.
// ---------------------------------------------------------------------------
template <int NV>
__device__ inline void block_reduce_store(double (&v)[NV], double *partial, int block_id) {
    __shared__ double red[NV][32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nwarps = (blockDim.x + 31) >> 5;
#pragma unroll
    for (int k = 0; k < NV; ++k) {
        double s = v[k];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (lane == 0) red[k][warp] = s;
    }
    __syncthreads();
    if (threadIdx.x < NV) {
        double s = 0.0;
        for (int w = 0; w < nwarps; ++w) s += red[threadIdx.x][w];
        partial[(size_t)block_id * NV + threadIdx.x] = s;
    }
}

// Double-float arithmetic (a value carried as hi + lo in two floats) by
// error-free transformations: Knuth's TwoSum gives s + e = a + b exactly.
// Used where FP32 kernels combine compensated partial sums across a block:
// B300's FP64 pipe is very narrow (one FP64 warp instruction occupies it for
// ~16 cycles), so an FP64 shuffle tree in every block, or every thread
// recomputing the same FP64 totals, costs microseconds at a kernel's tail.
__host__ __device__ __forceinline__ float2 two_sum(float a, float b) {
    const float s = a + b, bb = s - a;
    return make_float2(s, (a - (s - bb)) + (b - bb));
}
__host__ __device__ __forceinline__ float2 df_add(float2 x, float2 y) {
    const float2 t = two_sum(x.x, y.x);
    const float lo = t.y + (x.y + y.y);
    const float hi = t.x + lo;
    return make_float2(hi, lo - (hi - t.x));
}

// Block sums of NV double-float values, returned in FP64 to every thread
// (fixed order: xor shuffle tree, then warps in order; one FP64 add per value).
template <int NV>
__device__ inline void block_sum_df(const float2 (&v)[NV], double (&out)[NV]) {
    __shared__ float2 red[NV][32];
    __shared__ double res[NV];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nwarps = (blockDim.x + 31) >> 5;
#pragma unroll
    for (int k = 0; k < NV; ++k) {
        float2 s = v[k];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1)
            s = df_add(s, make_float2(__shfl_xor_sync(0xffffffffu, s.x, o), __shfl_xor_sync(0xffffffffu, s.y, o)));
        if (lane == 0) red[k][warp] = s;
    }
    __syncthreads();
    if (threadIdx.x < NV) {
        float2 s = red[threadIdx.x][0];
        for (int w = 1; w < nwarps; ++w) s = df_add(s, red[threadIdx.x][w]);
        res[threadIdx.x] = (double)s.x + (double)s.y;
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < NV; ++k) out[k] = res[k];
}

// Double-float number (hi + lo, |lo| <= ulp(hi) / 2; about 48 significant
// bits) with FP32 arithmetic only: sums by TwoSum, products by the FMA-exact
// product error (Dekker, Knuth; the sloppy double-float addition, whose error
// is bounded relative to the operands, which a residual f - K x needs).  The
// FP32-with-refinement solver forms its true residuals in this type: on B300
// that is ~3x faster than FP64, whose pipe is narrow.
struct __align__(8) dfloat {
    float hi, lo;
    dfloat() = default;
    __host__ __device__ constexpr dfloat(float h, float l) : hi(h), lo(l) {}
    __host__ __device__ constexpr dfloat(double d) : hi((float)d), lo((float)(d - (double)(float)d)) {}
    __host__ __device__ explicit operator double() const { return (double)hi + (double)lo; }
};
__host__ __device__ __forceinline__ dfloat operator+(dfloat a, dfloat b) {
    const float s = a.hi + b.hi, bb = s - a.hi;
    const float e = (a.hi - (s - bb)) + (b.hi - bb) + (a.lo + b.lo);
    const float hi = s + e;
    return dfloat(hi, e - (hi - s));
}
__host__ __device__ __forceinline__ dfloat operator-(dfloat a) { return dfloat(-a.hi, -a.lo); }
__host__ __device__ __forceinline__ dfloat operator-(dfloat a, dfloat b) { return a + (-b); }
__host__ __device__ __forceinline__ dfloat operator*(dfloat a, dfloat b) {
    const float p = a.hi * b.hi;
    float e = fmaf(a.hi, b.hi, -p);
    e = fmaf(a.hi, b.lo, fmaf(a.lo, b.hi, e));
    const float hi = p + e;
    return dfloat(hi, e - (hi - p));
}
__host__ __device__ __forceinline__ dfloat &operator+=(dfloat &a, dfloat b) { return a = a + b; }

// An exactly zero element modulus: a culled element of the active set
// (Sec. 4.2.1), whose stiffness contributions are exact zeros.
__host__ __device__ __forceinline__ bool zero_modulus(float v) { return v == 0.0f; }
__host__ __device__ __forceinline__ bool zero_modulus(double v) { return v == 0.0; }
__host__ __device__ __forceinline__ bool zero_modulus(dfloat v) { return v.hi == 0.0f && v.lo == 0.0f; }

// Conversions of the 18 planes (N values each) of the load cases in `mask`.
// (one thread per node and its 18 planes: no per-element division)
__global__ void to_dfloat_kernel(size_t N, int mask, const double *__restrict__ x, dfloat *__restrict__ y) {
    for (size_t n = blockIdx.x * (size_t)blockDim.x + threadIdx.x; n < N; n += (size_t)gridDim.x * blockDim.x)
#pragma unroll
        for (int pl = 0; pl < 18; ++pl)
            if ((mask >> (pl / 3)) & 1) y[(size_t)pl * N + n] = dfloat(x[(size_t)pl * N + n]);
}
// in place: element i is read as a dfloat and written back as a double
__global__ void dfloat_to_double_kernel(size_t N, int mask, double *xy) {
    const dfloat *y = reinterpret_cast<const dfloat *>(xy);
    for (size_t n = blockIdx.x * (size_t)blockDim.x + threadIdx.x; n < N; n += (size_t)gridDim.x * blockDim.x)
#pragma unroll
        for (int pl = 0; pl < 18; ++pl)
            if ((mask >> (pl / 3)) & 1) {
                const size_t i = (size_t)pl * N + n;
                const dfloat v = y[i];
                xy[i] = (double)v;
            }
}

// Per-thread dot-product accumulator.  FP64 vectors accumulate in FP64.  FP32
// vectors accumulate each thread's few products with compensated (Kahan)
// FP32 summation and hand the result to the FP64 block/grid reduction: the
// per-element work stays on the FP32 pipes (B300 has a very low FP64 rate)
// while the accumulated sum keeps FP64-class accuracy.
template <typename T>
struct DotAcc;
template <>
struct DotAcc<double> {
    double s = 0.0;
    __device__ __forceinline__ void add(double x) { s += x; }
    __device__ __forceinline__ double get() const { return s; }
};
template <>
struct DotAcc<dfloat> {
    dfloat s = dfloat(0.0f, 0.0f);
    __device__ __forceinline__ void add(dfloat x) { s += x; }
    __device__ __forceinline__ double get() const { return (double)s; }
};
template <>
struct DotAcc<float> {
    float s = 0.0f, c = 0.0f;
    __device__ __forceinline__ void add(float x) {
        const float y = x - c;
        const float t = s + y;
        c = (t - s) - y;
        s = t;
    }
    __device__ __forceinline__ double get() const { return (double)s - (double)c; }
    __device__ __forceinline__ float2 get_df() const { return two_sum(s, -c); }  // hi + lo = s - c exactly
};

// Returns true in every thread of the block that finished last.  Resets the
// ticket for the next launch.
__device__ inline bool last_block_ticket(unsigned *ticket, unsigned nblocks) {
    __shared__ bool is_last;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned t = atomicAdd(ticket, 1u);
        is_last = (t == nblocks - 1);
        if (is_last) *ticket = 0;
    }
    __syncthreads();
    if (is_last) __threadfence();
    return is_last;
}

// Sum partial[b*NV + v] over blocks (run by the last block).  Thread t adds
// blocks t, t+blockDim, ... in order, then a fixed shuffle/shared-memory
// tree combines the threads: the result depends only on the launch shape.
// out[v] is written by thread 0 and visible to the whole block on return.
template <int NV>
__device__ inline void sum_partials_ordered(const double *partial, unsigned nblocks, double *out) {
    __shared__ double red[NV][32];
    double s[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) s[v] = 0.0;
    for (unsigned b = threadIdx.x; b < nblocks; b += blockDim.x)
#pragma unroll
        for (int v = 0; v < NV; ++v) s[v] += __ldcg(partial + (size_t)b * NV + v);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nwarps = (blockDim.x + 31) >> 5;
#pragma unroll
    for (int v = 0; v < NV; ++v) {
        double x = s[v];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
        if (lane == 0) red[v][warp] = x;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int v = 0; v < NV; ++v) {
            double x = 0.0;
            for (int w = 0; w < nwarps; ++w) x += red[v][w];
            out[v] = x;
        }
    }
    __syncthreads();
}

}  // namespace shl
