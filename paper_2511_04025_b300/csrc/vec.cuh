// vec.cuh -- the per-iteration vector kernels of the batched PCG (Sec. 4.2.2:
// six load cases in the same kernels, per-case convergence and skip), laid
// out for bandwidth: every block works on one load case k (its three planes)
// and a strided range of 16-byte chunks (float4 / double2) of those planes,
// so loads are vectorised and coalesced and the case's scalars are uniform
// in the block.  The grid is 6 x bpk blocks, capped so that all of it is
// resident at once (one wave, no tail).
//
// Fused multigrid smoothing (fine level, 3x3 block-Jacobi D^-1 stored [9][N]):
//   vec_update  (MG mode) also writes the first pre-smoothing step z = w D^-1 r;
//   vec_jacobi_rz  does the last post-smoothing step z += w D^-1 (r - t) and
//                  the r.z product that gives beta.
// Reductions are deterministic: per-block partials, combined by the last
// block in a fixed order.
#pragma once

#include "apply.cuh"

namespace shl {

constexpr int kVecThreads = 256;
constexpr int kVecBlocksPerSM = 4;  // register budget 64 per thread: one wave of 6 x bpk blocks

// Launch shape of the vector kernels for n nodes.  With a chunk list (the
// active set's chunks, ascending) the kernels visit only the listed chunks:
// the others hold nodes with no active element, whose rows and columns of K
// and (block-)Jacobi inverses are zero, so nothing there can reach an active
// node or a dot product.
struct VecGeom {
    int V = 1;          // elements per chunk (16 bytes, or 1 for ragged sizes)
    size_t chunks = 0;  // chunks per plane (the loop bound: listed chunks when list != null)
    int bpk = 1;        // blocks per load case
    const unsigned *list = nullptr;  // chunk indices, or null for all chunks
    int blocks() const { return 6 * bpk; }
    __host__ __device__ size_t chunk(size_t i) const { return list ? (size_t)list[i] : i; }
};

inline int vec_bpk(size_t chunks) {
    size_t b = (chunks + kVecThreads - 1) / kVecThreads;
    const size_t cap = 148 * kVecBlocksPerSM / 6;  // the whole grid resident at once
    if (b > cap) b = cap;
    if (b < 1) b = 1;
    return (int)b;
}

template <typename T>
inline VecGeom vec_geom(size_t n) {
    VecGeom g;
    g.V = (n % (16 / sizeof(T)) == 0) ? (int)(16 / sizeof(T)) : 1;
    g.chunks = n / g.V;
    g.bpk = vec_bpk(g.chunks);
    return g;
}

// Active chunks of V consecutive nodes (a node is active when one of its 8
// incident elements has a positive density; den: mask bytes or culled rho),
// compacted in ascending order: per-block flags and counts, a one-block scan,
// then an ordered write.  kChunkBlock chunks per block of kVecThreads threads.
constexpr int kChunkPerThread = 4, kChunkBlock = kVecThreads * kChunkPerThread;

__device__ inline bool chunk_active(int r, int V, const uint8_t *mask, const double *rho, size_t c) {
    const size_t N = (size_t)r * r * r;
    for (int e = 0; e < V; ++e) {
        const size_t n = c * V + e;
        if (n >= N) return false;
        const int ix = n % r, iy = (n / r) % r, iz = n / ((size_t)r * r);
        for (int b = 0; b < 8; ++b) {
            const size_t el = ((size_t)wrapi(iz - (b >> 2), r) * r + wrapi(iy - ((b >> 1) & 1), r)) * r +
                              wrapi(ix - (b & 1), r);
            if (rho ? rho[el] > 0.0 : mask[el] != 0) return true;
        }
    }
    return false;
}

__global__ void __launch_bounds__(kVecThreads) chunk_count_kernel(int r, int V, size_t nchunks, const uint8_t *mask,
                                                                   const double *rho, unsigned *counts) {
    __shared__ unsigned wsum[kVecThreads / 32];
    unsigned cnt = 0;
    for (int u = 0; u < kChunkPerThread; ++u) {
        const size_t c = (size_t)blockIdx.x * kChunkBlock + threadIdx.x * kChunkPerThread + u;
        if (c < nchunks && chunk_active(r, V, mask, rho, c)) ++cnt;
    }
    for (int o = 16; o > 0; o >>= 1) cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
    if ((threadIdx.x & 31) == 0) wsum[threadIdx.x >> 5] = cnt;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned t = 0;
        for (int w = 0; w < kVecThreads / 32; ++w) t += wsum[w];
        counts[blockIdx.x] = t;
    }
}

// One block: counts[b] -> exclusive offsets in place; total into *total.
__global__ void __launch_bounds__(1024) chunk_scan_kernel(int nb, unsigned *counts, unsigned *total) {
    __shared__ unsigned carry;
    __shared__ unsigned wsum[32];
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int base = 0; base < nb; base += 1024) {
        const int i = base + threadIdx.x;
        const unsigned v = i < nb ? counts[i] : 0;
        unsigned x = v;  // inclusive warp scan
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned y = __shfl_up_sync(0xffffffffu, x, o);
            if ((threadIdx.x & 31) >= o) x += y;
        }
        if ((threadIdx.x & 31) == 31) wsum[threadIdx.x >> 5] = x;
        __syncthreads();
        unsigned before = carry;
        for (int w = 0; w < (int)(threadIdx.x >> 5); ++w) before += wsum[w];
        if (i < nb) counts[i] = before + x - v;
        __syncthreads();
        if (threadIdx.x == 1023) carry = before + x;
        __syncthreads();
    }
    if (threadIdx.x == 0) *total = carry;
}

__global__ void __launch_bounds__(kVecThreads) chunk_write_kernel(int r, int V, size_t nchunks, const uint8_t *mask,
                                                                   const double *rho, const unsigned *offsets,
                                                                   unsigned *list) {
    __shared__ unsigned wsum[kVecThreads / 32];
    bool f[kChunkPerThread];
    unsigned cnt = 0;
    for (int u = 0; u < kChunkPerThread; ++u) {
        const size_t c = (size_t)blockIdx.x * kChunkBlock + threadIdx.x * kChunkPerThread + u;
        f[u] = c < nchunks && chunk_active(r, V, mask, rho, c);
        cnt += f[u];
    }
    unsigned x = cnt;  // inclusive scan over the block
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned y = __shfl_up_sync(0xffffffffu, x, o);
        if ((threadIdx.x & 31) >= o) x += y;
    }
    if ((threadIdx.x & 31) == 31) wsum[threadIdx.x >> 5] = x;
    __syncthreads();
    unsigned pos = offsets[blockIdx.x] + x - cnt;
    for (int w = 0; w < (int)(threadIdx.x >> 5); ++w) pos += wsum[w];
    for (int u = 0; u < kChunkPerThread; ++u)
        if (f[u]) list[pos++] = (unsigned)((size_t)blockIdx.x * kChunkBlock + threadIdx.x * kChunkPerThread + u);
}

template <typename T, int V>
struct Chunk {
    T v[V];
};

template <typename T, int V>
__device__ __forceinline__ Chunk<T, V> ldc(const T *p) {
    Chunk<T, V> c;
    if constexpr (V * sizeof(T) == 16) {
        if constexpr (sizeof(T) == 4) {
            const float4 t = *reinterpret_cast<const float4 *>(p);
            c.v[0] = t.x, c.v[1] = t.y, c.v[2] = t.z, c.v[3] = t.w;
        } else {
            const double2 t = *reinterpret_cast<const double2 *>(p);
            c.v[0] = t.x, c.v[1] = t.y;
        }
    } else {
#pragma unroll
        for (int e = 0; e < V; ++e) c.v[e] = p[e];
    }
    return c;
}

template <typename T, int V>
__device__ __forceinline__ void stc(T *p, const Chunk<T, V> &c) {
    if constexpr (V * sizeof(T) == 16) {
        if constexpr (sizeof(T) == 4)
            *reinterpret_cast<float4 *>(p) = make_float4(c.v[0], c.v[1], c.v[2], c.v[3]);
        else
            *reinterpret_cast<double2 *>(p) = make_double2(c.v[0], c.v[1]);
    } else {
#pragma unroll
        for (int e = 0; e < V; ++e) p[e] = c.v[e];
    }
}

// Last block, warp 0 only (the caller's other warps have left): tot[v * 6 + k]
// = sum over the bpk blocks of case k of partial[(k * bpk + j) * 2 + v], in a
// fixed order, the same in every lane.  One warp: the FP64 adds are few
// (bpk / 32 per lane and value, then the shuffle tree), which matters on
// B300's narrow FP64 pipe.
__device__ inline void sum_case_partials_warp(const double *partial, int bpk, double (&tot)[12]) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int m = 0; m < 12; ++m) tot[m] = 0.0;
    for (int j = lane; j < bpk; j += 32)
#pragma unroll
        for (int k = 0; k < 6; ++k) {
            tot[k] += __ldcg(partial + ((size_t)k * bpk + j) * 2 + 0);
            tot[6 + k] += __ldcg(partial + ((size_t)k * bpk + j) * 2 + 1);
        }
#pragma unroll
    for (int m = 0; m < 12; ++m)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) tot[m] += __shfl_xor_sync(0xffffffffu, tot[m], o);
}

// Block partials (d0, d1) -> partial[blockIdx.x * 2 + {0, 1}].  FP32
// accumulators are combined as double-floats (no FP64 shuffle tree).
template <typename T>
__device__ inline void store_block_pair(const DotAcc<T> &d0, const DotAcc<T> &d1, double *partial) {
    if constexpr (std::is_same<T, float>::value) {
        const float2 v[2] = {d0.get_df(), d1.get_df()};
        double s[2];
        block_sum_df<2>(v, s);
        if (threadIdx.x < 2) partial[(size_t)blockIdx.x * 2 + threadIdx.x] = s[threadIdx.x];
    } else {
        double v[2] = {d0.get(), d1.get()};
        block_reduce_store<2>(v, partial, blockIdx.x);
    }
}

// v[off + k] for a run-time k < 6 without local-memory indexing.
template <int NV>
__device__ __forceinline__ double pick6(const double (&v)[NV], int off, int k) {
    double r = 0.0;
#pragma unroll
    for (int i = 0; i < 6; ++i)
        if (i == k) r = v[off + i];
    return r;
}

// Per-CTA partial sums of p.q left by the stiffness apply (deferred mode):
// partial[(k * per_case + b) * 6 + k] for the per_case CTAs of load case k.
struct ApplyDot {
    const double *partial;  // [rows][6]: a CTA's sum of each load case (zero for cases it did not touch)
    int rows;
};

// (p.q)_k of all six load cases at once, warp 0 only (one pass over the
// partials, one shuffle tree), the same values in every lane, fixed order.
__device__ inline void case_pq_warp(const ApplyDot &ad, double (&pq)[6]) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int k = 0; k < 6; ++k) pq[k] = 0.0;
    for (int b = lane; b < ad.rows; b += 32)
#pragma unroll
        for (int k = 0; k < 6; ++k) pq[k] += __ldcg(ad.partial + (size_t)b * 6 + k);
#pragma unroll
    for (int k = 0; k < 6; ++k)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) pq[k] += __shfl_xor_sync(0xffffffffu, pq[k], o);
}

// One block: alpha_k = rz_k / (p.q)_k for the active load cases, from the
// stiffness apply's deferred per-CTA partials; a non-positive or non-finite
// p.q stops the case with a numeric error.
__global__ void pcg_alpha_kernel(PcgState *st, ApplyDot ad) {
    pdl_enter();
    if (st->nactive == 0 || threadIdx.x >= 32) return;
    double pq[6];
    case_pq_warp(ad, pq);
    // lane k of warp 0 handles load case k (the state loads run in parallel)
    if (threadIdx.x < 32) {
        const int k = threadIdx.x;
        int act = 0;
        if (k < 6) {
            act = st->active[k];
            if (act) {
                const double p = pick6(pq, 0, k);
                if (!(p > 0.0) || !isfinite(p)) {
                    st->numeric_err = kNumErrPq;
                    st->alpha[k] = 0.0;
                    act = 0;
                    st->active[k] = 0;
                } else {
                    st->alpha[k] = st->rz[k] / p;
                }
            }
        }
        const int na = __reduce_add_sync(0xffffffffu, act);
        if (k == 0) st->nactive = na;
    }
}

struct FineJacobi {
    const float *Dinv;  // [9][N] 3x3 block inverses (row-major per node)
    float omega;
    float *z;           // output (update) / in-out (jacobi_rz), 18 planes
};

// x += alpha p ; r -= alpha q  (active cases, alpha from pcg_alpha_kernel), rr = r.r
//   Jacobi mode (MG = false): rz = r . D^-1 r with the point-Jacobi diagonal
//   a.dinv; the last block sets beta and rz.
//   Multigrid mode: z = w D^-1 r (first pre-smoothing step); beta comes later
//   from vec_jacobi_rz.
// Last block: iteration count, convergence and budget tests, nactive.
template <typename T, int V, bool MG>
__global__ void __launch_bounds__(kVecThreads, kVecBlocksPerSM)
    vec_update_kernel(VecArgs<T> a, VecGeom g, FineJacobi fj) {
    pdl_enter();
    PcgState *st = a.st;
    if (st->nactive == 0) return;  // uniform: the solve has finished
    const int k = blockIdx.x / g.bpk, j = blockIdx.x - k * g.bpk;
    const bool act = st->active[k] != 0;
    DotAcc<T> drz, drr;
    if (act) {
        const T al = (T)st->alpha[k];
        const size_t N = a.N;
        T *__restrict__ x = a.x + (size_t)3 * k * N;
        T *__restrict__ r = a.r + (size_t)3 * k * N;
        const T *__restrict__ p = a.p + (size_t)3 * k * N;
        const T *__restrict__ q = a.q + (size_t)3 * k * N;
        for (size_t ci = (size_t)j * kVecThreads + threadIdx.x; ci < g.chunks; ci += (size_t)g.bpk * kVecThreads) {
            const size_t n0 = g.chunk(ci) * V;
            Chunk<T, V> rn[3];
#pragma unroll
            for (int i = 0; i < 3; ++i) {
                const size_t o = (size_t)i * N + n0;
                Chunk<T, V> xv = ldc<T, V>(x + o), pv = ldc<T, V>(p + o), rv = ldc<T, V>(r + o),
                            qv = ldc<T, V>(q + o);
#pragma unroll
                for (int e = 0; e < V; ++e) {
                    xv.v[e] += al * pv.v[e];
                    rv.v[e] -= al * qv.v[e];
                    drr.add(rv.v[e] * rv.v[e]);
                }
                stc<T, V>(x + o, xv);
                stc<T, V>(r + o, rv);
                rn[i] = rv;
            }
            if constexpr (MG) {
                float D[9][V];
#pragma unroll
                for (int m = 0; m < 9; ++m) {
                    const Chunk<float, V> dv = ldc<float, V>(fj.Dinv + (size_t)m * N + n0);
#pragma unroll
                    for (int e = 0; e < V; ++e) D[m][e] = dv.v[e];
                }
#pragma unroll
                for (int i = 0; i < 3; ++i) {
                    Chunk<float, V> zv;
#pragma unroll
                    for (int e = 0; e < V; ++e)
                        zv.v[e] = fj.omega * (D[3 * i][e] * (float)rn[0].v[e] + D[3 * i + 1][e] * (float)rn[1].v[e] +
                                              D[3 * i + 2][e] * (float)rn[2].v[e]);
                    stc<float, V>(fj.z + (size_t)(3 * k + i) * N + n0, zv);
                }
            } else {
                const Chunk<T, V> dv = ldc<T, V>(a.dinv + n0);
#pragma unroll
                for (int i = 0; i < 3; ++i)
#pragma unroll
                    for (int e = 0; e < V; ++e) drz.add(rn[i].v[e] * (dv.v[e] * rn[i].v[e]));
            }
        }
    }
    store_block_pair<T>(drz, drr, a.partial);
    if (!last_block_ticket(&st->ticket_update, gridDim.x) || threadIdx.x >= 32) return;
    double tot[12];
    sum_case_partials_warp(a.partial, g.bpk, tot);
    // lane kk of warp 0 handles load case kk (the state loads run in parallel)
    if (threadIdx.x < 32) {
        const int kk = threadIdx.x;
        int act = 0;
        if (kk < 6) {
            act = st->active[kk];
            if (act) {
                const int it = st->iters[kk] + 1;
                st->iters[kk] = it;
                const double rz = pick6(tot, 0, kk), rr = pick6(tot, 6, kk);
                st->rr[kk] = rr;
                if (!isfinite(rz) || !isfinite(rr)) {
                    st->numeric_err = kNumErrResid;
                    act = 0;
                } else if (rr <= st->tol2 * st->bnorm2[kk]) {
                    act = 0;
                } else if (it >= st->maxit) {
                    act = 0;
                } else if (!MG) {
                    st->beta[kk] = rz / st->rz[kk];
                    st->rz[kk] = rz;
                }
                if (!act) st->active[kk] = 0;
            }
        }
        const int na = __reduce_add_sync(0xffffffffu, act);
        if (kk == 0) st->nactive = na;
    }
}

// Multigrid mode, last post-smoothing step at the fine level and beta:
// z += w D^-1 (r - t) (active cases; t = K z from the preceding apply), then
// rz = r . z; last block: beta = rz / rz_prev, rz_prev = rz.
template <int V>
__global__ void __launch_bounds__(kVecThreads, kVecBlocksPerSM)
    vec_jacobi_rz_kernel(VecArgs<float> a, VecGeom g, FineJacobi fj, const float *__restrict__ t) {
    pdl_enter();
    PcgState *st = a.st;
    if (st->nactive == 0) return;
    const int k = blockIdx.x / g.bpk, j = blockIdx.x - k * g.bpk;
    const bool act = st->active[k] != 0;
    DotAcc<float> drz, dnone;
    if (act) {
        const size_t N = a.N;
        const float *__restrict__ r = a.r + (size_t)3 * k * N;
        const float *__restrict__ tk = t + (size_t)3 * k * N;
        float *__restrict__ z = fj.z + (size_t)3 * k * N;
        for (size_t ci = (size_t)j * kVecThreads + threadIdx.x; ci < g.chunks; ci += (size_t)g.bpk * kVecThreads) {
            const size_t n0 = g.chunk(ci) * V;
            Chunk<float, V> rv[3], dv[3], zv[3];
#pragma unroll
            for (int i = 0; i < 3; ++i) {
                const size_t o = (size_t)i * N + n0;
                rv[i] = ldc<float, V>(r + o);
                const Chunk<float, V> tv = ldc<float, V>(tk + o);
                zv[i] = ldc<float, V>(z + o);
#pragma unroll
                for (int e = 0; e < V; ++e) dv[i].v[e] = rv[i].v[e] - tv.v[e];
            }
            float D[9][V];
#pragma unroll
            for (int m = 0; m < 9; ++m) {
                const Chunk<float, V> d = ldc<float, V>(fj.Dinv + (size_t)m * N + n0);
#pragma unroll
                for (int e = 0; e < V; ++e) D[m][e] = d.v[e];
            }
#pragma unroll
            for (int i = 0; i < 3; ++i) {
#pragma unroll
                for (int e = 0; e < V; ++e) {
                    zv[i].v[e] += fj.omega * (D[3 * i][e] * dv[0].v[e] + D[3 * i + 1][e] * dv[1].v[e] +
                                              D[3 * i + 2][e] * dv[2].v[e]);
                    drz.add(rv[i].v[e] * zv[i].v[e]);
                }
                stc<float, V>(z + (size_t)i * N + n0, zv[i]);
            }
        }
    }
    store_block_pair<float>(drz, dnone, a.partial);
    if (!last_block_ticket(&st->ticket_aux, gridDim.x) || threadIdx.x >= 32) return;
    double tot[12];
    sum_case_partials_warp(a.partial, g.bpk, tot);
    if (threadIdx.x < 32) {
        const int kk = threadIdx.x;
        int act = 0;
        if (kk < 6) {
            act = st->active[kk];
            if (act) {
                const double rz = pick6(tot, 0, kk);
                if (!isfinite(rz) || !(rz > 0.0)) {
                    st->numeric_err = kNumErrRz;
                    act = 0;
                    st->active[kk] = 0;
                } else {
                    st->beta[kk] = rz / st->rz[kk];
                    st->rz[kk] = rz;
                }
            }
        }
        const int na = __reduce_add_sync(0xffffffffu, act);
        if (kk == 0) st->nactive = na;
    }
}

// p = z + beta p (multigrid) or p = D^-1 r + beta p (point Jacobi), active cases.
template <typename T, int V>
__global__ void __launch_bounds__(kVecThreads, kVecBlocksPerSM) vec_direction_kernel(VecArgs<T> a, VecGeom g) {
    pdl_enter();
    PcgState *st = a.st;
    if (st->nactive == 0) return;
    const int k = blockIdx.x / g.bpk, j = blockIdx.x - k * g.bpk;
    if (!st->active[k]) return;
    const T be = (T)st->beta[k];
    const size_t N = a.N;
    T *__restrict__ p = a.p + (size_t)3 * k * N;
    const T *__restrict__ r = a.r + (size_t)3 * k * N;
    const T *__restrict__ z = a.z ? a.z + (size_t)3 * k * N : nullptr;
    for (size_t ci = (size_t)j * kVecThreads + threadIdx.x; ci < g.chunks; ci += (size_t)g.bpk * kVecThreads) {
        const size_t n0 = g.chunk(ci) * V;
        Chunk<T, V> di;
        if (!z) di = ldc<T, V>(a.dinv + n0);
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            const size_t o = (size_t)i * N + n0;
            Chunk<T, V> pv = ldc<T, V>(p + o);
            if (z) {
                const Chunk<T, V> zv = ldc<T, V>(z + o);
#pragma unroll
                for (int e = 0; e < V; ++e) pv.v[e] = zv.v[e] + be * pv.v[e];
            } else {
                const Chunk<T, V> rv = ldc<T, V>(r + o);
#pragma unroll
                for (int e = 0; e < V; ++e) pv.v[e] = di.v[e] * rv.v[e] + be * pv.v[e];
            }
            stc<T, V>(p + o, pv);
        }
    }
}

}  // namespace shl
