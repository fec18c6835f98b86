// chom.cuh -- homogenised tensor C^H_ij = sum_e E_e (chi^i + u^i_e)^T Khat
// (chi^j + u^j_e), |Y| = 1 (Eq. inv-design), and the element sensitivities
// of the energy form used by the adjoint (Eq. chain).  FP64 throughout.
//
// Per element the six total fields w^k = chi^k + u^k_e are moved to the
// Walsh-Hadamard basis (w-hat = chi-hat^k + H u^k_e) and the 21 unique
// energies w-hat^i^T G w-hat^j are formed with the 3x3 block operator
// (w^T Khat w' = w-hat^T G w-hat' since H H = 8 I and G = H Khat H / 64).
#pragma once

#include "apply.cuh"

namespace shl {

constexpr int kChomThreads = 64;

struct ChomArgs {
    int r;
    size_t N;
    const double *u;  // 18 SoA planes
    const uint8_t *mask;
    const double *rho;
    double E, Evoid;
    double *partial;  // [nblocks][21]
    unsigned *ticket;
    double *C;        // 36 (written by the last block)
    const double *G;  // sensitivity mode: dE/dC (36) -> g_e; null for C^H
    double *g;        // r^3 element sensitivities (sensitivity mode)
    ElemOp<double> op;
};

__device__ inline void load_element_field(const ChomArgs &a, int ix, int iy, int iz, int k, double (&w)[3][8]) {
    const int r = a.r;
#pragma unroll
    for (int b = 0; b < 8; ++b) {
        const size_t n = ((size_t)wrapi(iz + (b >> 2), r) * r + wrapi(iy + ((b >> 1) & 1), r)) * r +
                         wrapi(ix + (b & 1), r);
#pragma unroll
        for (int i = 0; i < 3; ++i) w[i][b] = a.u[(size_t)(3 * k + i) * a.N + n];
    }
#pragma unroll
    for (int i = 0; i < 3; ++i) wht8(w[i]);
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int m = 0; m < 8; ++m) w[i][m] += a.op.chihat[k][i][m];
}

__global__ void __launch_bounds__(kChomThreads) chom_kernel(const ChomArgs a) {
    extern __shared__ double wsm[];  // [6][24][blockDim] transformed total fields
    double acc[21];
#pragma unroll
    for (int t = 0; t < 21; ++t) acc[t] = 0.0;
    const int r = a.r;
    const size_t N = a.N;
    // warps step through 32 consecutive elements at a time (the element of
    // each thread is the one of a plain grid-stride loop)
    const unsigned lane = threadIdx.x & 31u;
    for (size_t e0 = blockIdx.x * (size_t)blockDim.x + (threadIdx.x - lane); e0 < N;
         e0 += (size_t)gridDim.x * blockDim.x) {
        const size_t e = e0 + lane;
        const bool in = e < N;
        const double Ee = !in ? 0.0 : (a.rho ? a.Evoid + a.rho[e] * (a.E - a.Evoid) : (a.mask[e] ? a.E : a.Evoid));
        // culled elements (E_e = 0, the active set) add exact zeros to every
        // energy sum: a warp of them skips the work (the sensitivity mode
        // still needs every g_e)
        if (__all_sync(0xffffffffu, Ee == 0.0 && !a.g)) continue;
        if (!in) continue;
        const int ix = e % r, iy = (e / r) % r, iz = e / ((size_t)r * r);
        for (int k = 0; k < 6; ++k) {
            double w[3][8];
            load_element_field(a, ix, iy, iz, k, w);
#pragma unroll
            for (int i = 0; i < 3; ++i)
#pragma unroll
                for (int m = 0; m < 8; ++m) wsm[((k * 3 + i) * 8 + m) * blockDim.x + threadIdx.x] = w[i][m];
        }
        double gsum = 0.0;
        int t = 0;
        for (int j = 0; j < 6; ++j) {
            double wj[3][8], gj[3][8];
#pragma unroll
            for (int i = 0; i < 3; ++i)
#pragma unroll
                for (int m = 0; m < 8; ++m) wj[i][m] = wsm[((j * 3 + i) * 8 + m) * blockDim.x + threadIdx.x];
            block_apply(a.op, wj, gj, 1.0);
            for (int i = 0; i <= j; ++i) {
                double s = 0.0;
#pragma unroll
                for (int c = 0; c < 3; ++c)
#pragma unroll
                    for (int m = 0; m < 8; ++m) s += wsm[((i * 3 + c) * 8 + m) * blockDim.x + threadIdx.x] * gj[c][m];
                if (a.g) {
                    const double gw = (i == j) ? a.G[6 * i + j] : a.G[6 * i + j] + a.G[6 * j + i];
                    gsum += gw * s;
                } else {
                    acc[t] += Ee * s;
                }
                ++t;
            }
        }
        if (a.g) a.g[e] = (a.E - a.Evoid) * gsum;
    }
    if (a.g) return;
    const unsigned nb = gridDim.x;
    block_reduce_store<21>(acc, a.partial, blockIdx.x);
    if (!last_block_ticket(a.ticket, nb)) return;
    __shared__ double tot[21];
    sum_partials_ordered<21>(a.partial, nb, tot);
    if (threadIdx.x == 0) {
        int t = 0;
        for (int j = 0; j < 6; ++j)
            for (int i = 0; i <= j; ++i, ++t) {
                a.C[6 * i + j] = tot[t];
                a.C[6 * j + i] = tot[t];
            }
    }
}

// C^H in double-float arithmetic, for the FP32 + refinement solver: the same
// element energies as chom_kernel, from u already converted to dfloat (FP32
// pairs, ~48 significant bits, far beyond that mode's tolerance), so the
// per-element work runs on the FP32 pipes instead of B300's narrow FP64 pipe.
//
// A CTA takes 32 consecutive elements with one thread per (element, load
// case): warp k moves load case k's total fields to the transformed basis
// (shared memory), then applies the element blocks to its own field and
// forms its energies with the load cases i <= k.  The per-thread state is
// one load case instead of six, so several CTAs share an SM.  Groups of 32
// elements that are all culled (E_e = 0, the active set) are skipped: their
// energies are exact zeros.
struct ChomDfArgs {
    int r;
    size_t N;
    const dfloat *u;  // 18 SoA planes
    const uint8_t *mask;
    const double *rho;
    double E, Evoid;
    double *partial;  // [nblocks][21]
    unsigned *ticket;
    double *C;        // 36 (written by the last block)
    ElemOp<dfloat> op;
};

constexpr int kChomDfElems = 32;                 // elements per CTA step (one per lane)
constexpr int kChomDfThreads = 6 * kChomDfElems;  // warp k = load case k

__global__ void __launch_bounds__(kChomDfThreads) chom_df_kernel(const ChomDfArgs a) {
    __shared__ dfloat wsm[6][24][kChomDfElems];  // transformed total fields [case][component * 8 + mode][element]
    const int r = a.r;
    const size_t N = a.N;
    const int lane = threadIdx.x & 31, k = threadIdx.x >> 5;
    dfloat acc[6];  // energies (i, k) for i <= k
#pragma unroll
    for (int i = 0; i < 6; ++i) acc[i] = dfloat(0.0f, 0.0f);
    for (size_t e0 = (size_t)blockIdx.x * kChomDfElems; e0 < N; e0 += (size_t)gridDim.x * kChomDfElems) {
        const size_t e = e0 + lane;
        const bool in = e < N;
        const double Ed = !in ? 0.0 : (a.rho ? a.Evoid + a.rho[e] * (a.E - a.Evoid) : (a.mask[e] ? a.E : a.Evoid));
        if (!__syncthreads_or(Ed != 0.0)) continue;  // all 32 elements culled (uniform)
        if (in) {
            const int ix = e % r, iy = (e / r) % r, iz = e / ((size_t)r * r);
            dfloat w[3][8];
#pragma unroll
            for (int b = 0; b < 8; ++b) {
                const size_t n = ((size_t)wrapi(iz + (b >> 2), r) * r + wrapi(iy + ((b >> 1) & 1), r)) * r +
                                 wrapi(ix + (b & 1), r);
#pragma unroll
                for (int i = 0; i < 3; ++i) w[i][b] = a.u[(size_t)(3 * k + i) * N + n];
            }
#pragma unroll
            for (int i = 0; i < 3; ++i) wht8(w[i]);
#pragma unroll
            for (int i = 0; i < 3; ++i)
#pragma unroll
                for (int m = 0; m < 8; ++m) wsm[k][i * 8 + m][lane] = w[i][m] + a.op.chihat[k][i][m];
        }
        __syncthreads();
        if (in) {
            dfloat wk[3][8], gk[3][8];
#pragma unroll
            for (int i = 0; i < 3; ++i)
#pragma unroll
                for (int m = 0; m < 8; ++m) wk[i][m] = wsm[k][i * 8 + m][lane];
            block_apply(a.op, wk, gk, dfloat(1.0f, 0.0f));
            const dfloat Ee = dfloat(Ed);
#pragma unroll
            for (int i = 0; i < 6; ++i) {
                if (i > k) break;  // uniform per warp
                dfloat s = dfloat(0.0f, 0.0f);
#pragma unroll
                for (int c = 0; c < 3; ++c)
#pragma unroll
                    for (int m = 0; m < 8; ++m) s += wsm[i][c * 8 + m][lane] * gk[c][m];
                acc[i] += Ee * s;
            }
        }
        __syncthreads();  // wsm is refilled by the next step
    }
    // energy (i, j), i <= j, is entry t = j (j + 1) / 2 + i of the 21
    float2 v[21];
#pragma unroll
    for (int t = 0; t < 21; ++t) v[t] = make_float2(0.f, 0.f);
#pragma unroll
    for (int j = 0; j < 6; ++j)
#pragma unroll
        for (int i = 0; i <= j; ++i)
            if (j == k) v[j * (j + 1) / 2 + i] = make_float2(acc[i].hi, acc[i].lo);
    double sum[21];
    block_sum_df<21>(v, sum);
#pragma unroll
    for (int t = 0; t < 21; ++t)
        if (threadIdx.x == (unsigned)t) a.partial[(size_t)blockIdx.x * 21 + t] = sum[t];
    const unsigned nb = gridDim.x;
    if (!last_block_ticket(a.ticket, nb)) return;
    __shared__ double tot[21];
    sum_partials_ordered<21>(a.partial, nb, tot);
    if (threadIdx.x == 0) {
        int t = 0;
        for (int j = 0; j < 6; ++j)
            for (int i = 0; i <= j; ++i, ++t) {
                a.C[6 * i + j] = tot[t];
                a.C[6 * j + i] = tot[t];
            }
    }
}

}  // namespace shl
