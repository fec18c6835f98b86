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
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < N; e += (size_t)gridDim.x * blockDim.x) {
        const int ix = e % r, iy = (e / r) % r, iz = e / ((size_t)r * r);
        const double Ee = a.rho ? a.Evoid + a.rho[e] * (a.E - a.Evoid) : (a.mask[e] ? a.E : a.Evoid);
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

__global__ void __launch_bounds__(kChomThreads) chom_df_kernel(const ChomDfArgs a) {
    extern __shared__ dfloat wdf[];  // [6][24][blockDim] transformed total fields
    dfloat acc[21];
#pragma unroll
    for (int t = 0; t < 21; ++t) acc[t] = dfloat(0.0f, 0.0f);
    const int r = a.r;
    const size_t N = a.N;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < N; e += (size_t)gridDim.x * blockDim.x) {
        const int ix = e % r, iy = (e / r) % r, iz = e / ((size_t)r * r);
        const dfloat Ee = dfloat(a.rho ? a.Evoid + a.rho[e] * (a.E - a.Evoid) : (a.mask[e] ? a.E : a.Evoid));
        for (int k = 0; k < 6; ++k) {
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
                for (int m = 0; m < 8; ++m)
                    wdf[((k * 3 + i) * 8 + m) * blockDim.x + threadIdx.x] = w[i][m] + a.op.chihat[k][i][m];
        }
        int t = 0;
        for (int j = 0; j < 6; ++j) {
            dfloat wj[3][8], gj[3][8];
#pragma unroll
            for (int i = 0; i < 3; ++i)
#pragma unroll
                for (int m = 0; m < 8; ++m) wj[i][m] = wdf[((j * 3 + i) * 8 + m) * blockDim.x + threadIdx.x];
            block_apply(a.op, wj, gj, dfloat(1.0f, 0.0f));
            for (int i = 0; i <= j; ++i) {
                dfloat s = dfloat(0.0f, 0.0f);
#pragma unroll
                for (int c = 0; c < 3; ++c)
#pragma unroll
                    for (int m = 0; m < 8; ++m) s += wdf[((i * 3 + c) * 8 + m) * blockDim.x + threadIdx.x] * gj[c][m];
                acc[t] += Ee * s;
                ++t;
            }
        }
    }
    float2 v[21];
#pragma unroll
    for (int t = 0; t < 21; ++t) v[t] = make_float2(acc[t].hi, acc[t].lo);
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
