// field.cuh -- charge field, distance proxy, threshold selection and
// voxelisation (Sec. 3.1 Eq. charge-field; Sec. 4.1 Eq. beta).
//
// Separable form.  With cos(2 pi n (x - x_j)) = C_n(x) C_n(x_j) + S_n(x) S_n(x_j)
// on each axis, the truncated series becomes a tensor-product expansion
//     F(x, y, z) = sum_{a,b,c} A_abc phi_a(x) phi_b(y) phi_c(z)
// over the per-axis basis phi_0 = 1, phi_n = cos(2 pi n x), phi_{K+n} =
// sin(2 pi n x) (n = 1..K), with the design's coefficient tensor
//     A_abc = alpha_hkl w_hkl / (h^2+k^2+l^2) sum_j q_j phi_a(x_j) phi_b(y_j) phi_c(z_j)
// (h, k, l the frequencies of a, b, c).  A costs O(N_c (2K+1)^3) once per
// design; every voxel then costs 4 x (2K+1) FMAs for F and grad F after two
// per-plane / per-line contractions, independent of the number of charges
// (the paper's field time grows linearly in 2N, Table 1).  All in FP64.
#pragma once

#include "common.cuh"

namespace shl {

constexpr int kMaxK = 7;
constexpr int kMaxBasis = 2 * kMaxK + 1;
constexpr int kSelW = 64;       // gap search window around k0 (ranks)
constexpr int kSelCap = 4096;   // keys gathered around the window
constexpr int kSelBins = 2048;  // radix histogram bins (11-bit digits)

__host__ __device__ inline int basis_freq(int a, int K) { return a <= K ? a : a - K; }

__device__ inline double mode_weight(int h, int k, int l) {
    const int zeros = (h == 0) + (k == 0) + (l == 0);
    return zeros == 0 ? 1.0 : zeros == 1 ? 0.5 : zeros == 2 ? 0.25 : 0.0;
}

// phi_a(x) for all a (x in cell units).
__device__ inline void basis_eval(double x, int K, double *phi) {
    phi[0] = 1.0;
    for (int n = 1; n <= K; ++n) {
        double s, c;
        sincospi(2.0 * n * x, &s, &c);
        phi[n] = c;
        phi[K + n] = s;
    }
}

// d phi_a / dx from the basis values themselves.
__device__ inline double basis_deriv(const double *phi, int a, int K) {
    if (a == 0) return 0.0;
    if (a <= K) return -2.0 * M_PI * a * phi[K + a];
    return 2.0 * M_PI * (a - K) * phi[a - K];
}

// --------------------------------------------------------------------------
// Coefficient tensor A (one block of 512 threads per design).
// --------------------------------------------------------------------------
__global__ void field_coef_kernel(int n, int K, const double *__restrict__ pos, const double *__restrict__ q,
                                  const double *__restrict__ alpha, double *__restrict__ A) {
    const int nb = 2 * K + 1;
    const int ncoef = nb * nb * nb;
    constexpr int CH = 64;
    __shared__ double phis[CH][3][kMaxBasis];
    __shared__ double qs[CH];
    double acc[7];  // coefficients owned by this thread: idx = tid + s*blockDim
    for (int s = 0; s < 7; ++s) acc[s] = 0.0;
    for (int j0 = 0; j0 < n; j0 += CH) {
        const int m = min(CH, n - j0);
        __syncthreads();
        for (int t = threadIdx.x; t < m * 3; t += blockDim.x) {
            const int j = t / 3, d = t % 3;
            basis_eval(pos[3 * (j0 + j) + d], K, phis[j][d]);
        }
        for (int t = threadIdx.x; t < m; t += blockDim.x) qs[t] = q[j0 + t];
        __syncthreads();
        for (int s = 0; s < 7; ++s) {
            const int idx = threadIdx.x + s * blockDim.x;
            if (idx >= ncoef) break;
            const int a = idx / (nb * nb), b = (idx / nb) % nb, c = idx % nb;
            double v = acc[s];
            for (int j = 0; j < m; ++j) v += qs[j] * (phis[j][0][a] * phis[j][1][b] * phis[j][2][c]);
            acc[s] = v;
        }
    }
    for (int s = 0; s < 7; ++s) {
        const int idx = threadIdx.x + s * blockDim.x;
        if (idx >= ncoef) break;
        const int a = idx / (nb * nb), b = (idx / nb) % nb, c = idx % nb;
        const int h = basis_freq(a, K), k = basis_freq(b, K), l = basis_freq(c, K);
        double coef = 0.0;
        if (h + k + l > 0) {
            const double al = alpha ? alpha[(h * (K + 1) + k) * (K + 1) + l] : 1.0;
            coef = al * mode_weight(h, k, l) / (double)(h * h + k * k + l * l);
        }
        A[idx] = coef * acc[s];
    }
}

// --------------------------------------------------------------------------
// Field on the voxel centres.  Block = one z-plane slice of lines.
// Writes F / gradF (optional) and d = |F - c| / |grad F| (optional).
// --------------------------------------------------------------------------
struct FieldArgs {
    int r, K;
    int lines_per_block;
    double iso;
    const double *A;
    double *F;   // r^3 or null
    double *gF;  // 3 r^3 or null (x,y,z per voxel)
    double *d;   // r^3 or null
};

__global__ void field_grid_kernel(FieldArgs a) {
    extern __shared__ double sm[];
    const int K = a.K, nb = 2 * K + 1, r = a.r;
    const int iz = blockIdx.x;
    const int y0 = blockIdx.y * a.lines_per_block;
    const int y1 = min(r, y0 + a.lines_per_block);
    const int nl = y1 - y0;
    double *phi = sm;                   // [r][nb] basis at voxel centres
    double *Bz = phi + (size_t)r * nb;  // [nb][nb]  sum_c A phi_c(z)
    double *Bzd = Bz + nb * nb;         // [nb][nb]  sum_c A phi'_c(z)
    double *H = Bzd + nb * nb;          // [nl][3][nb]
    for (int i = threadIdx.x; i < r; i += blockDim.x) basis_eval((i + 0.5) / r, K, phi + (size_t)i * nb);
    __syncthreads();
    const double *phz = phi + (size_t)iz * nb;
    for (int t = threadIdx.x; t < nb * nb; t += blockDim.x) {
        double s = 0.0, sd = 0.0;
        for (int c = 0; c < nb; ++c) {
            const double Av = a.A[t * nb + c];
            s += Av * phz[c];
            sd += Av * basis_deriv(phz, c, K);
        }
        Bz[t] = s;
        Bzd[t] = sd;
    }
    __syncthreads();
    for (int t = threadIdx.x; t < nl * nb; t += blockDim.x) {
        const int li = t / nb, aa = t % nb;
        const double *phy = phi + (size_t)(y0 + li) * nb;
        double h0 = 0.0, hy = 0.0, hz = 0.0;
        for (int b = 0; b < nb; ++b) {
            const double B = Bz[aa * nb + b];
            h0 += B * phy[b];
            hy += B * basis_deriv(phy, b, K);
            hz += Bzd[aa * nb + b] * phy[b];
        }
        H[(li * 3 + 0) * nb + aa] = h0;
        H[(li * 3 + 1) * nb + aa] = hy;
        H[(li * 3 + 2) * nb + aa] = hz;
    }
    __syncthreads();
    for (int t = threadIdx.x; t < nl * r; t += blockDim.x) {
        const int li = t / r, ix = t % r;
        const double *phx = phi + (size_t)ix * nb;
        const double *h0 = H + (li * 3 + 0) * nb, *hy = H + (li * 3 + 1) * nb, *hz = H + (li * 3 + 2) * nb;
        double F = 0.0, gx = 0.0, gy = 0.0, gz = 0.0;
        for (int aa = 0; aa < nb; ++aa) {
            const double p = phx[aa];
            F += h0[aa] * p;
            gx += h0[aa] * basis_deriv(phx, aa, K);
            gy += hy[aa] * p;
            gz += hz[aa] * p;
        }
        const size_t e = ((size_t)iz * r + (y0 + li)) * r + ix;
        if (a.F) a.F[e] = F;
        if (a.gF) {
            a.gF[3 * e] = gx;
            a.gF[3 * e + 1] = gy;
            a.gF[3 * e + 2] = gz;
        }
        if (a.d) {
            const double g = sqrt(gx * gx + gy * gy + gz * gz);
            a.d[e] = g > 0.0 ? fabs(F - a.iso) / g : __longlong_as_double(0x7ff0000000000000ll);
        }
    }
}

inline size_t field_smem_bytes(int r, int K, int lines) {
    const int nb = 2 * K + 1;
    return sizeof(double) * ((size_t)r * nb + 2 * nb * nb + (size_t)lines * 3 * nb);
}

// --------------------------------------------------------------------------
// Threshold selection: radix select on the FP64 bit patterns of d >= 0
// (monotone as unsigned integers), two ranks at once, then a sorted window.
// --------------------------------------------------------------------------
struct SelectState {
    unsigned long long prefix[2];  // key bits fixed so far (per rank)
    unsigned long long rank[2];    // 1-based rank still to find within the prefix
    unsigned long long key[2];     // selected keys (after the last pass)
    unsigned hist[2][kSelBins];
    unsigned count_less;  // keys < key[0] (gather)
    unsigned count_buf;   // keys gathered in [key[0], key[1]]
    int status;           // 0 ok, 1 no gap in window, 2 buffer overflow
    double t, margin;
    long long k;
    unsigned long long buf[kSelCap];
};

// Histogram of the digit (bits [shift, shift+width)) of the keys whose higher
// bits match each rank's prefix.
__global__ void select_hist_kernel(const unsigned long long *__restrict__ keys, size_t n, SelectState *st, int shift,
                                   int width) {
    __shared__ unsigned h[2][kSelBins];
    for (int i = threadIdx.x; i < 2 * kSelBins; i += blockDim.x) (&h[0][0])[i] = 0;
    __syncthreads();
    const unsigned long long hi_mask = (shift + width >= 64) ? 0ull : (~0ull << (shift + width));
    const unsigned dmask = (1u << width) - 1u;
    const unsigned long long p0 = st->prefix[0], p1 = st->prefix[1];
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const unsigned long long k = keys[i];
        const unsigned dig = (unsigned)((k >> shift) & dmask);
        if ((k & hi_mask) == (p0 & hi_mask)) atomicAdd(&h[0][dig], 1u);
        if ((k & hi_mask) == (p1 & hi_mask)) atomicAdd(&h[1][dig], 1u);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < 2 * kSelBins; i += blockDim.x) {
        const unsigned v = (&h[0][0])[i];
        if (v) atomicAdd(&(&st->hist[0][0])[i], v);
    }
}

// Choose the digit whose bin holds the wanted rank, for both ranks at once.
// One block of kSelChooseThreads threads: thread t owns bins
// [t * PER, (t + 1) * PER); a block-wide exclusive prefix sum of the per-thread
// counts finds the one thread whose range the rank falls in, which then walks
// its PER bins.  Same result as scanning the bins in order (bin = first b
// with count(<= b) >= rank; the last bin and the full total when none is).
constexpr int kSelChooseThreads = 256;
__global__ void __launch_bounds__(kSelChooseThreads) select_choose_kernel(SelectState *st, int shift) {
    constexpr int T = kSelChooseThreads, PER = kSelBins / T, NW = T / 32;
    static_assert(kSelBins % T == 0, "bins per thread");
    __shared__ unsigned long long wsum[2][NW];
    __shared__ unsigned long long total[2];
    __shared__ int hit[2];
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    unsigned c[2][PER];
    unsigned long long own[2], incl[2];
#pragma unroll
    for (int w = 0; w < 2; ++w) {
        own[w] = 0;
#pragma unroll
        for (int b = 0; b < PER; ++b) {
            c[w][b] = st->hist[w][t * PER + b];
            own[w] += c[w][b];
        }
        incl[w] = own[w];
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned long long v = __shfl_up_sync(0xffffffffu, incl[w], o);
            if (lane >= o) incl[w] += v;
        }
        if (lane == 31) wsum[w][warp] = incl[w];
    }
    if (t < 2) hit[t] = 0;
    __syncthreads();
#pragma unroll
    for (int w = 0; w < 2; ++w) {
        unsigned long long before = incl[w] - own[w];  // exclusive prefix within the warp
        for (int k = 0; k < warp; ++k) before += wsum[w][k];
        if (t == T - 1) total[w] = before + own[w];
        const unsigned long long rank = st->rank[w];
        if ((before < rank || t == 0) && rank <= before + own[w]) {  // the rank falls in this thread's bins
            unsigned long long acc = before;
            int bin = t * PER + PER - 1;
#pragma unroll
            for (int b = 0; b < PER; ++b)
                if (acc + c[w][b] >= rank) {
                    bin = t * PER + b;
                    break;
                } else {
                    acc += c[w][b];
                }
            hit[w] = 1;
            st->rank[w] = rank - acc;
            st->prefix[w] |= ((unsigned long long)bin) << shift;
            if (shift == 0) st->key[w] = st->prefix[w];
        }
    }
    __syncthreads();
    if (t < 2 && !hit[t]) {  // the rank exceeds the total: the last bin
        st->rank[t] = st->rank[t] - total[t];
        st->prefix[t] |= ((unsigned long long)(kSelBins - 1)) << shift;
        if (shift == 0) st->key[t] = st->prefix[t];
    }
    for (int i = t; i < 2 * kSelBins; i += T) (&st->hist[0][0])[i] = 0;
}

__global__ void select_gather_kernel(const unsigned long long *__restrict__ keys, size_t n, SelectState *st) {
    const unsigned long long lo = st->key[0], hi = st->key[1];
    unsigned less = 0;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const unsigned long long k = keys[i];
        if (k < lo)
            ++less;
        else if (k <= hi) {
            const unsigned slot = atomicAdd(&st->count_buf, 1u);
            if (slot < kSelCap) st->buf[slot] = k;
        }
    }
    for (int o = 16; o > 0; o >>= 1) less += __shfl_xor_sync(0xffffffffu, less, o);
    if ((threadIdx.x & 31) == 0 && less) atomicAdd(&st->count_less, less);
}

// One block of 1024 threads: sort the gathered keys (bitonic) and search the
// resolvable gap nearest k0.
__global__ void select_finish_kernel(SelectState *st, long long n, long long k0) {
    __shared__ unsigned long long s[kSelCap];
    const unsigned m = min(st->count_buf, (unsigned)kSelCap);
    for (int i = threadIdx.x; i < kSelCap; i += blockDim.x) s[i] = (i < (int)m) ? st->buf[i] : ~0ull;
    __syncthreads();
    for (int size = 2; size <= kSelCap; size <<= 1)
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            for (int i = threadIdx.x; i < kSelCap; i += blockDim.x) {
                const int j = i ^ stride;
                if (j > i) {
                    const bool up = ((i & size) == 0);
                    const unsigned long long a = s[i], b = s[j];
                    if ((a > b) == up) {
                        s[i] = b;
                        s[j] = a;
                    }
                }
            }
            __syncthreads();
        }
    if (threadIdx.x == 0) {
        st->status = 1;
        if (st->count_buf > (unsigned)kSelCap) {
            st->status = 2;
            return;
        }
        const long long base = (long long)st->count_less + 1;  // rank of s[0]
        for (int j = 0; j <= kSelW && st->status == 1; ++j) {
            for (int side = 0; side < (j ? 2 : 1); ++side) {
                const long long k = side ? k0 + j : k0 - j;
                if (k < 1 || k > n - 1) continue;
                const long long i0 = k - base, i1 = k + 1 - base;
                if (i0 < 0 || i1 >= (long long)m) continue;
                const double lo = __longlong_as_double((long long)s[i0]);
                const double hi = __longlong_as_double((long long)s[i1]);
                if (isfinite(hi) && hi - lo > 1e-9 * hi) {
                    st->t = 0.5 * (lo + hi);
                    st->margin = 0.5 * (hi - lo);
                    st->k = k;
                    st->status = 0;
                    break;
                }
            }
        }
    }
}

// mask / smooth density from d and t (t read from the device state, or the
// explicit value if sel == null); counts solid and ambiguous voxels.
__global__ void voxel_mask_kernel(const double *__restrict__ d, size_t n, const SelectState *sel, double t_explicit,
                                  double kappa, uint8_t *mask, double *rho, unsigned long long *counts) {
    const double t = sel ? sel->t : t_explicit;
    unsigned long long solid = 0, amb = 0;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const double di = d[i];
        const bool s = di <= t;
        solid += s;
        amb += fabs(di - t) <= 1e-9 * t;
        if (mask) mask[i] = s ? 1 : 0;
        if (rho) rho[i] = 1.0 / (1.0 + exp(-kappa * (t - di)));
    }
    for (int o = 16; o > 0; o >>= 1) {
        solid += __shfl_xor_sync(0xffffffffu, solid, o);
        amb += __shfl_xor_sync(0xffffffffu, amb, o);
    }
    if ((threadIdx.x & 31) == 0) {
        if (solid) atomicAdd(&counts[0], solid);
        if (amb) atomicAdd(&counts[1], amb);
    }
}

}  // namespace shl
