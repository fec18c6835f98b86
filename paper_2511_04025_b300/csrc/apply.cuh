// apply.cuh -- matrix-free periodic stiffness apply q = K p for up to six
// load cases at once (Eq. inv-design cell problems; Sec. 4.2.2: stiffness of
// the finest level computed on the fly, all right-hand sides in one kernel,
// converged right-hand sides skipped).
//
// Tiling.  A CTA owns a TX x TY x TZ block of output nodes.  Its threads own
// (TX+1) x (TY+1) element columns (one halo column towards -x and -y) and
// march along z.  Per step the CTA stages one new node plane ((TX+2) x
// (TY+2) nodes, periodic wrap, SoA planes) in a two-slot shared ring, every
// element thread applies E_e Khat to its 8 nodes in the Walsh-Hadamard form
// (element.cuh), keeps the contributions to its own node column in
// registers, and passes the other three corners of each node plane to its
// +x / +y / +xy neighbours through a double-buffered shared exchange.  The
// +z half of every element's output is carried in registers to the next
// step, so no atomics are used and the result is deterministic.
//
// Modes: plain apply (q = K p), residual (q = -sum_e K_e (p_e + chi^k), i.e.
// f - K p), optional node-0 pin (q = 0 there: the pinned system), and fused
// partial dot products (p.q or q.q per load case) reduced by the last CTA.
#pragma once

#include "common.cuh"
#include "element.cuh"

namespace shl {

// Device-resident scalars of one batched 6-RHS PCG solve.
struct PcgState {
    double rz[6];  // (r, z) of the current iterate
    double alpha[6], beta[6];
    double rr[6];      // ||r||^2 (recurrence residual)
    double bnorm2[6];  // ||b||^2 of the system being solved
    double tol2;       // stop when rr <= tol2 * bnorm2
    int active[6];     // 1 while the load case iterates
    int iters[6];
    int maxit;
    int nactive;
    int numeric_err;
    unsigned ticket_apply, ticket_update, ticket_aux;
};

template <typename T>
struct ApplyArgs {
    int r, tz, nvec;
    size_t N;
    const T *p;
    T *q;
    const uint8_t *mask;  // E_e = mask ? E : E_void        (when rho == null)
    const double *rho;    // E_e = E_void + rho (E - E_void)
    T E, Evoid;
    int pin;               // zero the output at node 0
    int resid;             // output -sum_e E_e Khat (p_e + chi^k)
    int dot;               // 0: none, 1: sum p.q, 2: sum q.q (per load case)
    double *partial;       // [nblocks][6]
    unsigned *ticket;      // last-block counter
    double *dot_out;       // 6 sums (may be null)
    PcgState *st;          // PCG mode: active flags in, alpha = rz / pq out
    const int *active_in;  // per load-case flags when st == null (may be null)
    ElemOp<T> op;
};

template <int TX, int TY>
struct ApplyShape {
    static constexpr int EX = TX + 1, EY = TY + 1, NX = TX + 2, NY = TY + 2;
    static constexpr int NT = EX * EY;
    static constexpr int PL = NX * NY;
    static constexpr int THREADS = (NT + 31) / 32 * 32;
    template <typename T>
    static constexpr size_t smem() {
        return sizeof(T) * (2 * 18 * PL + 2 * 18 * NT);
    }
};

template <typename T, int TX, int TY>
__global__ void __launch_bounds__(ApplyShape<TX, TY>::THREADS) apply_kernel(const ApplyArgs<T> a) {
    using S = ApplyShape<TX, TY>;
    constexpr int EX = S::EX, NX = S::NX, NT = S::NT, PL = S::PL;
    extern __shared__ __align__(16) unsigned char smraw[];
    T *sp = reinterpret_cast<T *>(smraw);  // [2][18][PL] node planes
    T *sx = sp + 2 * 18 * PL;              // [2][18][NT] corner exchange

    if (a.st && a.st->nactive == 0) return;  // uniform: the solve has finished
    const int r = a.r;
    const size_t N = a.N;
    const int tid = threadIdx.x;
    const bool el = tid < NT;
    const int exl = el ? tid % EX : 0, eyl = el ? tid / EX : 0;
    const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY, z0 = blockIdx.z * a.tz;
    const int ex = wrapi(x0 - 1 + exl, r), ey = wrapi(y0 - 1 + eyl, r);
    const int nx = x0 - 1 + exl, ny = y0 - 1 + eyl;
    const bool out_col = el && exl >= 1 && eyl >= 1 && nx < r && ny < r;

    bool act[6];
#pragma unroll
    for (int k = 0; k < 6; ++k) {
        bool on = k < a.nvec;
        if (on && a.st) on = a.st->active[k] != 0;
        if (on && a.active_in) on = a.active_in[k] != 0;
        act[k] = on;
    }

    T acc_hi[6][3];
#pragma unroll
    for (int k = 0; k < 6; ++k)
#pragma unroll
        for (int i = 0; i < 3; ++i) acc_hi[k][i] = T(0);
    DotAcc<T> dacc[6];

    auto load_plane = [&](int z, int slot) {
        const int zw = wrapi(z, r);
        const int total = 3 * a.nvec * PL;
        for (int idx = tid; idx < total; idx += blockDim.x) {
            const int c = idx / PL, rem = idx - c * PL;
            if (!act[c / 3]) continue;
            const int ly = rem / NX, lx = rem - ly * NX;
            const int gx = wrapi(x0 - 1 + lx, r), gy = wrapi(y0 - 1 + ly, r);
            sp[(slot * 18 + c) * PL + rem] = a.p[(size_t)c * N + ((size_t)zw * r + gy) * r + gx];
        }
    };

    load_plane(z0 - 1, 0);
    for (int s = 0; s <= a.tz; ++s) {
        const int ez = z0 - 1 + s;
        if (ez >= r) break;  // uniform across the block
        load_plane(ez + 1, (s + 1) & 1);
        __syncthreads();
        const int slo = s & 1, shi = (s + 1) & 1;
        const bool out_plane = (s >= 1);
        T Ee = T(0);
        if (el) {
            const size_t e = ((size_t)wrapi(ez, r) * r + ey) * r + ex;
            Ee = a.rho ? (T)(a.Evoid + a.rho[e] * (a.E - a.Evoid)) : (a.mask[e] ? a.E : a.Evoid);
            if (a.resid) Ee = -Ee;
        }
        int kb = 0;
#pragma unroll
        for (int k = 0; k < 6; ++k) {
            if (!act[k]) continue;
            T w[3][8];
            T *xb = sx + kb * 18 * NT;
            if (el) {
                T v[3][8];
#pragma unroll
                for (int b = 0; b < 8; ++b) {
                    const int sl = (b & 4) ? shi : slo;
                    const int li = (eyl + ((b >> 1) & 1)) * NX + exl + (b & 1);
#pragma unroll
                    for (int i = 0; i < 3; ++i) v[i][b] = sp[(sl * 18 + 3 * k + i) * PL + li];
                }
#pragma unroll
                for (int i = 0; i < 3; ++i) wht8(v[i]);
                if (a.resid) {
#pragma unroll
                    for (int i = 0; i < 3; ++i)
#pragma unroll
                        for (int m = 0; m < 8; ++m) v[i][m] += a.op.chihat[k][i][m];
                }
                block_apply(a.op, v, w, Ee);
#pragma unroll
                for (int i = 0; i < 3; ++i) wht8(w[i]);
                // corners (1,0,0),(0,1,0),(1,1,0),(1,0,1),(0,1,1),(1,1,1) -> exchange
                constexpr int cor[6] = {1, 2, 3, 5, 6, 7};
#pragma unroll
                for (int j = 0; j < 6; ++j)
#pragma unroll
                    for (int i = 0; i < 3; ++i) xb[(j * 3 + i) * NT + tid] = w[i][cor[j]];
            }
            __syncthreads();
            if (out_col) {
                const int tl = tid - 1, td = tid - EX, tdl = tid - EX - 1;
#pragma unroll
                for (int i = 0; i < 3; ++i) {
                    const T lo = w[i][0] + xb[(0 * 3 + i) * NT + tl] + xb[(1 * 3 + i) * NT + td] +
                                 xb[(2 * 3 + i) * NT + tdl];
                    const T hi = w[i][4] + xb[(3 * 3 + i) * NT + tl] + xb[(4 * 3 + i) * NT + td] +
                                 xb[(5 * 3 + i) * NT + tdl];
                    if (out_plane) {
                        const size_t n = ((size_t)ez * r + ny) * r + nx;
                        T qv = acc_hi[k][i] + lo;
                        if (a.pin && n == 0) qv = T(0);
                        a.q[(size_t)(3 * k + i) * N + n] = qv;
                        if (a.dot == 1)
                            dacc[k].add(qv * sp[(slo * 18 + 3 * k + i) * PL + eyl * NX + exl]);
                        else if (a.dot == 2)
                            dacc[k].add(qv * qv);
                    }
                    acc_hi[k][i] = hi;
                }
            }
            kb ^= 1;
        }
        __syncthreads();
    }

    if (!a.dot) return;
    const unsigned nblocks = gridDim.x * gridDim.y * gridDim.z;
    const unsigned bid = (blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
    double dsum[6];
#pragma unroll
    for (int k = 0; k < 6; ++k) dsum[k] = dacc[k].get();
    block_reduce_store<6>(dsum, a.partial, bid);
    if (!last_block_ticket(a.ticket, nblocks)) return;
    __shared__ double tot[6];
    sum_partials_ordered<6>(a.partial, nblocks, tot);
    if (threadIdx.x == 0) {
        if (a.dot_out)
            for (int k = 0; k < 6; ++k) a.dot_out[k] = tot[k];
        if (a.st) {
            for (int k = 0; k < 6; ++k) {
                if (!act[k]) continue;
                const double pq = tot[k];
                if (!(pq > 0.0) || !isfinite(pq)) {
                    a.st->numeric_err = 1;
                    a.st->active[k] = 0;
                    a.st->alpha[k] = 0.0;
                } else {
                    a.st->alpha[k] = a.st->rz[k] / pq;
                }
            }
            int na = 0;
            for (int k = 0; k < 6; ++k) na += a.st->active[k];
            a.st->nactive = na;
        }
    }
}

// --------------------------------------------------------------------------
// Node-wise kernels
// --------------------------------------------------------------------------

__device__ inline double elem_modulus(const uint8_t *mask, const double *rho, size_t e, double E, double Ev) {
    return rho ? Ev + rho[e] * (E - Ev) : (mask[e] ? E : Ev);
}

// Jacobi: inverse diagonal, diag(K)_n = Khat_diag * sum of E_e over the 8
// elements incident to node n (the same for the three DOFs).
template <typename T>
__global__ void dinv_kernel(int r, const uint8_t *mask, const double *rho, double E, double Ev, double kdiag,
                            T *dinv) {
    const size_t N = (size_t)r * r * r;
    for (size_t n = blockIdx.x * (size_t)blockDim.x + threadIdx.x; n < N; n += (size_t)gridDim.x * blockDim.x) {
        const int ix = n % r, iy = (n / r) % r, iz = n / ((size_t)r * r);
        double s = 0.0;
        for (int b = 0; b < 8; ++b) {
            const size_t e = ((size_t)wrapi(iz - (b >> 2), r) * r + wrapi(iy - ((b >> 1) & 1), r)) * r +
                             wrapi(ix - (b & 1), r);
            s += elem_modulus(mask, rho, e, E, Ev);
        }
        dinv[n] = (T)(1.0 / (kdiag * s));
    }
}

// f^(k)_n = - sum over the 8 incident elements of E_e (Khat chi^k)_(corner of n)
__global__ void rhs_kernel(int r, const uint8_t *mask, const double *rho, double E, double Ev, ElemOp<double> op,
                           double *f) {
    const size_t N = (size_t)r * r * r;
    for (size_t n = blockIdx.x * (size_t)blockDim.x + threadIdx.x; n < N; n += (size_t)gridDim.x * blockDim.x) {
        const int ix = n % r, iy = (n / r) % r, iz = n / ((size_t)r * r);
        double acc[6][3] = {};
        for (int b = 0; b < 8; ++b) {
            const size_t e = ((size_t)wrapi(iz - (b >> 2), r) * r + wrapi(iy - ((b >> 1) & 1), r)) * r +
                             wrapi(ix - (b & 1), r);
            const double Ee = elem_modulus(mask, rho, e, E, Ev);
            for (int k = 0; k < 6; ++k)
                for (int i = 0; i < 3; ++i) acc[k][i] -= Ee * op.kchi[k][i][b];
        }
        for (int k = 0; k < 6; ++k)
            for (int i = 0; i < 3; ++i) f[(size_t)(3 * k + i) * N + n] = acc[k][i];
    }
}

}  // namespace shl
