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
// step, so no atomics are used and the result is deterministic.  A warp
// whose elements of a plane are all culled (E_e = 0: the active set of
// Sec. 4.2.1) skips the element operator for that plane.
//
// Modes: plain apply (q = K p), residual (q = -sum_e K_e (p_e + chi^k), i.e.
// f - K p), optional node-0 pin (q = 0 there: the pinned system), and fused
// partial dot products (p.q or q.q per load case) reduced by the last CTA.
#pragma once

#include "common.cuh"
#include "element.cuh"

namespace shl {

// Device-resident scalars of one batched 6-RHS PCG solve.
// Why a PCG case stopped with a numeric error (PcgState::numeric_err).
constexpr int kNumErrPq = 1;       // p.q not positive or not finite (operator or direction)
constexpr int kNumErrRz = 2;       // r.z not positive or not finite (preconditioner not SPD)
constexpr int kNumErrResid = 3;    // recurrence r.z or r.r not finite
constexpr int kNumErrInit = 4;     // initial residual not finite
constexpr int kNumErrRestart = 5;  // true residual at a reliable update not finite

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
    int numeric_err;  // 0, or the kNumErr* reason the last case stopped for
    unsigned ticket_apply, ticket_update, ticket_aux;
};

template <typename T>
struct ApplyArgs {
    int r, zc, nvec;  // zc: z chunks of the grid (near-equal heights)
    size_t N;
    const T *p;
    T *q;
    const uint8_t *mask;  // E_e = mask ? E : E_void        (when rho == null)
    const double *rho;    // E_e = E_void + rho (E - E_void)
    T E, Evoid;
    int pin;               // zero the output at node 0
    int resid;             // output -sum_e E_e Khat (p_e + chi^k)
    int dot;               // 0: none, 1: sum p.q, 2: sum q.q (per load case)
    int defer;             // with dot: only write the per-CTA partials (no grid reduction here)
    double *partial;       // [nblocks][6]
    unsigned *ticket;      // last-block counter
    double *dot_out;       // 6 sums (may be null)
    PcgState *st;          // PCG mode: active flags in, alpha = rz / pq out
    const int *active_in;  // six per load-case flags when st == null (may be null)
    int case_mask;         // bit k: load case k is computed (others: output and dot left untouched)
    int vec_ok;            // p is 16-byte aligned and r is a multiple of 16 / sizeof(T)
    unsigned *err;         // device error bits (apply_rows.cuh), or null
    ElemOp<T> op;
};

// Grid reduction of the fused dot products, run by thread 0 of the last CTA
// with the six case totals: dot_out and, in PCG mode, alpha = rz / pq (a
// non-positive or non-finite p.q stops that case with a numeric error).
template <typename T>
__device__ inline void apply_dot_finish(const ApplyArgs<T> &a, const double (&tot)[6]) {
    if (a.dot_out)
        for (int kk = 0; kk < 6; ++kk)
            if ((a.case_mask >> kk) & 1) a.dot_out[kk] = tot[kk];
    if (a.st) {
        for (int kk = 0; kk < 6; ++kk) {
            if (!a.st->active[kk]) continue;
            const double pq = tot[kk];
            if (!(pq > 0.0) || !isfinite(pq)) {
                a.st->numeric_err = kNumErrPq;
                a.st->active[kk] = 0;
                a.st->alpha[kk] = 0.0;
            } else {
                a.st->alpha[kk] = a.st->rz[kk] / pq;
            }
        }
        int na = 0;
        for (int kk = 0; kk < 6; ++kk) na += a.st->active[kk];
        a.st->nactive = na;
    }
}

// ---------------------------------------------------------------------------
// Asynchronous global -> shared copies (cp.async; completion by group)
// ---------------------------------------------------------------------------
__device__ __forceinline__ void cp_async16(void *smem, const void *gmem) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem));
}
template <int B>
__device__ __forceinline__ void cp_async_small(void *smem, const void *gmem) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], %2;\n" ::"r"(s), "l"(gmem), "n"(B));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

template <typename T, int TX, int TY>
struct ApplyShape {
    static constexpr int EX = TX + 1, EY = TY + 1;  // element columns (one halo column towards -x, -y)
    static constexpr int NT = EX * EY;
    static constexpr int THREADS = (NT + 31) / 32 * 32;
    static constexpr int VEC = 16 / sizeof(T);      // elements per 16-byte chunk
    static constexpr int OFF = VEC - 1;             // shared position of node column lx = 0
    static constexpr int PITCH = TX + 2 * VEC;      // row pitch: interior lx = 1.. starts 16-byte aligned
    static constexpr int NY = TY + 2;
    static constexpr int PLANE = 3 * NY * PITCH;    // one node plane, three components
    static constexpr size_t smem() { return sizeof(T) * (2 * PLANE + 2 * 9 * NT); }
};

__host__ __device__ inline int wrap_near(int v, int r) { return v < 0 ? v + r : (v >= r ? v - r : v); }

// One CTA = one load case k (blockIdx.z) x a TX x TY column tile (blockIdx.x)
// x tz node planes (blockIdx.y).  Per z step: wait for the prefetched node
// plane, start the copy of the next one (cp.async, 16-byte chunks for the
// tile interior, wrapped scalars for the halo), transform the element's top
// face (x, y butterflies), combine with the bottom face kept from the
// previous step (z butterfly), apply the 3x3 blocks, split the result into
// bottom/top faces, add the bottom face to the carried top face of the
// element below, untransform and hand the three foreign corners of the node
// plane to the +x / +y / +xy neighbours.
// SMOOTH selects the density at compile time (a.rho, else a.mask): the
// smoothed modulus is formed in FP64 from rho, and a run-time branch lets the
// compiler issue those FP64 instructions, predicated off, on every z step of
// the binary-mask path too (B300's FP64 pipe is narrow).
template <typename T, int TX, int TY, bool RESID, bool SMOOTH>
__global__ void __launch_bounds__(ApplyShape<T, TX, TY>::THREADS, sizeof(T) == 4 ? 2 : 1)
    apply_kernel(const ApplyArgs<T> a) {
    pdl_enter();
    using S = ApplyShape<T, TX, TY>;
    constexpr int EX = S::EX, NT = S::NT, PITCH = S::PITCH, NY = S::NY, PLANE = S::PLANE, OFF = S::OFF,
                  VEC = S::VEC;
    extern __shared__ __align__(16) unsigned char smraw[];
    T *sp = reinterpret_cast<T *>(smraw);  // [2][3][NY][PITCH] node planes
    T *sx = sp + 2 * PLANE;                // [2][9][NT] corner exchange

    if (a.st && a.st->nactive == 0) return;  // uniform: the solve has finished
    const int r = a.r;
    const size_t N = a.N;
    const int k = blockIdx.z;
    bool act = k < a.nvec;
    if (act && a.st) act = a.st->active[k] != 0;
    if (act && a.active_in) act = a.active_in[k] != 0;
    act = act && ((a.case_mask >> k) & 1);
    DotAcc<T> dacc;

    if (act) {
        const int tid = threadIdx.x;
        const bool el = tid < NT;
        const int exl = el ? tid % EX : 0, eyl = el ? tid / EX : 0;
        const int tiles_x = (r + TX - 1) / TX;
        const int x0 = (blockIdx.x % tiles_x) * TX, y0 = (blockIdx.x / tiles_x) * TY;
        const int z0 = (int)(blockIdx.y * r) / a.zc, tz = (int)((blockIdx.y + 1) * r) / a.zc - z0;
        const int ex = wrapi(x0 - 1 + exl, r), ey = wrapi(y0 - 1 + eyl, r);
        const int nx = x0 - 1 + exl, ny = y0 - 1 + eyl;
        const bool out_col = el && exl >= 1 && eyl >= 1 && nx < r && ny < r;
        const bool vec_ok = a.vec_ok && (x0 + TX <= r);
        const bool zero_in = (a.p == nullptr);  // residual of x = 0 (the loads f)
        const T *pk = zero_in ? nullptr : a.p + (size_t)(3 * k) * N;
        const size_t rr = (size_t)r * r;

        // Copy descriptors of this thread's share of a node plane, computed once
        // for the 16-byte path: (component, row, chunk) -> shared offset and
        // global offset within a z-plane (interior chunks of 16 bytes, wrapped
        // scalars for the halo).  Ragged tiles and grids that are not a multiple
        // of the chunk take the scalar path, indexed on the fly.
        constexpr int NCH = TX / VEC + 2;
        constexpr int NITEM_V = 3 * NY * NCH;
        constexpr int MAXIT = (NITEM_V + S::THREADS - 1) / S::THREADS;
        int dst_off[MAXIT];
        size_t src_off[MAXIT];
        int kind[MAXIT];  // 0 none, 1 scalar, 2 sixteen bytes
#pragma unroll
        for (int u = 0; u < MAXIT; ++u) {
            const int idx = tid + u * S::THREADS;
            kind[u] = 0;
            dst_off[u] = 0;
            src_off[u] = 0;
            if (!vec_ok || zero_in || idx >= NITEM_V) continue;
            const int c = idx / (NY * NCH), rem = idx - c * (NY * NCH);
            const int ly = rem / NCH, ch = rem - ly * NCH;
            const size_t row = (size_t)c * N + (size_t)wrapi(y0 - 1 + ly, r) * r;
            const int drow = (c * NY + ly) * PITCH + OFF;
            if (ch == 0) {
                kind[u] = 1;
                dst_off[u] = drow;
                src_off[u] = row + wrapi(x0 - 1, r);
            } else if (ch == NCH - 1) {
                kind[u] = 1;
                dst_off[u] = drow + TX + 1;
                src_off[u] = row + wrapi(x0 + TX, r);
            } else {
                kind[u] = 2;
                dst_off[u] = drow + 1 + (ch - 1) * VEC;
                src_off[u] = row + x0 + (ch - 1) * VEC;
            }
        }
        auto load_plane = [&](int z, int slot) {
            if (zero_in) return;
            const int zw = z < 0 ? z + r : (z >= r ? z - r : z);
            const T *base = pk + (size_t)zw * rr;
            T *dst = sp + slot * PLANE;
            if (vec_ok) {
#pragma unroll
                for (int u = 0; u < MAXIT; ++u) {
                    if (kind[u] == 2)
                        cp_async16(dst + dst_off[u], base + src_off[u]);
                    else if (kind[u] == 1)
                        cp_async_small<sizeof(T)>(dst + dst_off[u], base + src_off[u]);
                }
            } else {
                constexpr int NXX = TX + 2;
                for (int idx = tid; idx < 3 * NY * NXX; idx += S::THREADS) {
                    const int c = idx / (NY * NXX), rem = idx - c * (NY * NXX);
                    const int ly = rem / NXX, lx = rem - ly * NXX;
                    const T *src = base + (size_t)c * N + (size_t)wrapi(y0 - 1 + ly, r) * r + wrapi(x0 - 1 + lx, r);
                    cp_async_small<sizeof(T)>(dst + (c * NY + ly) * PITCH + OFF + lx, src);
                }
            }
            cp_async_commit();
        };

        // top face of node plane in `slot`: x, y butterflies; also the raw own-node value
        auto face = [&](int slot, T (&ft)[3][4], T (&own)[3]) {
            const T *s = sp + slot * PLANE;
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                if (zero_in) {
                    own[c] = ft[c][0] = ft[c][1] = ft[c][2] = ft[c][3] = T(0);
                    continue;
                }
                const T *row0 = s + (c * NY + eyl) * PITCH + OFF + exl;
                const T *row1 = row0 + PITCH;
                const T a00 = row0[0], a10 = row0[1], a01 = row1[0], a11 = row1[1];
                own[c] = a00;
                const T s0 = a00 + a10, d0 = a00 - a10, s1 = a01 + a11, d1 = a01 - a11;
                ft[c][0] = s0 + s1;
                ft[c][1] = d0 + d1;
                ft[c][2] = s0 - s1;
                ft[c][3] = d0 - d1;
            }
        };

        // Residual mode: H chi^k of the element-local test displacement.  chi^k
        // is linear (chi_i = sum_d eps_id X_d, X on [0,h]^3), so only the
        // constant mode (4 h sum_d eps_id) and the three linear modes m = 2^d
        // (-4 h eps_id) are non-zero.
        T ch0[3], chd[3][3];
        if (RESID) {
            const T h4 = T(4.0 / (double)r);
#pragma unroll
            for (int i = 0; i < 3; ++i) {
                T sum = T(0);
#pragma unroll
                for (int d = 0; d < 3; ++d) {
                    const bool diag = (k < 3) && (i == k) && (d == k);
                    const bool shear = (k >= 3) && (i != d) && (i != k - 3) && (d != k - 3);
                    const T eps = diag ? T(1) : (shear ? T(0.5) : T(0));
                    chd[i][d] = -h4 * eps;
                    sum += eps;
                }
                ch0[i] = h4 * sum;
            }
        }

        const size_t exy = (size_t)ey * r + ex;
        auto modulus = [&](int ez) -> T {
            if (!el) return T(0);
            const size_t e = (size_t)(ez < 0 ? ez + r : (ez >= r ? ez - r : ez)) * rr + exy;
            T Ee;
            if constexpr (SMOOTH)
                Ee = T((double)a.Evoid + a.rho[e] * ((double)a.E - (double)a.Evoid));
            else
                Ee = a.mask[e] ? a.E : a.Evoid;
            return RESID ? -Ee : Ee;
        };

        T ftb[3][4], carry[3][4], own_b[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            own_b[c] = T(0);
#pragma unroll
            for (int j = 0; j < 4; ++j) carry[c][j] = T(0);
        }
        load_plane(z0 - 1, 0);
        load_plane(z0, 1);
        cp_async_wait_all();
        __syncthreads();
        if (el) face(0, ftb, own_b);
        T Ee = modulus(z0 - 1);

        for (int s = 0; s <= tz; ++s) {
            const int ez = z0 - 1 + s;  // element plane; node planes ez (bottom), ez + 1 (top)
            if (ez >= r) break;          // uniform
            // node plane ez + 1 has landed, and every thread is done reading
            // the slot the next copy overwrites (at s = 0: the bottom face)
            if (s > 0) cp_async_wait_all();
            __syncthreads();
            const bool more = (s < tz) && (ez + 1 < r);
            if (more) load_plane(ez + 2, s & 1);  // slot of node plane ez, already in registers
            const T Ee_next = more ? modulus(ez + 1) : T(0);
            T own_t[3];
            T ftt[3][4];
            T w[3][4];  // node-plane ez corner values (x, y butterflies undone)
            // A warp whose elements of this plane are all culled (E_e = 0, the
            // active set) adds exact zeros: it skips the element operator and
            // only hands on the top faces carried from the plane below.
            const bool void_warp = __all_sync(0xffffffffu, !el || zero_modulus(Ee));
            if (el) {
                face((s + 1) & 1, ftt, own_t);
                T F[3][4];
                if (void_warp) {
#pragma unroll
                    for (int c = 0; c < 3; ++c)
#pragma unroll
                        for (int j = 0; j < 4; ++j) {
                            F[c][j] = carry[c][j];
                            carry[c][j] = T(0);
                        }
                } else {
                    T u[3][8], y[3][8];
#pragma unroll
                    for (int c = 0; c < 3; ++c)
#pragma unroll
                        for (int j = 0; j < 4; ++j) {
                            u[c][j] = ftb[c][j] + ftt[c][j];
                            u[c][j + 4] = ftb[c][j] - ftt[c][j];
                        }
                    if (RESID) {
#pragma unroll
                        for (int c = 0; c < 3; ++c) {
                            u[c][0] += ch0[c];
                            u[c][1] += chd[c][0];
                            u[c][2] += chd[c][1];
                            u[c][4] += chd[c][2];
                        }
                    }
                    block_apply(a.op, u, y, Ee);
#pragma unroll
                    for (int c = 0; c < 3; ++c)
#pragma unroll
                        for (int j = 0; j < 4; ++j) {
                            F[c][j] = carry[c][j] + (y[c][j] + y[c][j + 4]);
                            carry[c][j] = y[c][j] - y[c][j + 4];
                        }
                }
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    const T t0 = F[c][0] + F[c][1], t1 = F[c][0] - F[c][1], t2 = F[c][2] + F[c][3],
                            t3 = F[c][2] - F[c][3];
                    w[c][0] = t0 + t2;
                    w[c][1] = t1 + t3;
                    w[c][2] = t0 - t2;
                    w[c][3] = t1 - t3;
                    ftb[c][0] = ftt[c][0];
                    ftb[c][1] = ftt[c][1];
                    ftb[c][2] = ftt[c][2];
                    ftb[c][3] = ftt[c][3];
                }
            }
            if (s > 0) {
                T *xb = sx + (s & 1) * 9 * NT;
                if (el) {
#pragma unroll
                    for (int j = 0; j < 3; ++j)
#pragma unroll
                        for (int c = 0; c < 3; ++c) xb[(j * 3 + c) * NT + tid] = w[c][j + 1];
                }
                __syncthreads();
                if (out_col) {
                    const int tl = tid - 1, td = tid - EX, tdl = tid - EX - 1;
                    const size_t n = ((size_t)ez * r + ny) * r + nx;
#pragma unroll
                    for (int c = 0; c < 3; ++c) {
                        T qv = w[c][0] + xb[(0 * 3 + c) * NT + tl] + xb[(1 * 3 + c) * NT + td] +
                               xb[(2 * 3 + c) * NT + tdl];
                        if (a.pin && n == 0) qv = T(0);
                        a.q[(size_t)(3 * k + c) * N + n] = qv;
                        if (a.dot == 1)
                            dacc.add(qv * own_b[c]);
                        else if (a.dot == 2)
                            dacc.add(qv * qv);
                    }
                }
            }
#pragma unroll
            for (int c = 0; c < 3; ++c) own_b[c] = own_t[c];
            Ee = Ee_next;
        }
        cp_async_wait_all();
    }

    if (!a.dot) return;
    const unsigned nblocks = gridDim.x * gridDim.y * gridDim.z;
    const unsigned bid = (blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
    // the CTA's row: its own case's sum in column k, zeros elsewhere
    if constexpr (std::is_same<T, float>::value) {
        const float2 v[1] = {dacc.get_df()};
        double sum[1];
        block_sum_df<1>(v, sum);
        if (threadIdx.x < 6) a.partial[(size_t)bid * 6 + threadIdx.x] = threadIdx.x == (unsigned)k ? sum[0] : 0.0;
    } else {
        double dcase[6];
        const double mine = dacc.get();
#pragma unroll
        for (int kk = 0; kk < 6; ++kk) dcase[kk] = (kk == k) ? mine : 0.0;
        block_reduce_store<6>(dcase, a.partial, bid);
    }
    if (a.defer) return;  // the consumer reduces the per-CTA partials itself
    if (!last_block_ticket(a.ticket, nblocks)) return;
    __shared__ double tot[6];
    sum_partials_ordered<6>(a.partial, nblocks, tot);
    if (threadIdx.x == 0) apply_dot_finish(a, tot);
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
        dinv[n] = s > 0.0 ? (T)(1.0 / (kdiag * s)) : T(0);  // no active element: the node drops out
    }
}

// Densities of the active set (Sec. 4.2.1): rho_e where rho_e > theta, else 0.
__global__ void cull_rho_kernel(size_t N, const double *rho, double theta, double *out) {
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < N; e += (size_t)gridDim.x * blockDim.x)
        out[e] = rho[e] > theta ? rho[e] : 0.0;
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
