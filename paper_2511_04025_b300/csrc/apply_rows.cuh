// apply_rows.cuh -- FP32 matrix-free stiffness apply q = K p (six load cases,
// Eq. inv-design cell problems; Sec. 4.2.2: finest level on the fly, all
// right-hand sides in one launch, converged right-hand sides skipped) for the
// grids r = 32, 48, 64, 96, 128, 256 (any multiple of 16 works: a row's pairs
// fill a group of 16 lanes or of whole warps, the rest of the group pads).
// Other grids, and the FP64 / double-float kinds, use apply_kernel
// (apply.cuh); both compute the same operator.
//
// Work split.  A CTA takes TY node rows (y) over the whole periodic x extent
// and a run of node planes (z) of one load case at a time (see the kernel).
// Its threads form TY + 1 element rows (row 0 is the halo row just below the
// tile); in a row, thread j holds the x-adjacent element pair (2j, 2j+1) and
// computes both elements at once with packed FP32 pairs (one f32x2
// instruction per two elements).  The CTA marches along z:
//  - the node rows (and density rows) of every plane arrive by bulk
//    asynchronous copies (one per component and contiguous run of rows),
//    issued by one warp several planes ahead into a ring of shared-memory
//    slots; each slot has an mbarrier that counts the bytes landed;
//  - per plane a thread transforms the top face of its two elements
//    (Walsh-Hadamard over x and y), combines it with the bottom face kept in
//    registers from the previous plane (z), applies the element operator in
//    its closed form (below) scaled by the two moduli, and transforms back;
//  - the +z half of the result is carried in registers to the next plane;
//    the +x corner goes to the next thread of the row by a warp shuffle
//    (the row is periodic: it wraps within the lane group, or through shared
//    memory when a row spans several warps); padding lanes compute on a copy
//    of the row's last pair and write nothing; the +y corner row goes to the
//    next element row through shared memory (one barrier per plane).
// A warp whose element pairs of a plane are all culled (E_e = 0: the active
// set of Sec. 4.2.1) skips the element operator for that plane.
// Deterministic, no atomics.
//
// Closed form of the transformed element blocks (element.cuh: G[c][i][j],
// character c, components i, j).  For the isotropic hex8 element the 45
// structural non-zeros take seven values for every Poisson ratio:
//   G[0] = (A-B) I + B J                    (J: all ones)
//   G[7] = D (I + J)
//   G[1<<t]     : rows/columns t zero, the other two [[P, Q], [Q, P]]
//   G[7^(1<<t)] : entry (t,t) = R, the other two [[F, F], [F, F]]
// so one element and load case costs 33 multiply/adds instead of 45 (7 more
// scale the constants by the element's modulus).  build_row_consts() reads
// the seven values off G and checks every block against this form.
#pragma once

#include "apply.cuh"

namespace shl {

struct RowConsts {
    float amb, b, p, q, f, rr, d;  // A-B, B, P, Q, F, R, D (h-scaled, E = 1)
};

// Returns the largest deviation of G from the closed form relative to
// max |G| (round-off when the form holds).
inline double build_row_consts(const ElemOp<double> &op, RowConsts *rc) {
    const auto &G = op.G;
    const double A = G[0][0][0], B = G[0][0][1], P = G[1][1][1], Q = G[1][1][2];
    const double F = G[3][0][0], R = G[3][2][2], D = G[7][0][1];
    double gmax = 0.0, dev = 0.0;
    for (int c = 0; c < 8; ++c)
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) {
                double want = 0.0;
                if (c == 0) {
                    want = i == j ? A : B;
                } else if (c == 7) {
                    want = i == j ? 2.0 * D : D;
                } else if (c == 1 || c == 2 || c == 4) {
                    const int t = c == 1 ? 0 : (c == 2 ? 1 : 2);
                    want = (i == t || j == t) ? 0.0 : (i == j ? P : Q);
                } else {
                    const int t = c == 6 ? 0 : (c == 5 ? 1 : 2);
                    want = (i == t && j == t) ? R : ((i == t || j == t) ? 0.0 : F);
                }
                gmax = std::fmax(gmax, std::fabs(G[c][i][j]));
                dev = std::fmax(dev, std::fabs(G[c][i][j] - want));
            }
    rc->amb = (float)(A - B);
    rc->b = (float)B;
    rc->p = (float)P;
    rc->q = (float)Q;
    rc->f = (float)F;
    rc->rr = (float)R;
    rc->d = (float)D;
    return gmax > 0.0 ? dev / gmax : 1.0;
}

// ---------------------------------------------------------------------------
// Packed FP32 pairs (f32x2)
// ---------------------------------------------------------------------------
__device__ __forceinline__ float2 p2add(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 p2mul(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 p2fma(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 p2sub(float2 a, float2 b) { return __fadd2_rn(a, make_float2(-b.x, -b.y)); }
__device__ __forceinline__ float2 p2splat(float v) { return make_float2(v, v); }

// ---------------------------------------------------------------------------
// mbarrier and bulk asynchronous copies (shared-memory addresses as u32)
// ---------------------------------------------------------------------------
__device__ __forceinline__ unsigned smem_u32(const void *p) { return (unsigned)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void mbar_init(unsigned bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(unsigned bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(unsigned bar, unsigned parity) {
    unsigned ok;
    asm volatile(
        "{\n .reg .pred p;\n"
        " mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}
// Bounded wait: false after `limit` unsuccessful polls (each poll itself
// blocks for a hardware-defined while), so a copy that never lands cannot
// hang the kernel.
__device__ __forceinline__ bool mbar_wait_bounded(unsigned bar, unsigned parity, unsigned limit = 1u << 22) {
    for (unsigned it = 0; it < limit; ++it)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}
__device__ __forceinline__ void bulk_g2s(unsigned dst, const void *src, unsigned bytes, unsigned bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(dst),
        "l"(src), "r"(bytes), "r"(bar)
        : "memory");
}
__device__ __forceinline__ void fence_barrier_init() { asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory"); }

// Error bits of the row apply (ApplyArgs::err).
constexpr unsigned kApplyErrWaitTimeout = 1u;

// Failure-detection probe: one CTA waits on an mbarrier that nothing
// completes, with at most `polls` bounded polls, and records the timeout in
// err as the row apply does; the kernel then returns normally.
__global__ void probe_wait_timeout_kernel(unsigned polls, unsigned *err) {
    __shared__ __align__(8) unsigned long long bar;
    const unsigned b = smem_u32(&bar);
    if (threadIdx.x == 0) {
        mbar_init(b, 1);
        fence_barrier_init();
    }
    __syncthreads();
    const bool ok = mbar_wait_bounded(b, 0, polls);  // phase 0 never completes: no arrival, no copy
    if (!ok && threadIdx.x == 0) atomicOr(err, kApplyErrWaitTimeout);
}

// ---------------------------------------------------------------------------
// Shape of one CTA
// ---------------------------------------------------------------------------
// Output node rows per CTA (TY) and resident CTAs per SM the registers are
// budgeted for (MINB), per grid size.  A CTA's warps spread over the SM's four
// schedulers, whose register files bound the registers per thread; the
// per-plane barrier makes the scheduler with the most warps set the pace, so
// the warps per CTA are best a multiple of four, with the CTAs of all load
// cases filling the 148 SMs.  Measured on B300 (us per launch): r = 32: TY 8
// (5 warps) 6.45, 11 (6 warps, 2 CTAs per SM) 5.48; r = 64: TY 7 (8 warps)
// 26.2, 8 (9 warps) 22.2, 11 (12 warps, 6 x 4 x 6 = 144 CTAs) 18.1, 15 (16
// warps) 22.8; r = 128: TY 3 (8 warps) 174, 4 (10) 163, 5 (12) 153, 7 (16)
// 139; r = 256: TY 2 (12 warps) 1248, 3 (16) 1116.
#ifndef SHL_ROWS_TY32
#define SHL_ROWS_TY32 11
#endif
#ifndef SHL_ROWS_MINB32
#define SHL_ROWS_MINB32 1
#endif
#ifndef SHL_ROWS_TY64
#define SHL_ROWS_TY64 11
#endif
#ifndef SHL_ROWS_MINB64
#define SHL_ROWS_MINB64 1
#endif
#ifndef SHL_ROWS_TY128
#define SHL_ROWS_TY128 7
#endif
#ifndef SHL_ROWS_MINB128
#define SHL_ROWS_MINB128 1
#endif
#ifndef SHL_ROWS_TY256
#define SHL_ROWS_TY256 3
#endif
#ifndef SHL_ROWS_MINB256
#define SHL_ROWS_MINB256 1
#endif
// Planes in flight ahead of use (PD) per grid size: measured on B300 (us),
// r = 64: PD 2 29.2, 3 17.8, 4 16.9, 5 17.0, 6 17.5; r = 128: 3 121.4, 4
// 119.9; r = 256: 3 1021, 4 1037; r = 32: 3 5.37, 4 5.48.
#ifndef SHL_ROWS_PD
#define SHL_ROWS_PD 3
#endif
#ifndef SHL_ROWS_PD64
#define SHL_ROWS_PD64 4
#endif
#ifndef SHL_ROWS_PD128
#define SHL_ROWS_PD128 4
#endif
__host__ __device__ constexpr int rows_pd_of(int r) {
    return r == 64 ? SHL_ROWS_PD64 : (r == 128 ? SHL_ROWS_PD128 : SHL_ROWS_PD);
}
#ifndef SHL_ROWS_ZUNROLL
#define SHL_ROWS_ZUNROLL 2
#endif
#ifndef SHL_ROWS_TY48
#define SHL_ROWS_TY48 8
#endif
#ifndef SHL_ROWS_TY96
#define SHL_ROWS_TY96 7
#endif
__host__ __device__ constexpr int rows_ty_of(int r) {
    return r == 32    ? SHL_ROWS_TY32
           : r == 48  ? SHL_ROWS_TY48
           : r == 64  ? SHL_ROWS_TY64
           : r == 96  ? SHL_ROWS_TY96
           : r == 128 ? SHL_ROWS_TY128
                      : SHL_ROWS_TY256;
}
__host__ __device__ constexpr int rows_minb_of(int r) {
    return r == 32 ? SHL_ROWS_MINB32 : (r == 64 ? SHL_ROWS_MINB64 : (r == 128 ? SHL_ROWS_MINB128 : SHL_ROWS_MINB256));
}

template <int R>
struct RowShape {
    // rows of 16-byte multiples for the bulk copies of the mask rows; one row's
    // element pairs fill a lane group of 16 lanes or whole warps
    static_assert(R % 16 == 0 && R >= 32 && R <= 256, "row apply: r must be a multiple of 16 in [32, 256]");
    static constexpr int TY = rows_ty_of(R);
    // TY need not divide r: the last tile's rows past the grid wrap around,
    // are computed and not stored
    static_assert(TY >= 1 && TY + 2 <= R, "row apply: 1 <= TY <= r - 2");
    static constexpr int MINB = rows_minb_of(R);
    static constexpr int P = R / 2;                // element pairs per row
    static constexpr int LPR = P <= 16 ? 16 : (P + 31) / 32 * 32;  // lanes per row (the last P..LPR-1 pad)
    static constexpr int NR = TY + 1;              // element rows, row 0 = halo
    static constexpr int NYR = TY + 2;             // node rows per plane
    static constexpr int LIVE = NR * LPR;          // threads with a row slot
    static constexpr int THREADS = (LIVE + 31) / 32 * 32;
    static constexpr int S = LPR >= 32 ? LPR / 32 : 1;  // warps per row
    static constexpr int PD = rows_pd_of(R);       // planes copied ahead of use
    static constexpr int NSLOT = PD + 1;           // ring slots
    static constexpr int NODE_BYTES = 3 * NYR * R * 4;
    template <bool SMOOTH>
    __host__ __device__ static constexpr int den_bytes() { return NR * R * (SMOOTH ? 8 : 1); }
    template <bool SMOOTH>
    __host__ __device__ static constexpr int slot_bytes() { return (NODE_BYTES + den_bytes<SMOOTH>() + 127) / 128 * 128; }
    template <bool SMOOTH>
    __host__ __device__ static constexpr int copy_bytes() { return NODE_BYTES + den_bytes<SMOOTH>(); }
    static constexpr int YTOP_FLOATS = 2 * NR * 3 * R;
    static constexpr int SPILL_FLOATS = S > 1 ? 2 * NR * S * 6 : 0;
    template <bool SMOOTH>
    __host__ __device__ static constexpr size_t smem() {
        return (size_t)NSLOT * slot_bytes<SMOOTH>() + sizeof(float) * (YTOP_FLOATS + SPILL_FLOATS) + 8 * NSLOT;
    }
};

// Density of one element pair -> its two moduli (EA, EB).
template <bool SMOOTH>
__device__ __forceinline__ float2 pair_modulus(const unsigned char *den_row, int x, float E, float Ev) {
    if constexpr (SMOOTH) {
        const double2 rho = *reinterpret_cast<const double2 *>(den_row + (size_t)x * 8);
        const float2 rf = make_float2(__double2float_rn(rho.x), __double2float_rn(rho.y));
        return p2fma(rf, p2splat(E - Ev), p2splat(Ev));
    } else {
        const unsigned m = *reinterpret_cast<const unsigned short *>(den_row + x);
        return make_float2((m & 0xffu) ? E : Ev, (m >> 8) ? E : Ev);
    }
}

// Work split.  The units are (load case, row tile, node plane) triples of the
// computed load cases, ordered by case, then tile, then z; CTA b takes the
// b-th of gridDim.x near-equal contiguous ranges.  A range cuts into z
// segments of row-tile columns, each one z march (two halo planes), so the
// grid balances over the SMs whatever the number of columns, and load cases
// that have converged take no CTAs.  With as many CTAs as a multiple of the
// columns, every range is one column chunk.
// DOT: the fused reduction, fixed per instantiation (a.dot must match): 0
// none, 1 p.q (q.q, mode 2, is left to the tile kernel, which serves the
// residual applies that use it); a CTA writes one row of six per-case sums.
// CULL (the culled void of the active set, a.Evoid = 0): a warp whose
// element pairs of a plane are all culled skips the element operator.
// Launched on a 1-D grid with exactly RowShape<R>::THREADS threads.
template <int R, bool SMOOTH, int DOT, bool CULL>
__global__ void __launch_bounds__(RowShape<R>::THREADS, RowShape<R>::MINB)
    apply_rows_kernel(const ApplyArgs<float> a, const RowConsts kc) {
    static_assert(DOT == 0 || DOT == 1, "row apply: DOT is 0 or 1");
    pdl_enter();
    using Sh = RowShape<R>;
    constexpr int TY = Sh::TY, P = Sh::P, NR = Sh::NR, NYR = Sh::NYR, S = Sh::S, PD = Sh::PD, NSLOT = Sh::NSLOT;
    constexpr int GY = (R + TY - 1) / TY;  // row tiles per load case
    constexpr int SLOT = Sh::template slot_bytes<SMOOTH>();
    constexpr int DEN_ROW = R * (SMOOTH ? 8 : 1);
    extern __shared__ __align__(16) unsigned char rows_smem[];  // 16-byte aligned: bulk-copy destinations
    unsigned char *const smraw = rows_smem;
    float *ytop = reinterpret_cast<float *>(smraw + (size_t)NSLOT * SLOT);  // [2][NR][3][R]
    float *spill = ytop + Sh::YTOP_FLOATS;                                  // [2][NR][S][2][3]
    unsigned long long *mbar = reinterpret_cast<unsigned long long *>(spill + Sh::SPILL_FLOATS);
    __shared__ double case_sum[6];  // p.q of each load case over the CTA's segments

    if (a.st && a.st->nactive == 0) return;  // uniform: the solve has finished
    // the load cases computed (bit k), the same in every CTA (flags loaded together)
    unsigned act = (unsigned)a.case_mask & ((1u << min(a.nvec, 6)) - 1u);
    {
        int fs[6], fi[6];
#pragma unroll
        for (int k = 0; k < 6; ++k) {
            fs[k] = a.st ? a.st->active[k] : 1;
            fi[k] = a.active_in ? a.active_in[k] : 1;
        }
#pragma unroll
        for (int k = 0; k < 6; ++k)
            if (fs[k] == 0 || fi[k] == 0) act &= ~(1u << k);
    }
    // this CTA's range of (case, row tile, node plane) units: W / gridDim.x
    // each, the first W % gridDim.x ranges one longer
    static_assert(6LL * GY * R < (1LL << 31), "row apply: unit count fits 32 bits");
    const unsigned W = (unsigned)__popc(act) * GY * R;
    const unsigned wq = W / gridDim.x, wr = W % gridDim.x;
    const unsigned w0 = blockIdx.x * wq + min(blockIdx.x, wr), w1 = w0 + wq + (blockIdx.x < wr ? 1u : 0u);

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    constexpr int LPR = Sh::LPR;
    // every thread holds a pair when the rows fill the CTA exactly (no padding)
    constexpr bool kFull = Sh::LIVE == Sh::THREADS && LPR == P;
    const bool slot_ok = kFull || tid < Sh::LIVE;
    const int jl = slot_ok ? tid % LPR : 0;          // lane within the row's lane group
    const bool live = kFull || (slot_ok && jl < P);  // holds an element pair (padding lanes write nothing)
    const int i = slot_ok ? tid / LPR : NR - 1;      // element row (idle threads shadow the last row)
    const int jp = live ? jl : P - 1;                // element pair (padding lanes shadow the last pair)
    const int x = 2 * jp;
    const int xn = x + 2 == R ? 0 : x + 2;  // node x + 2, periodic
    const int seg = jl / 32;
    // the left neighbour pair's lane (the row is periodic: pair 0's is pair P - 1);
    // across warps (S > 1) lane 0 takes it from the previous warp's spill word
    const int src_lane = S > 1 ? ((lane + 31) & 31) : ((lane & ~(LPR - 1)) + (jl == 0 ? P - 1 : jl - 1));
    const bool patch = (S > 1) && live && (lane == 0);
    const int last_lane = S > 1 ? min(31, P - 1 - 32 * seg) : 31;  // this warp's last pair
    const int segm1 = (seg + S - 1) % S;
    const size_t N = (size_t)R * R * R;
    const unsigned char *den = SMOOTH ? reinterpret_cast<const unsigned char *>(a.rho) : a.mask;
    const unsigned smem0 = smem_u32(smraw);
    const unsigned bar0 = smem_u32(mbar);

    if (tid == 0) {
        for (int b = 0; b < NSLOT; ++b) mbar_init(bar0 + 8 * b, 1);
        fence_barrier_init();
    }
    if (DOT != 0 && tid < 6) case_sum[tid] = 0.0;
    __syncthreads();

    // packed compensated sum of this thread's p.q over the current segment
    float2 ds = make_float2(0.f, 0.f), dc = make_float2(0.f, 0.f);
    bool wait_ok = true;
    unsigned g0 = 0;  // planes copied by earlier segments: plane t of this one uses ring position g0 + t

    for (unsigned w = w0; w < w1;) {
        // segment: node planes z0 .. z0 + tz - 1 of one row-tile column
        const int col = (int)(w / R), z0 = (int)(w % R);
        const int tz = (int)min((unsigned)(R - z0), w1 - w);
        int k;  // the (col / GY)-th computed load case
        {
            unsigned m = act;
            for (int j = col / GY; j > 0; --j) m &= m - 1;
            k = __ffs(m) - 1;
        }
        const int y0 = (col % GY) * TY;
        const float *pk = a.p + (size_t)(3 * k) * N;

        // plane t of the segment = node plane z0 - 1 + t (and its element plane's density rows)
        auto issue = [&](int t) {
            if (t > tz + 1) return;
            const int slot = (g0 + t) % NSLOT;
            const unsigned bar = bar0 + 8 * slot;
            const unsigned dst0 = smem0 + slot * SLOT;
            const int zt = wrapi(z0 - 1 + t, R);
            if (lane == 0) mbar_expect_tx(bar, (unsigned)Sh::template copy_bytes<SMOOTH>());
            __syncwarp();
            // The NYR node rows y0 - 1 .. y0 + TY of a component are contiguous
            // in memory except across the periodic wrap, so each component takes
            // one copy (two at the first and last tile), likewise the NR density
            // rows: at most 8 copies per plane, lanes 0..7.
            const int ys = wrapi(y0 - 1, R);
            const int n1 = ys + NYR <= R ? NYR : R - ys;  // node rows before the wrap
            const int d1 = ys + NR <= R ? NR : R - ys;    // density rows before the wrap
            if (lane < 8) {
                const int c = lane >> 1, part = lane & 1;
                if (c < 3) {
                    const int rows = part ? NYR - n1 : n1;
                    const int yg = part ? 0 : ys;     // first global row of the run
                    const int jj = part ? n1 : 0;     // first slot row of the run
                    if (rows > 0)
                        bulk_g2s(dst0 + (c * NYR + jj) * R * 4, pk + (size_t)c * N + ((size_t)zt * R + yg) * R,
                                 rows * R * 4, bar);
                } else {
                    const int rows = part ? NR - d1 : d1;
                    const int yg = part ? 0 : ys;
                    const int ii = part ? d1 : 0;
                    if (rows > 0)
                        bulk_g2s(dst0 + Sh::NODE_BYTES + ii * DEN_ROW,
                                 den + ((size_t)zt * R + yg) * (size_t)DEN_ROW, rows * DEN_ROW, bar);
                }
            }
        };
        auto wait_plane = [&](int t) {
            const unsigned gt = g0 + t;
            if (!mbar_wait_bounded(bar0 + 8 * (gt % NSLOT), (gt / NSLOT) & 1)) wait_ok = false;
        };

        // top face of plane t: Walsh-Hadamard over x, y of both elements' faces
        auto face = [&](int t, float2 (&ft)[3][4]) {
            const float *sb = reinterpret_cast<const float *>(smraw + ((g0 + t) % NSLOT) * SLOT);
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                const float *rb = sb + (c * NYR + i) * R;
                const float *rt = rb + R;
                const float2 b0 = *reinterpret_cast<const float2 *>(rb + x);
                const float b1 = rb[xn];
                const float2 t0 = *reinterpret_cast<const float2 *>(rt + x);
                const float t1 = rt[xn];
                const float2 a10 = make_float2(b0.y, b1), a11 = make_float2(t0.y, t1);
                const float2 s0 = p2add(b0, a10), d0 = p2sub(b0, a10);
                const float2 s1 = p2add(t0, a11), d1 = p2sub(t0, a11);
                ft[c][0] = p2add(s0, s1);
                ft[c][1] = p2add(d0, d1);
                ft[c][2] = p2sub(s0, s1);
                ft[c][3] = p2sub(d0, d1);
            }
        };

        // prologue: the first planes in flight, the bottom face of element plane z0 - 1
        if (warp == 0)
#pragma unroll 1
            for (int t = 0; t < PD; ++t) issue(t);
        float2 ftb[3][4], carry[3][4];
#pragma unroll
        for (int c = 0; c < 3; ++c)
#pragma unroll
            for (int j = 0; j < 4; ++j) carry[c][j] = make_float2(0.f, 0.f);
        wait_plane(0);
        face(0, ftb);

        // unrolled by two: the face arrays alternate roles between the copies
        // instead of being copied every plane
        constexpr int ZU = SHL_ROWS_ZUNROLL;
#pragma unroll ZU
        for (int s = 0; s <= tz; ++s) {
            wait_plane(s + 1);
            // moduli of element plane z0 - 1 + s (density rows of plane s)
            const float2 Ee = pair_modulus<SMOOTH>(smraw + ((g0 + s) % NSLOT) * SLOT + Sh::NODE_BYTES + i * DEN_ROW,
                                                   x, a.E, a.Evoid);
            float2 ftt[3][4];
            face(s + 1, ftt);
            // A warp whose element pairs of this plane are all culled (E_e = 0,
            // the active set) adds exact zeros: it skips the element operator
            // and only hands on the top faces carried from the plane below.
            bool void_warp = false;
            if constexpr (CULL) void_warp = __all_sync(0xffffffffu, Ee.x == 0.f && Ee.y == 0.f);
            // back to corners: z split (bottom face = node plane z0 - 1 + s, top
            // face carried), then x, y.  W[c][b]: corner b = bx + 2 by of both
            // elements (packed).
            float2 W[3][4];
            auto corners = [&](int c, const float2 (&F)[4]) {
                const float2 t0 = p2add(F[0], F[1]), t1 = p2sub(F[0], F[1]), t2 = p2add(F[2], F[3]),
                             t3 = p2sub(F[2], F[3]);
                W[c][0] = p2add(t0, t2);
                W[c][1] = p2add(t1, t3);
                W[c][2] = p2sub(t0, t2);
                W[c][3] = p2sub(t1, t3);
            };
            if (void_warp) {
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    float2 F[4];
                    F[0] = make_float2(-carry[c][0].x, -carry[c][0].y);
                    carry[c][0] = make_float2(0.f, 0.f);
#pragma unroll
                    for (int j = 1; j < 4; ++j) {
                        F[j] = carry[c][j];
                        carry[c][j] = make_float2(0.f, 0.f);
                    }
                    corners(c, F);
                }
            } else {
                // transformed element displacements u[c][m] (mode m = x + 2y + 4z bits)
                float2 u[3][8];
#pragma unroll
                for (int c = 0; c < 3; ++c) {
#pragma unroll
                    for (int j = 1; j < 4; ++j) u[c][j] = p2add(ftb[c][j], ftt[c][j]);
#pragma unroll
                    for (int j = 0; j < 4; ++j) u[c][j + 4] = p2sub(ftb[c][j], ftt[c][j]);
                }
                // y = E G u in the closed form (the translation modes u[c][0] and
                // y[c][0] are zero)
                // E-scaled constants: scalar products with the parameter-bank values
                // (no registers held for the constants)
                const float2 eA = p2mul(Ee, p2splat(kc.amb)), eB = p2mul(Ee, p2splat(kc.b)),
                             eP = p2mul(Ee, p2splat(kc.p)), eQ = p2mul(Ee, p2splat(kc.q)),
                             eF = p2mul(Ee, p2splat(kc.f)), eR = p2mul(Ee, p2splat(kc.rr)),
                             eD = p2mul(Ee, p2splat(kc.d));
                float2 y[3][8];
                {  // c = 0: (u01, u12, u24) -> (y01, y12, y24)
                    const float2 t0 = p2mul(eB, p2add(p2add(u[0][1], u[1][2]), u[2][4]));
                    y[0][1] = p2fma(eA, u[0][1], t0);
                    y[1][2] = p2fma(eA, u[1][2], t0);
                    y[2][4] = p2fma(eA, u[2][4], t0);
                }
                {  // c = 7: (u06, u15, u23)
                    const float2 t7 = p2mul(eD, p2add(p2add(u[0][6], u[1][5]), u[2][3]));
                    y[0][6] = p2fma(eD, u[0][6], t7);
                    y[1][5] = p2fma(eD, u[1][5], t7);
                    y[2][3] = p2fma(eD, u[2][3], t7);
                }
                // c = 1 (t = 0): (u13, u25); c = 2 (t = 1): (u03, u26); c = 4 (t = 2): (u05, u16)
                y[1][3] = p2fma(eP, u[1][3], p2mul(eQ, u[2][5]));
                y[2][5] = p2fma(eP, u[2][5], p2mul(eQ, u[1][3]));
                y[0][3] = p2fma(eP, u[0][3], p2mul(eQ, u[2][6]));
                y[2][6] = p2fma(eP, u[2][6], p2mul(eQ, u[0][3]));
                y[0][5] = p2fma(eP, u[0][5], p2mul(eQ, u[1][6]));
                y[1][6] = p2fma(eP, u[1][6], p2mul(eQ, u[0][5]));
                // c = 6 (t = 0): u07 -> y07, (u14, u22) -> y14 = y22; c = 5 (t = 1): u17, (u04, u21);
                // c = 3 (t = 2): u27, (u02, u11)
                y[0][7] = p2mul(eR, u[0][7]);
                y[1][4] = y[2][2] = p2mul(eF, p2add(u[1][4], u[2][2]));
                y[1][7] = p2mul(eR, u[1][7]);
                y[0][4] = y[2][1] = p2mul(eF, p2add(u[0][4], u[2][1]));
                y[2][7] = p2mul(eR, u[2][7]);
                y[0][2] = y[1][1] = p2mul(eF, p2add(u[0][2], u[1][1]));

#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    float2 F[4];
                    F[0] = p2sub(y[c][4], carry[c][0]);  // carry[c][0] holds -(top of mode 0) = y_prev[c][4]
                    carry[c][0] = y[c][4];
#pragma unroll
                    for (int j = 1; j < 4; ++j) {
                        F[j] = p2add(carry[c][j], p2add(y[c][j], y[c][j + 4]));
                        carry[c][j] = p2sub(y[c][j], y[c][j + 4]);
                    }
                    corners(c, F);
                }
            }
            // x exchange: node x gets the +x corner of the left neighbour's second element
            float rb1[3], rb3[3];
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                rb1[c] = __shfl_sync(0xffffffffu, W[c][1].y, src_lane);
                rb3[c] = __shfl_sync(0xffffffffu, W[c][3].y, src_lane);
            }
            // top-row partial for the next element row (node row i + 1)
            const int par = s & 1;
            float *yt = ytop + ((size_t)(par * NR + i) * 3) * R;
            if (live) {
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    const float2 ot = p2add(W[c][2], make_float2(patch ? 0.f : rb3[c], W[c][3].x));
                    *reinterpret_cast<float2 *>(yt + c * R + x) = ot;
                }
                if (S > 1 && lane == last_lane) {
                    float *sp = spill + ((size_t)((par * NR + i) * S + seg) * 2) * 3;
#pragma unroll
                    for (int c = 0; c < 3; ++c) {
                        sp[c] = W[c][1].y;
                        sp[3 + c] = W[c][3].y;
                    }
                }
            }
            __syncthreads();
            // Refill the slot of plane s - 1: every read of it (its face at step
            // s - 2, its density rows and own-node values at step s - 1) came
            // before this barrier.  Its values were consumed into registers, so
            // no proxy fence is needed (one would also wait for this thread's
            // outstanding global stores).
            if (warp == 0) issue(s + PD);
            const int ez = z0 - 1 + s;
            if (s >= 1 && live && i >= 1 && y0 - 1 + i < R) {
                const float *ytp = ytop + ((size_t)(par * NR + i - 1) * 3) * R;
                const float *spb = spill + ((size_t)((par * NR + i) * S + segm1) * 2) * 3;      // own row, left warp
                const float *spt = spill + ((size_t)((par * NR + i - 1) * S + segm1) * 2) * 3;  // row below, left warp
                const int ny = y0 - 1 + i;  // node row (inside the tile and the grid)
                const size_t nrow = ((size_t)ez * R + ny) * R + x;
                float *qrow = a.q + (size_t)(3 * k) * N + nrow;
                const bool pin_here = a.pin && ez == 0 && ny == 0 && x == 0;
                // p at the pair's own nodes (x, x + 1) of node row i, bottom plane s (for p.q)
                const float *own = reinterpret_cast<const float *>(smraw + ((g0 + s) % NSLOT) * SLOT) + i * R + x;
                float2 v = make_float2(0.f, 0.f);  // this plane's three products (per element of the pair)
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    float2 otp = *reinterpret_cast<const float2 *>(ytp + c * R + x);
                    float recv1 = rb1[c];
                    if (patch) {
                        recv1 = spb[c];
                        otp.x += spt[3 + c];
                    }
                    float2 qv = p2add(p2add(W[c][0], make_float2(recv1, W[c][1].x)), otp);
                    if (pin_here) qv.x = 0.f;
                    *reinterpret_cast<float2 *>(qrow + (size_t)c * N) = qv;
                    if constexpr (DOT != 0) {
                        const float2 w = *reinterpret_cast<const float2 *>(own + c * NYR * R);
                        v = c == 0 ? p2mul(qv, w) : p2fma(qv, w, v);
                    }
                }
                if constexpr (DOT != 0) {  // one packed compensated add per plane
                    const float2 yv = p2sub(v, dc);
                    const float2 tv = p2add(ds, yv);
                    dc = p2sub(p2sub(tv, ds), yv);
                    ds = tv;
                }
            }
#pragma unroll
            for (int c = 0; c < 3; ++c)
#pragma unroll
                for (int j = 0; j < 4; ++j) ftb[c][j] = ftt[c][j];
        }
        // every plane issued was waited for in the loop; nothing is in flight
        g0 += tz + 2;
        if constexpr (DOT != 0) {  // the segment's p.q into its load case's sum
            const float2 v[1] = {df_add(two_sum(ds.x, -dc.x), two_sum(ds.y, -dc.y))};
            double sum[1];
            block_sum_df<1>(v, sum);
            if (tid == 0) case_sum[k] += sum[0];
            ds = dc = make_float2(0.f, 0.f);
        }
        __syncthreads();  // ring slots and +y rows are free for the next segment
        w += tz;
    }
    if (!wait_ok && a.err) atomicOr(a.err, kApplyErrWaitTimeout);

    if constexpr (DOT != 0) {
        // the CTA's row of partials: one sum per load case (zero where it had no segment)
        const unsigned nblocks = gridDim.x;
        if (tid < 6) a.partial[(size_t)blockIdx.x * 6 + tid] = case_sum[tid];
        if (a.defer) return;  // the consumer reduces the per-CTA partials itself
        if (!last_block_ticket(a.ticket, nblocks)) return;
        __shared__ double tot[6];
        sum_partials_ordered<6>(a.partial, nblocks, tot);
        if (tid == 0) apply_dot_finish(a, tot);
    }
}

}  // namespace shl
