// shl.cu -- libshl C-ABI entry points (include/shl.h) and the host drivers of
// the solve.  One translation unit for the whole library.
#include "apply_rows.cuh"
#include "chom.cuh"
#include "common.cuh"
#include "element.cuh"
#include "field.cuh"
#include "pcg.cuh"
#include "probe.cuh"
#include "adjoint.cuh"
#include "mg.cuh"
#include "vec.cuh"

#include <atomic>
#include <functional>
#include <type_traits>
#include <utility>

using namespace shl;

namespace shl {

constexpr int kTX = 16, kTY = 16;

inline int grid1d(size_t n, int threads = kBlk, int cap = 148 * 8) {
    size_t b = (n + threads - 1) / threads;
    if (b < 1) b = 1;
    if (b > (size_t)cap) b = cap;
    return (int)b;
}

// Dynamic shared-memory opt-in of the apply kernels, once per device
// (thread-safe; setting it twice is harmless).
template <typename T>
void apply_smem_attr() {
    static std::atomic<unsigned long long> done{0};
    int dev = 0;
    cudaGetDevice(&dev);
    const unsigned long long bit = 1ull << (dev & 63);
    if (done.load(std::memory_order_acquire) & bit) return;
    const int sm = (int)ApplyShape<T, kTX, kTY>::smem();
    cudaFuncSetAttribute(apply_kernel<T, kTX, kTY, false, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
    cudaFuncSetAttribute(apply_kernel<T, kTX, kTY, true, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
    cudaFuncSetAttribute(apply_kernel<T, kTX, kTY, false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
    cudaFuncSetAttribute(apply_kernel<T, kTX, kTY, true, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
    done.fetch_or(bit, std::memory_order_release);
}

// Raise a kernel's dynamic shared-memory limit to at least `bytes` on the
// current device.  The limit is a per-function attribute shared by every
// thread, so it only ever grows: a concurrent launch that needs less is never
// refused because another thread lowered it.
inline void raise_smem_limit(const void *fn, size_t bytes) {
    static std::mutex mu;
    static std::map<std::pair<const void *, int>, size_t> cur;
    int dev = 0;
    cudaGetDevice(&dev);
    std::lock_guard<std::mutex> lk(mu);
    size_t &c = cur[{fn, dev}];
    if (bytes <= c) return;
    if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes) == cudaSuccess)
        c = bytes;
    else
        cudaGetLastError();
}

// Launch with programmatic stream serialisation (the kernel starts with
// pdl_enter(): it waits for the preceding kernel before touching memory, and
// its launch overlaps that kernel's tail).  SHL_PDL=0 at compile time makes
// these ordinary launches.
#ifndef SHL_PDL
#define SHL_PDL 1
#endif
template <typename... KArgs, typename... Args>
inline void pdl_launch(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                       Args &&...args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = SHL_PDL;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
}

// Number of z chunks of the apply grid.  Chunk heights differ by at most one
// plane; the count minimises the modelled makespan
//   ceil(CTAs / resident CTA slots) x (tallest chunk + 1 halo plane + 1 for the prologue),
// i.e. it keeps whole waves of equal-work CTAs on the 148 SMs.
inline int pick_zc(int r, int nvec, int ctas_per_sm) {
    const long long nxy = (long long)((r + kTX - 1) / kTX) * ((r + kTY - 1) / kTY) * nvec;
    const long long slots = 148LL * ctas_per_sm;
    int best = 1;
    long long best_cost = -1;
    for (int zc = 1; zc <= r && zc <= 128; ++zc) {
        const long long h = (r + zc - 1) / zc;
        const long long cost = ((nxy * zc + slots - 1) / slots) * (h + 2);
        if (best_cost < 0 || cost < best_cost) {
            best = zc;
            best_cost = cost;
        }
    }
    return best;
}

template <typename T>
inline int apply_zc(int r, int nvec) {
    return pick_zc(r, nvec, sizeof(T) == 4 ? 2 : 1);
}

// ---------------------------------------------------------------------------
// Row apply (apply_rows.cuh): FP32, r = 32, 48, 64, 96, 128, 256
// ---------------------------------------------------------------------------
inline bool rows_grid(int r) { return r == 32 || r == 48 || r == 64 || r == 96 || r == 128 || r == 256; }
inline int rows_ty(int r) { return rows_ty_of(r); }

// Shared-memory opt-in and resident CTAs per SM of one row-apply kernel on
// the current device (queried once per device).
template <int R, bool SMOOTH>
inline int rows_prepare() {
    static std::mutex mu;
    static int occ[64] = {0};
    int dev = 0;
    cudaGetDevice(&dev);
    dev &= 63;
    std::lock_guard<std::mutex> lk(mu);
    if (occ[dev] == 0) {
        const size_t sm = RowShape<R>::template smem<SMOOTH>();
        // one geometry (and partials layout) for every DOT / CULL variant
        const void *fns[4] = {(const void *)apply_rows_kernel<R, SMOOTH, 0, false>,
                              (const void *)apply_rows_kernel<R, SMOOTH, 1, false>,
                              (const void *)apply_rows_kernel<R, SMOOTH, 0, true>,
                              (const void *)apply_rows_kernel<R, SMOOTH, 1, true>};
        int n = 1 << 30;
        for (const void *f : fns) {
            int nf = 0;
            if (cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm) != cudaSuccess ||
                cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nf, f, RowShape<R>::THREADS, sm) != cudaSuccess) {
                cudaGetLastError();
                nf = 0;
            }
            n = std::min(n, nf);
        }
        occ[dev] = n > 0 ? n : -1;
    }
    return occ[dev];
}
inline int rows_occupancy(int r, bool smooth) {
    switch (r) {
        case 32: return smooth ? rows_prepare<32, true>() : rows_prepare<32, false>();
        case 48: return smooth ? rows_prepare<48, true>() : rows_prepare<48, false>();
        case 64: return smooth ? rows_prepare<64, true>() : rows_prepare<64, false>();
        case 96: return smooth ? rows_prepare<96, true>() : rows_prepare<96, false>();
        case 128: return smooth ? rows_prepare<128, true>() : rows_prepare<128, false>();
        case 256: return smooth ? rows_prepare<256, true>() : rows_prepare<256, false>();
    }
    return -1;
}
// CTAs of the row apply (a 1-D grid over contiguous ranges of (case, row
// tile, node plane) units; see apply_rows_kernel).  Two candidates by their
// makespan in planes per CTA (each z segment adds two halo planes): a
// multiple of the row-tile columns, every CTA one equal z chunk of one column
// (balanced when the columns divide the resident CTAs well), or every
// resident CTA with ranges that straddle column ends.
inline int rows_ctas(int r, int nvec, int ctas_per_sm) {
    const long long ncol = (long long)((r + rows_ty(r) - 1) / rows_ty(r)) * nvec;
    const long long slots = 148LL * ctas_per_sm;
    const long long W = ncol * r;
    long long best_nb = 0, best_cost = -1;
    if (ncol <= slots) {
        const long long m = std::min<long long>(slots / ncol, r);
        best_nb = ncol * m;
        best_cost = (r + m - 1) / m + 2;
    }
    {
        const long long nb = std::max(1LL, std::min(slots, W / 4));
        const long long L = (W + nb - 1) / nb;
        const long long cost = L + 2 * (1 + (L - 1 + r - 1) / r);
        if (best_cost < 0 || cost < best_cost) best_nb = nb;
    }
    return (int)best_nb;
}

// Launch geometry of the apply for grid r, nvec load cases and a density
// buffer: the row kernel when it serves this grid (FP32, r = 32..256, density
// rows 16-byte aligned for the bulk copies), else the tile kernel.  The
// deferred p.q partials are laid out by it (gx * gy rows per load case).
struct ApplyGeom {
    int gx, gy, rows;
    // rows of per-CTA p.q partials: one per CTA of the 1-D row-apply grid, one
    // per CTA and load case of the tile kernel's (gx, gy, nvec) grid
    size_t partial_rows(int nvec) const { return rows ? (size_t)gx : (size_t)gx * gy * nvec; }
};
template <typename T>
inline ApplyGeom apply_geom(int r, int nvec, const uint8_t *mask, const double *rho) {
    const void *den = rho ? (const void *)rho : (const void *)mask;
    if (std::is_same<T, float>::value && rows_grid(r) && den && (reinterpret_cast<uintptr_t>(den) & 15) == 0) {
        const int occ = rows_occupancy(r, rho != nullptr);
        if (occ > 0) return ApplyGeom{rows_ctas(r, nvec, occ), 1, 1};
    }
    return ApplyGeom{((r + kTX - 1) / kTX) * ((r + kTY - 1) / kTY), apply_zc<T>(r, nvec), 0};
}

template <int R, bool SMOOTH>
inline void rows_launch(dim3 g, cudaStream_t s, const ApplyArgs<float> &a, const RowConsts &kc) {
    constexpr int NT = RowShape<R>::THREADS;
    const size_t sm = RowShape<R>::template smem<SMOOTH>();
    const bool cull = a.Evoid == 0.0f;  // the active set: culled elements carry no stiffness
    if (a.dot == 1)
        pdl_launch(cull ? apply_rows_kernel<R, SMOOTH, 1, true> : apply_rows_kernel<R, SMOOTH, 1, false>, g, NT, sm,
                   s, a, kc);
    else
        pdl_launch(cull ? apply_rows_kernel<R, SMOOTH, 0, true> : apply_rows_kernel<R, SMOOTH, 0, false>, g, NT, sm,
                   s, a, kc);
}
template <int R>
inline void rows_launch_r(dim3 g, cudaStream_t s, const ApplyArgs<float> &a, const RowConsts &kc) {
    if (a.rho)
        rows_launch<R, true>(g, s, a, kc);
    else
        rows_launch<R, false>(g, s, a, kc);
}

template <typename T>
inline int launch_apply_rows(shl_ctx *ctx, ApplyArgs<T> a, const ApplyGeom &geo, cudaStream_t s) {
    if constexpr (!std::is_same<T, float>::value) {
        return set_err(ctx, SHL_EINVAL, "internal: row apply is FP32 only");
    } else {
        RowConsts kc;
        double dev = 0.0;
        {
            ElemOp<double> od;
            for (int c = 0; c < 8; ++c)
                for (int i = 0; i < 3; ++i)
                    for (int j = 0; j < 3; ++j) od.G[c][i][j] = (double)a.op.G[c][i][j];
            dev = build_row_consts(od, &kc);
        }
        if (!(dev < 1e-5)) return set_err(ctx, SHL_EINVAL, "element blocks off their closed form (%g)", dev);
        if (!a.err) SHL_TRY(ws_get_t(ctx, "apply_err", 1, &a.err));
        a.zc = 1;
        const dim3 g(geo.gx, 1, 1);
        switch (a.r) {
            case 32: rows_launch_r<32>(g, s, a, kc); break;
            case 48: rows_launch_r<48>(g, s, a, kc); break;
            case 64: rows_launch_r<64>(g, s, a, kc); break;
            case 96: rows_launch_r<96>(g, s, a, kc); break;
            case 128: rows_launch_r<128>(g, s, a, kc); break;
            case 256: rows_launch_r<256>(g, s, a, kc); break;
            default:
                return set_err(ctx, SHL_EINVAL, "internal: row apply for r=%d", a.r);
        }
        ++ctx->launches;
        SHL_CUDA(ctx, cudaGetLastError());
        return SHL_OK;
    }
}

template <typename T>
int launch_apply(shl_ctx *ctx, ApplyArgs<T> a, cudaStream_t s) {
    using S = ApplyShape<T, kTX, kTY>;
    ApplyGeom geo = apply_geom<T>(a.r, a.nvec, a.mask, a.rho);
    if (geo.rows) {
        // the bulk row copies need 16-byte aligned rows of p, the paired stores 8-byte aligned q
        const bool ok = !a.resid && (a.dot == 0 || a.dot == 1) && a.p && (reinterpret_cast<uintptr_t>(a.p) & 15) == 0 &&
                        (reinterpret_cast<uintptr_t>(a.q) & 7) == 0;
        if (!ok && a.dot && a.defer)
            return set_err(ctx, SHL_EINVAL, "internal: deferred apply partials need aligned p and q");
        if (ok) {
            if (a.dot) {
                if (!a.partial) {
                    double *partial = nullptr;
                    SHL_TRY(ws_get_t(ctx, "apply_partial", geo.partial_rows(a.nvec) * 6, &partial));
                    a.partial = partial;
                }
                if (!a.ticket) {
                    unsigned *ticket = nullptr;
                    SHL_TRY(ws_get_t(ctx, "apply_ticket", 1, &ticket));
                    a.ticket = ticket;
                }
            }
            return launch_apply_rows<T>(ctx, a, geo, s);
        }
        geo = ApplyGeom{((a.r + kTX - 1) / kTX) * ((a.r + kTY - 1) / kTY), apply_zc<T>(a.r, a.nvec), 0};
    }
    apply_smem_attr<T>();
    a.zc = geo.gy;
    const dim3 g(geo.gx, a.zc, a.nvec);
    a.vec_ok = (a.r % S::VEC == 0) && ((reinterpret_cast<uintptr_t>(a.p) & 15) == 0);
    if (a.dot) {
        if (!a.partial) {
            double *partial = nullptr;
            SHL_TRY(ws_get_t(ctx, "apply_partial", (size_t)g.x * g.y * g.z * 6, &partial));
            a.partial = partial;
        }
        if (!a.ticket) {
            unsigned *ticket = nullptr;
            SHL_TRY(ws_get_t(ctx, "apply_ticket", 1, &ticket));
            a.ticket = ticket;
        }
    }
    if (a.rho) {
        if (a.resid)
            pdl_launch(apply_kernel<T, kTX, kTY, true, true>, g, S::THREADS, S::smem(), s, a);
        else
            pdl_launch(apply_kernel<T, kTX, kTY, false, true>, g, S::THREADS, S::smem(), s, a);
    } else {
        if (a.resid)
            pdl_launch(apply_kernel<T, kTX, kTY, true, false>, g, S::THREADS, S::smem(), s, a);
        else
            pdl_launch(apply_kernel<T, kTX, kTY, false, false>, g, S::THREADS, S::smem(), s, a);
    }
    ++ctx->launches;
    SHL_CUDA(ctx, cudaGetLastError());
    return SHL_OK;
}

// Transformed element operator for (nu, r), built on the host once and kept
// in a small process-wide cache (building it costs tens of microseconds, more
// than an apply launch at small grids).
template <typename T>
int get_op(shl_ctx *ctx, double nu, int r, ElemOp<T> *op) {
    static std::mutex mu;
    static std::map<std::pair<double, int>, ElemOp<T>> cache;
    {
        std::lock_guard<std::mutex> lk(mu);
        auto it = cache.find({nu, r});
        if (it != cache.end()) {
            *op = it->second;
            return SHL_OK;
        }
    }
    const double off = build_elem_op<T>(nu, r, op);
    if (!(off < 1e-12)) return set_err(ctx, SHL_EINVAL, "element operator is not block diagonal (%g)", off);
    std::lock_guard<std::mutex> lk(mu);
    if (cache.size() >= 64) cache.clear();
    cache[{nu, r}] = *op;
    return SHL_OK;
}

struct Uploaded {
    double *pos, *q, *alpha;
};

inline int validate_design(shl_ctx *ctx, const shl_design *d, int r) {
    if (!d) return set_err(ctx, SHL_EINVAL, "design is NULL");
    if (d->n < 1 || d->n > (1 << 20)) return set_err(ctx, SHL_EINVAL, "charge count %d out of range [1, 2^20]", d->n);
    if (d->K < 1 || d->K > kMaxK)
        return set_err(ctx, SHL_EINVAL, "truncation order K=%d out of range [1, %d]", d->K, kMaxK);
    if (!d->pos || !d->q) return set_err(ctx, SHL_EINVAL, "design pos/q is NULL");
    if (r < 2 || r > 1024) return set_err(ctx, SHL_EINVAL, "grid size r=%d out of range [2, 1024]", r);
    for (int j = 0; j < 3 * d->n; ++j)
        if (!std::isfinite(d->pos[j])) return set_err(ctx, SHL_EINVAL, "non-finite charge position");
    for (int j = 0; j < d->n; ++j)
        if (!std::isfinite(d->q[j])) return set_err(ctx, SHL_EINVAL, "non-finite charge magnitude");
    if (!std::isfinite(d->iso)) return set_err(ctx, SHL_EINVAL, "non-finite iso-level");
    if (!(d->t > 0.0) && !(d->vf > 0.0 && d->vf < 1.0))
        return set_err(ctx, SHL_EINVAL, "design needs t > 0 or a volume fraction in (0,1), got t=%g vf=%g", d->t,
                       d->vf);
    return SHL_OK;
}

inline int upload_design(shl_ctx *ctx, const shl_design *d, cudaStream_t s, Uploaded *u, const char *tag) {
    const int na = (d->K + 1) * (d->K + 1) * (d->K + 1);
    double *buf = nullptr;
    SHL_TRY(ws_get_t(ctx, std::string("design_") + tag, (size_t)4 * d->n + na, &buf));
    u->pos = buf;
    u->q = buf + 3 * d->n;
    u->alpha = d->alpha ? buf + 4 * d->n : nullptr;
    SHL_CUDA(ctx, cudaMemcpyAsync(u->pos, d->pos, sizeof(double) * 3 * d->n, cudaMemcpyHostToDevice, s));
    SHL_CUDA(ctx, cudaMemcpyAsync(u->q, d->q, sizeof(double) * d->n, cudaMemcpyHostToDevice, s));
    if (d->alpha) SHL_CUDA(ctx, cudaMemcpyAsync(u->alpha, d->alpha, sizeof(double) * na, cudaMemcpyHostToDevice, s));
    return SHL_OK;
}

// F / gradF / d on the grid.
inline int run_field(shl_ctx *ctx, const shl_design *d, int r, double *F, double *gF, double *dd, cudaStream_t s) {
    Uploaded u;
    SHL_TRY(upload_design(ctx, d, s, &u, "field"));
    const int nb = 2 * d->K + 1;
    double *A = nullptr;
    SHL_TRY(ws_get_t(ctx, "field_A", (size_t)nb * nb * nb, &A));
    field_coef_kernel<<<1, 512, 0, s>>>(d->n, d->K, u.pos, u.q, u.alpha, A);
    ++ctx->launches;
    SHL_CUDA(ctx, cudaGetLastError());
    int lines = r;
    while (lines > 1 && field_smem_bytes(r, d->K, lines) > 96 * 1024) lines = (lines + 1) / 2;
    while (lines > 4 && (size_t)r * ((r + lines - 1) / lines) < 4 * 148) lines = (lines + 1) / 2;
    FieldArgs fa{r, d->K, lines, d->iso, A, F, gF, dd};
    const size_t smem = field_smem_bytes(r, d->K, lines);
    raise_smem_limit((const void *)field_grid_kernel, smem);
    field_grid_kernel<<<dim3(r, (r + lines - 1) / lines), 256, smem, s>>>(fa);
    ++ctx->launches;
    SHL_CUDA(ctx, cudaGetLastError());
    return SHL_OK;
}

// Threshold selection from d (device); result left in the device SelectState.
inline int run_select(shl_ctx *ctx, const double *dd, size_t n, double vf, cudaStream_t s, SelectState **out) {
    SelectState *st = nullptr;
    SHL_TRY(ws_get_t(ctx, "select_state", 1, &st));
    long long k0 = llround(vf * (double)n);
    if (k0 < 1) k0 = 1;
    if (k0 > (long long)n - 1) k0 = (long long)n - 1;
    const long long lo = std::max(1LL, k0 - kSelW), hi = std::min((long long)n, k0 + kSelW + 1);
    static thread_local SelectState init;  // host staging (only the header part is copied)
    std::memset(&init, 0, offsetof(SelectState, buf));
    init.rank[0] = (unsigned long long)lo;
    init.rank[1] = (unsigned long long)hi;
    SHL_CUDA(ctx, cudaMemcpyAsync(st, &init, offsetof(SelectState, buf), cudaMemcpyHostToDevice, s));
    const unsigned long long *keys = reinterpret_cast<const unsigned long long *>(dd);
    const int g = grid1d(n, 256, 148 * 4);
    const int shifts[6] = {53, 42, 31, 20, 9, 0};
    const int widths[6] = {11, 11, 11, 11, 11, 9};
    for (int p = 0; p < 6; ++p) {
        select_hist_kernel<<<g, 256, 0, s>>>(keys, n, st, shifts[p], widths[p]);
        select_choose_kernel<<<1, kSelChooseThreads, 0, s>>>(st, shifts[p]);
        ctx->launches += 2;
    }
    select_gather_kernel<<<g, 256, 0, s>>>(keys, n, st);
    ++ctx->launches;
    select_finish_kernel<<<1, 1024, 0, s>>>(st, (long long)n, k0);
    ++ctx->launches;
    SHL_CUDA(ctx, cudaGetLastError());
    // the host staging struct is reused: make sure its copy has completed
    SHL_CUDA(ctx, cudaStreamSynchronize(s));
    *out = st;
    return SHL_OK;
}

struct VoxOut {
    double t = 0, margin = 0;
    long long n_solid = 0, n_amb = 0;
};

inline int run_voxelize(shl_ctx *ctx, const shl_design *d, int r, double kappa, uint8_t *mask, double *rho,
                        double *d_out, cudaStream_t s, VoxOut *res) {
    const size_t n = (size_t)r * r * r;
    const bool choose = !(d->t > 0.0);
    double *dd = d_out;
    if (!dd) SHL_TRY(ws_get_t(ctx, "vox_d", n, &dd));
    SHL_TRY(run_field(ctx, d, r, nullptr, nullptr, dd, s));
    SelectState *sel = nullptr;
    if (choose) SHL_TRY(run_select(ctx, dd, n, d->vf, s, &sel));
    unsigned long long *counts = nullptr;
    SHL_TRY(ws_get_t(ctx, "vox_counts", 2, &counts));
    SHL_CUDA(ctx, cudaMemsetAsync(counts, 0, 2 * sizeof(unsigned long long), s));
    if (kappa <= 0.0) kappa = std::log(9.0) * r;
    voxel_mask_kernel<<<grid1d(n, 256, 148 * 8), 256, 0, s>>>(dd, n, sel, d->t, kappa, mask, rho, counts);
    ++ctx->launches;
    SHL_CUDA(ctx, cudaGetLastError());
    unsigned long long hc[2];
    SHL_CUDA(ctx, cudaMemcpyAsync(hc, counts, sizeof(hc), cudaMemcpyDeviceToHost, s));
    if (choose) {
        int status = 0;
        double t = 0, margin = 0;
        SHL_CUDA(ctx, cudaMemcpyAsync(&status, &sel->status, sizeof(int), cudaMemcpyDeviceToHost, s));
        SHL_CUDA(ctx, cudaMemcpyAsync(&t, &sel->t, sizeof(double), cudaMemcpyDeviceToHost, s));
        SHL_CUDA(ctx, cudaMemcpyAsync(&margin, &sel->margin, sizeof(double), cudaMemcpyDeviceToHost, s));
        SHL_CUDA(ctx, cudaStreamSynchronize(s));
        if (status == 2) return set_err(ctx, SHL_EINVAL, "threshold selection: too many tied distances near rank");
        if (status != 0) return set_err(ctx, SHL_EINVAL, "threshold selection: no resolvable gap within 64 ranks");
        res->t = t;
        res->margin = margin;
    } else {
        SHL_CUDA(ctx, cudaStreamSynchronize(s));
        res->t = d->t;
        res->margin = 0.0;
    }
    res->n_solid = (long long)hc[0];
    res->n_amb = (long long)hc[1];
    return SHL_OK;
}

// ---------------------------------------------------------------------------
// Solver
// ---------------------------------------------------------------------------

__global__ void pcg_config_kernel(PcgState *st, double tol2, int maxit, int reset) {
    if (threadIdx.x == 0) {
        if (reset) {
            for (int k = 0; k < 6; ++k) {
                st->rz[k] = st->alpha[k] = st->beta[k] = st->rr[k] = st->bnorm2[k] = 0.0;
                st->active[k] = 0;
                st->iters[k] = 0;
            }
            st->nactive = 0;
            st->numeric_err = 0;
            st->ticket_apply = st->ticket_update = st->ticket_aux = 0;
        }
        st->tol2 = tol2;
        st->maxit = maxit;
    }
}

template <typename T>
struct Bufs {
    T *x, *r, *p, *q, *dinv;
};

struct Density {
    const uint8_t *mask;
    const double *rho;
    double E, Ev;
};

template <typename T>
ApplyArgs<T> make_apply(int r, const Density &den, const ElemOp<T> &op) {
    ApplyArgs<T> a{};
    a.r = r;
    a.N = (size_t)r * r * r;
    a.nvec = 6;
    a.case_mask = 0x3f;
    a.mask = den.mask;
    a.rho = den.rho;
    a.E = (T)den.E;
    a.Evoid = (T)den.Ev;
    a.op = op;
    return a;
}

// One PCG iteration recorded as a CUDA graph and replayed: the V-cycle alone
// is ~40 small kernels, whose host launch cost would otherwise dominate.
inline const char *numeric_err_text(int code) {
    switch (code) {
        case kNumErrPq: return "p.q not positive or not finite";
        case kNumErrRz: return "r.z not positive or not finite (preconditioner not SPD)";
        case kNumErrResid: return "recurrence residual not finite";
        case kNumErrInit: return "initial residual not finite";
        case kNumErrRestart: return "true residual at a reliable update not finite";
        default: return "numeric error";
    }
}

struct IterGraph {
    cudaGraphExec_t exec = nullptr;
    bool owned = true;                // false: the context's graph cache owns exec
    unsigned long long launches = 0;  // kernels per replay
    std::function<int()> direct;      // fallback: launch the iteration's kernels
    ~IterGraph() {
        if (exec && owned) cudaGraphExecDestroy(exec);
    }
};

// Records one iteration; if capture or instantiation fails, the iteration is
// replayed by launching its kernels directly (same work, more host time).
// With a key, the instantiated graph is kept in the context and later solves
// of the same shape update it in place with the newly captured parameters
// (instantiated again only if the update is refused).
template <typename F>
inline int capture_iteration(shl_ctx *ctx, cudaStream_t s, IterGraph *g, F &&record, const std::string &key = "") {
    g->direct = [record]() mutable { return record(); };
    const unsigned long long l0 = ctx->launches;
    cudaGraph_t graph = nullptr;
    if (cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
        cudaGetLastError();
        return SHL_OK;
    }
    const int rc = record();
    const cudaError_t e = cudaStreamEndCapture(s, &graph);
    const unsigned long long per_iter = ctx->launches - l0;
    ctx->launches = l0;
    if (e != cudaSuccess || !graph) {
        // capture invalidated (e.g. by another thread's synchronising call):
        // clear the sticky capture error and launch the kernels directly
        if (graph) cudaGraphDestroy(graph);
        cudaGetLastError();
        return SHL_OK;
    }
    if (rc != SHL_OK) {
        cudaGraphDestroy(graph);
        return rc;
    }
    if (!key.empty()) {
        cudaGraphExec_t &cached = ctx->graphs[key];
        if (cached) {
            cudaGraphExecUpdateResultInfo info{};
            if (cudaGraphExecUpdate(cached, graph, &info) != cudaSuccess) {
                cudaGetLastError();
                cudaGraphExecDestroy(cached);
                cached = nullptr;
            }
        }
        if (!cached && cudaGraphInstantiate(&cached, graph, 0) != cudaSuccess) {
            cudaGetLastError();
            cached = nullptr;
        }
        cudaGraphDestroy(graph);
        g->exec = cached;
        g->owned = false;
        g->launches = per_iter;
        return SHL_OK;
    }
    const cudaError_t e2 = cudaGraphInstantiate(&g->exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e2 != cudaSuccess) {
        cudaGetLastError();
        g->exec = nullptr;
        return SHL_OK;
    }
    g->launches = per_iter;
    return SHL_OK;
}

inline int replay(shl_ctx *ctx, cudaStream_t s, IterGraph *g, int times) {
    if (!g->exec) {
        for (int i = 0; i < times; ++i) SHL_TRY(g->direct());
        return SHL_OK;
    }
    for (int i = 0; i < times; ++i) SHL_CUDA(ctx, cudaGraphLaunch(g->exec, s));
    ctx->launches += g->launches * (unsigned long long)times;
    return SHL_OK;
}

// Runs PCG from the residual in b.r and the iterate in b.x for the load cases
// in want.  The device deactivates each case at convergence or st->maxit; the
// host polls the active count every chunk of iterations.
// Vector-kernel launches (vec.cuh): 16-byte chunks when the plane length
// allows, scalar otherwise.
template <typename T>
inline void launch_vec_update(shl_ctx *ctx, const VecArgs<T> &va, const VecGeom &g, const FineJacobi &fj, bool mg,
                              const ApplyDot &ad, cudaStream_t s) {
    constexpr int VW = (int)(16 / sizeof(T));
    pdl_launch(pcg_alpha_kernel, 1, kVecThreads, 0, s, va.st, ad);
    ++ctx->launches;
    if (mg) {  // also writes the first fine pre-smoothing step z = w D^-1 r (FP32)
        if (g.V == VW)
            pdl_launch(vec_update_kernel<T, VW, true>, g.blocks(), kVecThreads, 0, s, va, g, fj);
        else
            pdl_launch(vec_update_kernel<T, 1, true>, g.blocks(), kVecThreads, 0, s, va, g, fj);
        ++ctx->launches;
        return;
    }
    if (g.V == VW)
        pdl_launch(vec_update_kernel<T, VW, false>, g.blocks(), kVecThreads, 0, s, va, g, fj);
    else
        pdl_launch(vec_update_kernel<T, 1, false>, g.blocks(), kVecThreads, 0, s, va, g, fj);
    ++ctx->launches;
}

// Active set: the vector kernels visit only the chunks holding a node with an
// active element (listed in ascending order, so every reduction keeps a fixed
// order).  One host synchronisation (the count), at setup.
inline int active_chunk_list(shl_ctx *ctx, int r, const Density &den, VecGeom *g, cudaStream_t s) {
    const size_t nchunks = g->chunks;
    const int nb = (int)((nchunks + kChunkBlock - 1) / kChunkBlock);
    unsigned *counts = nullptr, *list = nullptr;
    SHL_TRY(ws_get_t(ctx, "active_chunk_counts", (size_t)nb + 1, &counts));
    SHL_TRY(ws_get_t(ctx, "active_chunk_list", nchunks, &list));
    chunk_count_kernel<<<nb, kVecThreads, 0, s>>>(r, g->V, nchunks, den.mask, den.rho, counts);
    chunk_scan_kernel<<<1, 1024, 0, s>>>(nb, counts, counts + nb);
    chunk_write_kernel<<<nb, kVecThreads, 0, s>>>(r, g->V, nchunks, den.mask, den.rho, counts, list);
    ctx->launches += 3;
    unsigned total = 0;
    SHL_CUDA(ctx, cudaMemcpyAsync(&total, counts + nb, sizeof(unsigned), cudaMemcpyDeviceToHost, s));
    SHL_CUDA(ctx, cudaStreamSynchronize(s));
    g->list = list;
    g->chunks = total;
    g->bpk = vec_bpk(total);
    return SHL_OK;
}

// Rows of deferred p.q partials the six-case apply writes.
template <typename T>
inline int apply_partial_rows(int r, const Density &den) {
    return (int)apply_geom<T>(r, 6, den.mask, den.rho).partial_rows(6);
}

template <typename T>
inline void launch_vec_direction(shl_ctx *ctx, const VecArgs<T> &va, const VecGeom &g, cudaStream_t s) {
    constexpr int VW = (int)(16 / sizeof(T));
    if (g.V == VW)
        pdl_launch(vec_direction_kernel<T, VW>, g.blocks(), kVecThreads, 0, s, va, g);
    else
        pdl_launch(vec_direction_kernel<T, 1>, g.blocks(), kVecThreads, 0, s, va, g);
    ++ctx->launches;
}

inline void launch_vec_jacobi_rz(shl_ctx *ctx, const VecArgs<float> &va, const VecGeom &g, const FineJacobi &fj,
                                 const float *t, cudaStream_t s) {
    if (g.V == 4)
        pdl_launch(vec_jacobi_rz_kernel<4>, g.blocks(), kVecThreads, 0, s, va, g, fj, t);
    else
        pdl_launch(vec_jacobi_rz_kernel<1>, g.blocks(), kVecThreads, 0, s, va, g, fj, t);
    ++ctx->launches;
}

template <typename T>
int pcg_run(shl_ctx *ctx, int r, const Density &den, const ElemOp<T> &op, Bufs<T> &b, PcgState *st, int want,
            int set_bnorm, cudaStream_t s, int *host_nactive, int max_iters_backstop) {
    const size_t N = (size_t)r * r * r;
    double *partial = nullptr;
    const int gv = grid1d(N, kBlk, 148 * 4);
    SHL_TRY(ws_get_t(ctx, "pcg_partial", (size_t)gv * 12, &partial));
    VecArgs<T> va{N, b.x, b.r, b.p, b.q, b.dinv, st, partial};
    pcg_init_kernel<T><<<gv, kBlk, 0, s>>>(va, want, set_bnorm);
    ++ctx->launches;
    SHL_CUDA(ctx, cudaGetLastError());
    ApplyArgs<T> a = make_apply<T>(r, den, op);
    a.p = b.p;
    a.q = b.q;
    a.pin = 1;
    a.dot = 1;
    a.defer = 1;  // p.q is reduced by the update kernel
    a.st = st;
    a.ticket = &st->ticket_apply;
    const int chunk = 32;
    {
        const size_t nblk = (size_t)apply_partial_rows<T>(r, den);
        double *ap = nullptr;
        SHL_TRY(ws_get_t(ctx, "apply_partial", nblk * 6, &ap));
        a.partial = ap;
    }
    const VecGeom vg = vec_geom<T>((size_t)r * r * r);
    IterGraph graph;
    SHL_TRY(capture_iteration(ctx, s, &graph, [&]() -> int {
        SHL_TRY(launch_apply<T>(ctx, a, s));
        launch_vec_update<T>(ctx, va, vg, FineJacobi{}, false, ApplyDot{a.partial, apply_partial_rows<T>(r, den)},
                             s);
        launch_vec_direction<T>(ctx, va, vg, s);
        return SHL_OK;
    }, "pcg" + std::to_string(sizeof(T)) + "_" + std::to_string(r)));
    // the device deactivates every load case by st->maxit; the host cap is a backstop
    const long long cap = (long long)max_iters_backstop + 2 * chunk;
    for (long long it = 0;; it += chunk) {
        if (it > cap) return set_err(ctx, SHL_ENOCONV, "PCG did not stop within %lld iterations", cap);
        SHL_TRY(replay(ctx, s, &graph, chunk));
        SHL_CUDA(ctx, cudaMemcpyAsync(host_nactive, &st->nactive, sizeof(int), cudaMemcpyDeviceToHost, s));
        SHL_CUDA(ctx, cudaStreamSynchronize(s));
        if (*host_nactive == 0) break;
    }
    return SHL_OK;
}

struct SolveOut {
    int iters[6] = {0, 0, 0, 0, 0, 0};
    double relres[6] = {0, 0, 0, 0, 0, 0};
    int n_refine = 0;
    int status = SHL_OK;
    int precond = SHL_PRECOND_JACOBI;
};

// Residual f - K x (FP64) with its squared norms per load case; pin selects
// the pinned system; x == nullptr means x = 0 (the loads f themselves).
// out = f - K x (pinned), FP64, for the load cases in mask (others untouched),
// and |out|^2 per computed case into dot_out.
// With opdf the residual is formed in double-float arithmetic (x converted on
// the way in, the result converted back in place): ~3x faster than FP64 on
// B300 and far more accurate than the refinement needs.  The FP64 solver
// keeps FP64.
// With opdf the residual is formed in double-float arithmetic: x is converted
// first (or taken as already converted from xdf_in), and the result is left
// as double-floats in out when out_df, else converted to doubles in place.
inline int resid64(shl_ctx *ctx, int r, const Density &den, const ElemOp<double> &op, const double *x, double *out,
                   int pin, double *dot_out, cudaStream_t s, int mask = 0x3f, const ElemOp<dfloat> *opdf = nullptr,
                   const dfloat *xdf_in = nullptr, bool out_df = false) {
    if (opdf) {
        const size_t N = (size_t)r * r * r;
        dfloat *xdf = const_cast<dfloat *>(xdf_in);
        double *partial = nullptr;
        if (x && !xdf) SHL_TRY(ws_get_t(ctx, "resid_xdf", 18 * N, &xdf));
        const size_t rows = (size_t)((r + kTX - 1) / kTX) * ((r + kTY - 1) / kTY) * apply_zc<dfloat>(r, 6) * 6;
        SHL_TRY(ws_get_t(ctx, "resid_partial", rows * 6, &partial));
        if (x && !xdf_in) {  // x == null: the residual of the zero iterate (the loads)
            to_dfloat_kernel<<<grid1d(N, kBlk, 148 * 8), kBlk, 0, s>>>(N, mask, x, xdf);
            ++ctx->launches;
        }
        ApplyArgs<dfloat> a = make_apply<dfloat>(r, den, *opdf);
        a.case_mask = mask;
        a.p = xdf;
        a.q = reinterpret_cast<dfloat *>(out);
        a.pin = pin;
        a.resid = 1;
        a.dot = 2;
        a.dot_out = dot_out;
        a.partial = partial;
        SHL_TRY(launch_apply<dfloat>(ctx, a, s));
        if (!out_df) {
            dfloat_to_double_kernel<<<grid1d(N, kBlk, 148 * 8), kBlk, 0, s>>>(N, mask, out);
            ++ctx->launches;
        }
        return SHL_OK;
    }
    ApplyArgs<double> a = make_apply<double>(r, den, op);
    a.case_mask = mask;
    a.p = x;
    a.q = out;
    a.pin = pin;
    a.resid = 1;
    a.dot = 2;
    a.dot_out = dot_out;
    return launch_apply<double>(ctx, a, s);
}

struct HostPinned {
    int *nactive = nullptr;
    double *v = nullptr;  // 64 doubles
};

inline int host_pinned(shl_ctx *ctx, HostPinned *hp) {
    static thread_local HostPinned cache;
    if (!cache.nactive) {
        SHL_CUDA(ctx, cudaMallocHost(&cache.nactive, sizeof(int) * 4));
        SHL_CUDA(ctx, cudaMallocHost(&cache.v, sizeof(double) * 64));
    }
    *hp = cache;
    return SHL_OK;
}

// ---------------------------------------------------------------------------
// Multigrid preconditioner (mg.cuh): plan, per-density setup, V-cycle
// ---------------------------------------------------------------------------
// Sweeps per leg on the levels >= 2 take the weights 1 / root_k of the
// Chebyshev polynomial of degree nu_coarse on [b / kMgChebAlpha, b], b =
// kMgChebSafety lambda_max (the power iteration's estimate, from below):
// the error components with eigenvalues of D^-1 A in that range shrink by
// 1 / T_nu((alpha + 1) / (alpha - 1)) (three sweeps: 0.48, against 0.78 for
// three sweeps of the fixed damping 1.6 / lambda_max).  The weights' product
// is a polynomial in D^-1 A, so their order does not matter and the cycle
// stays symmetric.
constexpr int kMgMaxNuCoarse = 64;
constexpr double kMgChebSafety = 1.3, kMgChebAlpha = 20.0;

struct MgLevel {
    int r = 0;
    size_t N = 0;
    float omega = 0.6f;     // damping, 1.2 / lambda_max(D^-1 A) estimated at setup
    float wk[kMgMaxNuCoarse] = {};  // levels >= 2: per-sweep weights (Chebyshev roots)
    float *S = nullptr;     // stencil (levels >= 1)
    float *Dinv = nullptr;  // 3x3 block-Jacobi inverses
    float *x = nullptr, *b = nullptr, *t = nullptr;
    float *xa = nullptr, *xb = nullptr;  // ping-pong iterate buffers (levels >= 1)
    // active set only (null otherwise): node activity, and per group of 32
    // nodes whether one is active (levels run by mg_stencil_nc_kernel)
    uint8_t *act = nullptr, *blk = nullptr;
};

struct Mg {
    int L = 0;  // coarsest level index
    MgLevel lv[kMgMaxLevels];
    float *Y = nullptr, *YT = nullptr;  // coarsest: inverse Cholesky factor and its transpose
    float *w = nullptr;                 // coarsest: Y b, 6 x n3
    int n3 = 0;
    int nu = 2;         // sweeps per leg on levels 0 and 1
    int nu_coarse = 3;  // sweeps per leg on levels >= 2
    int gamma = 1;      // visits of each level >= 2 per visit of the level above
};

// Levels: halve while even and >= 6; usable when the coarsest is small.
inline bool mg_plan(int r, Mg *mg) {
    int rl = r, L = 0;
    while (rl % 2 == 0 && rl >= 6 && L + 1 < kMgMaxLevels) {
        rl /= 2;
        ++L;
    }
    if (L == 0 || (size_t)rl * rl * rl > (size_t)kMgMaxCoarse) return false;
    mg->L = L;
    for (int l = 0, rr = r; l <= L; ++l, rr /= 2) {
        mg->lv[l].r = rr;
        mg->lv[l].N = (size_t)rr * rr * rr;
    }
    return true;
}

// The 8 child matrices for Poisson ratio nu, uploaded into this context's
// workspace on stream s (a per-context copy: concurrent contexts may use
// different nu).
inline int mg_child_matrices(shl_ctx *ctx, double nu, cudaStream_t s, float **out) {
    static thread_local float Mc[8][24][24];
    const double err = build_child_matrices(nu, Mc);
    if (!(err < 1e-12)) return set_err(ctx, SHL_EINVAL, "child matrices do not sum to the coarse element (%g)", err);
    SHL_TRY(ws_get_t(ctx, "mg_childM", (size_t)8 * 24 * 24, out));
    SHL_CUDA(ctx, cudaMemcpyAsync(*out, Mc, sizeof(Mc), cudaMemcpyHostToDevice, s));
    return SHL_OK;
}

// Smallest level (nodes) whose stencil passes run a thread per (node, load
// case); smaller levels run a warp per node.
#ifndef SHL_NC_MIN_NODES
#define SHL_NC_MIN_NODES 32768
#endif
constexpr size_t kStencilNcMinNodes = SHL_NC_MIN_NODES;

// Stencil pass on one coarse level: one thread per (node, load case) with the
// stencils staged in shared memory from 32^3 nodes up (bandwidth and issue
// bound), one warp per node below (latency bound: few nodes, and the warp form
// keeps more loads in flight per node).  The caller counts the launch.
inline void launch_stencil(const MgLevel &L, const float *x, const float *b, float w, int mode, float *out,
                           const PcgState *st, cudaStream_t s) {
    if (L.N >= kStencilNcMinNodes)
        pdl_launch(L.blk ? mg_stencil_nc_kernel<true> : mg_stencil_nc_kernel<false>,
                   (unsigned)((L.N + kStencilNodes - 1) / kStencilNodes), 6 * kStencilNodes, 0, s, L.r,
                   (const float *)L.S, x, b, (const float *)L.Dinv, w, mode, out, st, (const uint8_t *)L.blk);
    else
        pdl_launch(mg_stencil_kernel, grid1d(32 * L.N, kBlk, 148 * 16), kBlk, 0, s, L.r, (const float *)L.S, x, b,
                   (const float *)L.Dinv, w, mode, out, st);
}

inline int mg_setup(shl_ctx *ctx, int r, const Density &den, const shl_solve_opts *o, Mg *mg, cudaStream_t s) {
    float *childM = nullptr;
    SHL_TRY(mg_child_matrices(ctx, o->nu, s, &childM));
    mg->nu = o->mg_nu > 0 ? o->mg_nu : 1;
    // Chebyshev degree on the small levels: 2 at r <= 32 (where those levels are
    // 8^3 and below), 3 above (measured best with 16 designs in flight)
    mg->nu_coarse = o->mg_nu_coarse > 0 ? o->mg_nu_coarse : (r <= 32 ? 2 : 3);
    mg->gamma = o->mg_gamma > 0 ? o->mg_gamma : (r >= 128 ? 2 : 1);
    char nm[64];
    for (int l = 0; l <= mg->L; ++l) {
        MgLevel &L = mg->lv[l];
        snprintf(nm, sizeof(nm), "mg_dinv%d", l);
        SHL_TRY(ws_get_t(ctx, nm, L.N * 9, &L.Dinv));
        snprintf(nm, sizeof(nm), "mg_t%d", l);
        SHL_TRY(ws_get_t(ctx, nm, L.N * 18, &L.t));
        if (l >= 1) {
            snprintf(nm, sizeof(nm), "mg_S%d", l);
            SHL_TRY(ws_get_t(ctx, nm, L.N * 27 * 9, &L.S));
            snprintf(nm, sizeof(nm), "mg_x%d", l);
            SHL_TRY(ws_get_t(ctx, nm, L.N * 18, &L.xa));
            snprintf(nm, sizeof(nm), "mg_y%d", l);
            SHL_TRY(ws_get_t(ctx, nm, L.N * 18, &L.xb));
            L.x = L.xa;
            snprintf(nm, sizeof(nm), "mg_b%d", l);
            SHL_TRY(ws_get_t(ctx, nm, L.N * 18, &L.b));
        }
    }
    // active set: node activity per level, node groups of the streaming stencil passes
    for (int l = 0; l <= mg->L; ++l) mg->lv[l].act = mg->lv[l].blk = nullptr;
    if (den.Ev == 0.0) {
        for (int l = 0; l <= mg->L; ++l) {
            MgLevel &L = mg->lv[l];
            snprintf(nm, sizeof(nm), "mg_act%d", l);
            SHL_TRY(ws_get_t(ctx, nm, L.N, &L.act));
            if (l == 0)
                mg_node_active_fine_kernel<<<grid1d(L.N), kBlk, 0, s>>>(r, den.mask, den.rho, den.E, den.Ev, L.act);
            else
                mg_node_active_coarse_kernel<<<grid1d(L.N), kBlk, 0, s>>>(L.r, mg->lv[l - 1].act, L.act);
            ++ctx->launches;
            if (l >= 1 && L.N >= kStencilNcMinNodes) {
                snprintf(nm, sizeof(nm), "mg_blk%d", l);
                SHL_TRY(ws_get_t(ctx, nm, (L.N + 31) / 32, &L.blk));
                mg_block_active_kernel<<<grid1d((L.N + 31) / 32), kBlk, 0, s>>>(L.N, L.act, L.blk);
                ++ctx->launches;
            }
        }
    }
    // fine block-Jacobi
    double Ku[24][24];
    unit_hex8_stiffness(o->nu, Ku);
    CornerBlocks cb;
    for (int b = 0; b < 8; ++b)
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) cb.K[b][3 * i + j] = (float)(Ku[3 * b + i][3 * b + j] / r);
    mg_dinv_fine_kernel<<<grid1d(mg->lv[0].N), kBlk, 0, s>>>(r, den.mask, den.rho, (float)den.E, (float)den.Ev, cb,
                                                             mg->lv[0].Dinv);
    ++ctx->launches;
    for (int l = 1; l <= mg->L; ++l) {
        MgLevel &L = mg->lv[l];
        const int g = grid1d(L.N * 27, kBlk, 148 * 16);
        const int gc = (int)std::min<size_t>(L.N, 148 * 8);  // coarse-from-coarse: a block per coarse node
        if (l == 1)
            mg_galerkin_fine_kernel<<<g, kBlk, 0, s>>>(L.r, den.mask, den.rho, (float)den.E, (float)den.Ev,
                                                       (float)(1.0 / r), childM, L.S, L.act);
        else if (L.act)
            mg_galerkin_coarse_kernel<true><<<gc, kGalerkinThreads, 0, s>>>(L.r, mg->lv[l - 1].S, L.S,
                                                                           mg->lv[l - 1].act, L.act);
        else
            mg_galerkin_coarse_kernel<false><<<gc, kGalerkinThreads, 0, s>>>(L.r, mg->lv[l - 1].S, L.S, nullptr,
                                                                            nullptr);
        mg_dinv_stencil_kernel<<<grid1d(L.N), kBlk, 0, s>>>(L.N, L.S, L.Dinv, L.act);
        ctx->launches += 2;
    }
    SHL_CUDA(ctx, cudaGetLastError());
    // Page-locked host staging (allocated once per context at its largest
    // size): [coarsest stencil | power-iteration norms | coarse factor upload]
    constexpr int kPow = 15;
    const size_t pin_s = (size_t)kMgMaxCoarse * 243 * sizeof(float);
    const size_t pin_w = (size_t)kMgMaxLevels * kPow * sizeof(double);
    const size_t pin_y = (size_t)2 * (3 * kMgMaxCoarse) * (3 * kMgMaxCoarse) * sizeof(float);
    if (!ctx->pinned) SHL_CUDA(ctx, cudaMallocHost(&ctx->pinned, pin_s + pin_w + pin_y));
    float *hS = static_cast<float *>(ctx->pinned);
    double *hpw = reinterpret_cast<double *>(static_cast<char *>(ctx->pinned) + pin_s);
    float *hY = reinterpret_cast<float *>(static_cast<char *>(ctx->pinned) + pin_s + pin_w);
    // the coarsest stencil goes to the host first; the host assembles and
    // factors the coarse operator while the GPU runs the power iterations
    const MgLevel &C = mg->lv[mg->L];
    const int n3 = (int)(3 * C.N);
    mg->n3 = n3;
    SHL_CUDA(ctx, cudaMemcpyAsync(hS, C.S, C.N * 243 * sizeof(float), cudaMemcpyDeviceToHost, s));
    cudaEvent_t s_ready = nullptr;
    SHL_CUDA(ctx, cudaEventCreateWithFlags(&s_ready, cudaEventDisableTiming));
    SHL_CUDA(ctx, cudaEventRecord(s_ready, s));
    // damping per smoothed level from lambda_max(D^-1 A) (power iteration on
    // one vector, every level enqueued before a single read of the norms)
    {
        ElemOp<float> op32;
        SHL_TRY(get_op(ctx, o->nu, r, &op32));
        double *pw = nullptr, *ppart = nullptr;
        unsigned *ptick = nullptr;
        float *py = nullptr;
        PcgState *pst = nullptr;
        // per level: its own scratch vector, partials and ticket, so that the
        // levels' chains (each a serial run of small, latency-bound launches)
        // run side by side on the context's side streams
        constexpr size_t kPowPart = 148 * 8;
        size_t ny = 0;
        for (int l = 0; l < mg->L; ++l) ny += 3 * mg->lv[l].N;
        SHL_TRY(ws_get_t(ctx, "mg_pow", (size_t)kMgMaxLevels * kPow, &pw));
        SHL_TRY(ws_get_t(ctx, "mg_pow_partial", kPowPart * kMgMaxLevels, &ppart));
        SHL_TRY(ws_get_t(ctx, "mg_pow_ticket", (size_t)kMgMaxLevels, &ptick));
        SHL_TRY(ws_get_t(ctx, "mg_pow_y", ny, &py));
        SHL_TRY(ws_get_t(ctx, "mg_pow_state", 1, &pst));
        float *x0 = nullptr;
        SHL_TRY(ws_get_t(ctx, "z32", 18 * mg->lv[0].N, &x0));
        unsigned *apply_err = nullptr;  // the fine apply's error word exists before the capture
        SHL_TRY(ws_get_t(ctx, "apply_err", 1, &apply_err));
        SHL_TRY(aux_streams(ctx));
        // every level's chain, captured once per grid and density kind (the
        // launches are host-bound: hundreds of short kernels) and replayed
        auto power = [&]() -> int {
        mg_power_state_kernel<<<1, 32, 0, s>>>(pst);
        ++ctx->launches;
        SHL_CUDA(ctx, cudaEventRecord(ctx->aux_ev[shl_ctx::kAux], s));
        size_t yo = 0;
        for (int l = 0; l < mg->L; ++l) {
            MgLevel &L = mg->lv[l];
            const cudaStream_t sl = ctx->aux[l % shl_ctx::kAux];
            if (l < shl_ctx::kAux) SHL_CUDA(ctx, cudaStreamWaitEvent(sl, ctx->aux_ev[shl_ctx::kAux], 0));
            float *x = l == 0 ? x0 : L.x;
            float *yl = py + yo;
            yo += 3 * L.N;
            mg_power_seed_kernel<<<grid1d(3 * L.N), kBlk, 0, sl>>>(L.N, x);
            ++ctx->launches;
            for (int it = 0; it < kPow; ++it) {
                if (l == 0) {
                    ApplyArgs<float> a = make_apply<float>(r, den, op32);
                    a.nvec = 1;
                    a.p = x;
                    a.q = L.t;
                    a.pin = 1;
                    a.err = apply_err;
                    SHL_TRY(launch_apply<float>(ctx, a, sl));
                } else {
                    launch_stencil(L, x, nullptr, 1.0f, 0, L.t, pst, sl);
                    ++ctx->launches;
                }
                const int g = grid1d(L.N, kBlk, (int)kPowPart);
                mg_power_dinv_kernel<<<g, kBlk, 0, sl>>>(L.N, L.t, L.Dinv, yl, ppart + kPowPart * l, ptick + l,
                                                         pw + l * kPow + it);
                mg_power_scale_kernel<<<grid1d(3 * L.N), kBlk, 0, sl>>>(L.N, yl, pw + l * kPow + it, x);
                ctx->launches += 2;
            }
        }
        for (int i = 0; i < std::min(mg->L, shl_ctx::kAux); ++i) {  // join
            SHL_CUDA(ctx, cudaEventRecord(ctx->aux_ev[i], ctx->aux[i]));
            SHL_CUDA(ctx, cudaStreamWaitEvent(s, ctx->aux_ev[i], 0));
        }
        return SHL_OK;
        };
        IterGraph pg;
        // one cached graph per grid, density kind and void model (the active
        // set launches other kernel variants, so the two do not update in place)
        SHL_TRY(capture_iteration(ctx, s, &pg, power,
                                  "mgpow_" + std::to_string(r) + (den.rho ? "_s" : "_m") + (den.Ev == 0.0 ? "_a" : "")));
        SHL_TRY(replay(ctx, s, &pg, 1));
        SHL_CUDA(ctx, cudaMemcpyAsync(hpw, pw, (size_t)mg->L * kPow * sizeof(double), cudaMemcpyDeviceToHost, s));
    }
    // coarsest: dense, coarse node 0 pinned, factored in FP64 on the host
    const cudaError_t se = cudaEventSynchronize(s_ready);
    cudaEventDestroy(s_ready);
    if (se != cudaSuccess) return set_err(ctx, SHL_ECUDA, "coarse stencil copy: %s", cudaGetErrorString(se));
    const float *Sh = hS;
    const int m = n3 - 3;  // pinned: DOFs of node 0 removed
    std::vector<double> A((size_t)m * m, 0.0);
    const int rc = C.r;
    for (size_t I = 0; I < C.N; ++I) {
        const int ix = I % rc, iy = (I / rc) % rc, iz = I / ((size_t)rc * rc);
        for (int dl = 0; dl < 27; ++dl) {
            const int dx = dl % 3 - 1, dy = (dl / 3) % 3 - 1, dz = dl / 9 - 1;
            const size_t J = ((size_t)wrapi(iz + dz, rc) * rc + wrapi(iy + dy, rc)) * rc + wrapi(ix + dx, rc);
            if (I == 0 || J == 0) continue;
            for (int i = 0; i < 3; ++i)
                for (int j = 0; j < 3; ++j)
                    A[(3 * (I - 1) + i) * (size_t)m + 3 * (J - 1) + j] += Sh[(I * 27 + dl) * 9 + 3 * i + j];
        }
    }
    // + eps E A_hom: the all-solid stiffness of the coarsest grid, h_c Khat per
    // element (the Galerkin product of a uniform fine mesh, exact for
    // trilinear elements).  A piece of solid held only by the ersatz void has
    // a mechanism whose stiffness here (~E_void) is below the FP32 rounding of
    // the Galerkin sums; unregularised, the coarse solve amplifies it by ~1e15
    // and CG loses the sign of r.z.  The shift lifts such modes in proportion
    // to their geometric stiffness and leaves the pinned translations alone.
    {
        double Ku[24][24];
        unit_hex8_stiffness(o->nu, Ku);
        const double w = kMgCoarseReg * o->E / rc;
        for (int ez = 0; ez < rc; ++ez)
            for (int ey = 0; ey < rc; ++ey)
                for (int ex = 0; ex < rc; ++ex) {
                    int nd[8];
                    for (int b = 0; b < 8; ++b)
                        nd[b] = ((ez + ((b >> 2) & 1)) % rc * rc + (ey + ((b >> 1) & 1)) % rc) * rc + (ex + (b & 1)) % rc;
                    for (int a = 0; a < 8; ++a) {
                        if (nd[a] == 0) continue;
                        for (int b = 0; b < 8; ++b) {
                            if (nd[b] == 0) continue;
                            for (int i = 0; i < 3; ++i)
                                for (int j = 0; j < 3; ++j)
                                    A[(size_t)(3 * (nd[a] - 1) + i) * m + 3 * (nd[b] - 1) + j] +=
                                        w * Ku[3 * a + i][3 * b + j];
                        }
                    }
                }
    }
    // symmetrise (FP32 stencil rounding), Cholesky, inverse factor Y = L^-1
    for (int i = 0; i < m; ++i)
        for (int j = 0; j < i; ++j)
            A[(size_t)i * m + j] = A[(size_t)j * m + i] = 0.5 * (A[(size_t)i * m + j] + A[(size_t)j * m + i]);
    // A pivot at or below the FP32 rounding level of the stencil sums (a
    // near-rigid mode of a nearly void coarse cell) is raised to that level:
    // L L^T stays SPD whenever L has a positive diagonal, which is all the
    // preconditioner needs.
    double dmax = 0.0;
    for (int j = 0; j < m; ++j) dmax = std::max(dmax, std::fabs(A[(size_t)j * m + j]));
    std::vector<double> Lc((size_t)m * m, 0.0);
    for (int j = 0; j < m; ++j) {
        double d = A[(size_t)j * m + j];
        const double floor_j = 1e-7 * std::max(std::fabs(d), 1e-6 * dmax);
        for (int k = 0; k < j; ++k) d -= Lc[(size_t)j * m + k] * Lc[(size_t)j * m + k];
        if (!std::isfinite(d) || !(floor_j > 0.0))
            return set_err(ctx, SHL_ENUMERIC, "coarsest multigrid operator is not finite");
        if (!(d > floor_j)) d = floor_j;
        const double ljj = std::sqrt(d);
        Lc[(size_t)j * m + j] = ljj;
        for (int i = j + 1; i < m; ++i) {
            double v = A[(size_t)i * m + j];
            for (int k = 0; k < j; ++k) v -= Lc[(size_t)i * m + k] * Lc[(size_t)j * m + k];
            Lc[(size_t)i * m + j] = v / ljj;
        }
    }
    // A^-1 = L^-T L^-1 with Y = L^-1 (lower triangular) by row operations;
    // the V-cycle applies Y^T (Y b), stored in FP32 with node 0's rows and
    // columns zero, plus Y^T row-major for coalesced reads
    std::vector<double> Y((size_t)m * m, 0.0);
    for (int i = 0; i < m; ++i) {  // row i of L Y = I: Y[i][:i+1] = (e_i - sum_k<i L[i][k] Y[k]) / L[i][i]
        double *yi = &Y[(size_t)i * m];
        yi[i] = 1.0;
        for (int k = 0; k < i; ++k) {
            const double lik = Lc[(size_t)i * m + k];
            const double *yk = &Y[(size_t)k * m];
            for (int c = 0; c <= k; ++c) yi[c] -= lik * yk[c];
        }
        const double inv = 1.0 / Lc[(size_t)i * m + i];
        for (int c = 0; c <= i; ++c) yi[c] *= inv;
    }
    float *Yf = hY, *YTf = hY + (size_t)n3 * n3;
    std::memset(hY, 0, sizeof(float) * 2 * (size_t)n3 * n3);
    for (int a = 0; a < m; ++a)
        for (int c = 0; c <= a; ++c) {
            const float v = (float)Y[(size_t)a * m + c];
            Yf[(size_t)(a + 3) * n3 + (c + 3)] = v;
            YTf[(size_t)(c + 3) * n3 + (a + 3)] = v;
        }
    SHL_TRY(ws_get_t(ctx, "mg_Y", (size_t)2 * n3 * n3 + (size_t)6 * n3, &mg->Y));
    mg->YT = mg->Y + (size_t)n3 * n3;
    mg->w = mg->YT + (size_t)n3 * n3;
    SHL_CUDA(ctx, cudaMemcpyAsync(mg->Y, hY, sizeof(float) * 2 * (size_t)n3 * n3, cudaMemcpyHostToDevice, s));
    SHL_CUDA(ctx, cudaStreamSynchronize(s));
    // smoother damping from the power iterations' last Rayleigh estimate
    for (int l = 0; l < mg->L; ++l) {
        const double lam = std::sqrt(hpw[l * kPow + kPow - 1]);
        const double base = o->mg_omega > 0.0 ? o->mg_omega : 1.6;  // omega * lambda_max
        mg->lv[l].omega = (float)(lam > 0.0 && std::isfinite(lam) ? base / lam : 0.3);
        const int m = mg->nu_coarse;
        const double b = kMgChebSafety * lam, a = b / kMgChebAlpha;
        for (int k = 0; k < m && k < kMgMaxNuCoarse; ++k) {
            const double root = 0.5 * (b + a) + 0.5 * (b - a) * std::cos(M_PI * (2 * k + 1) / (2.0 * m));
            mg->lv[l].wk[k] = (float)(lam > 0.0 && std::isfinite(lam) ? 1.0 / root : 0.3);
        }
    }
    return SHL_OK;
}

// z = V-cycle(b) for the pinned fine system; `fine` carries the density and
// operator of the matrix-free apply.  Coarse levels use the fused stencil
// kernel (residual, or a full Jacobi sweep into the other ping-pong buffer).
// Fusion flags of the fine level: the first pre-smoothing step (x0 = w D^-1 b0)
// was done by the caller; the last post-smoothing step is left to the caller
// (on return lv[0].t = K x0 of the current x0).
constexpr int kVcFirstFused = 1, kVcLastExternal = 2;

inline int mg_vcycle(shl_ctx *ctx, Mg *mg, const ApplyArgs<float> &fine, const float *b0, float *x0, PcgState *st,
                     cudaStream_t s, int fuse = 0) {
    auto fine_apply = [&](const float *x, float *t) -> int {
        ApplyArgs<float> a = fine;
        a.p = x;
        a.q = t;
        a.pin = 1;
        a.dot = 0;
        a.resid = 0;
        a.st = st;
        return launch_apply<float>(ctx, a, s);
    };
    // coarse level: mode 1 residual into t, mode 2 a Jacobi sweep with weight wgt (default: the level's damping)
    auto sweep = [&](MgLevel &L, int mode, float wgt = -1.0f) {
        float *out = mode == 1 ? L.t : (L.x == L.xa ? L.xb : L.xa);
        launch_stencil(L, L.x, L.b, wgt > 0.0f ? wgt : L.omega, mode, out, st, s);
        ++ctx->launches;
        if (mode == 2) L.x = out;
    };
    mg->lv[0].b = const_cast<float *>(b0);
    mg->lv[0].x = x0;
    for (int l = 1; l <= mg->L; ++l) mg->lv[l].x = mg->lv[l].xa;
    // restriction into level l + 1; a level that is smoothed (l + 1 < L) also
    // gets its first Jacobi step x = w D^-1 b there
    auto restrict_to = [&](int l, const float *bf, const float *tf) {
        MgLevel &Cl = mg->lv[l + 1];
        if (l + 1 < mg->L)
            pdl_launch(mg_restrict_jacobi_kernel, dim3(grid1d(Cl.N, kBlk, 148), 6), kBlk, 0, s, Cl.r, bf, tf, Cl.b,
                       (const float *)Cl.Dinv, l + 1 >= 2 ? Cl.wk[0] : Cl.omega, Cl.x, st, (const uint8_t *)Cl.act);
        else
            pdl_launch(mg_restrict_kernel, dim3(grid1d(Cl.N, kBlk, 148), 18), kBlk, 0, s, Cl.r, bf, tf, Cl.b, st,
                       (const uint8_t *)Cl.act);
        ++ctx->launches;
    };
    // fine level: pre-smoothing and the restriction of its residual
    {
        MgLevel &L = mg->lv[0];
        const int g = grid1d(L.N);
        if (!(fuse & kVcFirstFused)) {
            pdl_launch(mg_jacobi_kernel, g, kBlk, 0, s, L.N, L.b, nullptr, L.Dinv, L.omega, L.x, 1, st);
            ++ctx->launches;
        }
        for (int it = 1; it < mg->nu; ++it) {
            SHL_TRY(fine_apply(L.x, L.t));
            pdl_launch(mg_jacobi_kernel, g, kBlk, 0, s, L.N, L.b, L.t, L.Dinv, L.omega, L.x, 0, st);
            ++ctx->launches;
        }
        SHL_TRY(fine_apply(L.x, L.t));
        restrict_to(0, L.b, L.t);
    }
    // Coarse levels, recursively: level l's b is set; on the first visit its x
    // holds the restriction's zero-start Jacobi step.  Levels >= 2 are visited
    // gamma times per visit of the level above (V-cycle: 1, W-cycle: 2).
    std::function<void(int, bool)> cycle = [&](int l, bool first) {
        if (l == mg->L) {  // coarsest: x = Y^T (Y b)
            MgLevel &C = mg->lv[mg->L];
            const int g = grid1d((size_t)6 * mg->n3 * 32, kBlk, 148 * 4);
            pdl_launch(mg_dense_y_kernel, g, kBlk, 0, s, mg->n3, (const float *)mg->Y, (const float *)C.b, mg->w, st);
            pdl_launch(mg_dense_yt_kernel, g, kBlk, 0, s, mg->n3, (const float *)mg->YT, (const float *)mg->w, C.x,
                       st);
            ctx->launches += 2;
            return;
        }
        MgLevel &L = mg->lv[l];
        const int nu = l >= 2 ? mg->nu_coarse : mg->nu;
        for (int it = first ? 1 : 0; it < nu; ++it) sweep(L, 2, l >= 2 ? L.wk[it] : -1.0f);
        sweep(L, 1);
        restrict_to(l, L.t, nullptr);
        const int visits = (l + 1 >= 2 && l + 1 < mg->L) ? mg->gamma : 1;
        cycle(l + 1, true);
        for (int v = 1; v < visits; ++v) cycle(l + 1, false);
        pdl_launch(mg_prolong_kernel, dim3(grid1d(mg->lv[l + 1].N, kBlk, 148), 18), kBlk, 0, s, mg->lv[l + 1].r,
                   mg->lv[l + 1].x, L.x, 0, st, (const uint8_t *)mg->lv[l + 1].act);
        ++ctx->launches;
        for (int it = 0; it < nu; ++it) sweep(L, 2, l >= 2 ? L.wk[nu - 1 - it] : -1.0f);
    };
    if (mg->L >= 1) cycle(1, true);
    // fine level: prolongation of the correction and post-smoothing
    {
        MgLevel &L = mg->lv[0];
        const int g = grid1d(L.N);
        pdl_launch(mg_prolong_kernel, dim3(grid1d(mg->lv[1].N, kBlk, 148), 18), kBlk, 0, s, mg->lv[1].r,
                   mg->lv[1].x, L.x, 1, st, (const uint8_t *)mg->lv[1].act);
        ++ctx->launches;
        for (int it = 0; it < mg->nu; ++it) {
            SHL_TRY(fine_apply(L.x, L.t));
            if (it == mg->nu - 1 && (fuse & kVcLastExternal)) break;
            pdl_launch(mg_jacobi_kernel, g, kBlk, 0, s, L.N, L.b, L.t, L.Dinv, L.omega, L.x, 0, st);
            ++ctx->launches;
        }
    }
    SHL_CUDA(ctx, cudaGetLastError());
    return SHL_OK;
}

// FP64 PCG preconditioned by the FP32 multigrid V-cycle (SHL_FP64 with
// SHL_PRECOND_MG): per iteration q = K p and the x, r updates in FP64 (the
// update also takes the V-cycle's first fine smoothing step in FP32), r is
// rounded to FP32 for the V-cycle, the correction z comes back to FP64, and
// r.z, beta and the direction p = z + beta p are FP64.  The V-cycle is a
// fixed symmetric operator, so this is ordinary PCG with an FP32-accurate
// preconditioner; convergence is judged on FP64 residuals.
inline int pcg_run_mg64(shl_ctx *ctx, int r, const Density &den, const ElemOp<double> &op, Bufs<double> &b,
                        PcgState *st, int want, cudaStream_t s, int *host_nactive, int max_iters_backstop, Mg &mg,
                        const ApplyArgs<float> &a32, float *r32, float *z32, double *z64) {
    const size_t N = (size_t)r * r * r;
    double *partial = nullptr;
    const int gv = grid1d(N, kBlk, 148 * 4);
    const int gc = grid1d(18 * N, kBlk, 148 * 8);
    SHL_TRY(ws_get_t(ctx, "pcg_partial", (size_t)gv * 12, &partial));
    VecArgs<double> va{N, b.x, b.r, b.p, b.q, b.dinv, st, partial, z64};
    // start: z = M^-1 r, p = z, rz = r.z for the wanted load cases
    cvt_f64_f32_kernel<<<gc, kBlk, 0, s>>>(N, nullptr, b.r, r32);
    ++ctx->launches;
    SHL_TRY(mg_vcycle(ctx, &mg, a32, r32, z32, nullptr, s));
    cvt_f32_f64_kernel<<<gc, kBlk, 0, s>>>(N, nullptr, z32, z64);
    pcg_init_kernel<double><<<gv, kBlk, 0, s>>>(va, want, 0);
    ctx->launches += 2;
    SHL_CUDA(ctx, cudaGetLastError());
    ApplyArgs<double> a = make_apply<double>(r, den, op);
    a.p = b.p;
    a.q = b.q;
    a.pin = 1;
    a.dot = 1;
    a.defer = 1;  // p.q is reduced by the update kernel
    a.st = st;
    a.ticket = &st->ticket_apply;
    {
        const size_t nblk = (size_t)apply_partial_rows<double>(r, den);
        double *ap = nullptr;
        SHL_TRY(ws_get_t(ctx, "apply_partial", nblk * 6, &ap));
        a.partial = ap;
    }
    const VecGeom vg = vec_geom<double>(N);
    const FineJacobi fj{mg.lv[0].Dinv, mg.lv[0].omega, z32};
    const int chunk = 8;
    IterGraph graph;
    SHL_TRY(capture_iteration(ctx, s, &graph, [&]() -> int {
        SHL_TRY(launch_apply<double>(ctx, a, s));
        launch_vec_update<double>(ctx, va, vg, fj, true, ApplyDot{a.partial, apply_partial_rows<double>(r, den)},
                                  s);
        pdl_launch(cvt_f64_f32_kernel, gc, kBlk, 0, s, N, (const PcgState *)st, (const double *)b.r, r32);
        SHL_TRY(mg_vcycle(ctx, &mg, a32, r32, z32, st, s, kVcFirstFused));
        pdl_launch(cvt_f32_f64_kernel, gc, kBlk, 0, s, N, (const PcgState *)st, (const float *)z32, z64);
        pcg_rz_kernel<double><<<gv, kBlk, 0, s>>>(va);
        pcg_direction_kernel<double><<<gv, kBlk, 0, s>>>(va);
        ctx->launches += 4;
        return SHL_OK;
    }, "pcg64mg_" + std::to_string(r) + (den.Ev == 0.0 ? "_a" : "")));
    const long long cap = (long long)max_iters_backstop + 2 * chunk;
    for (long long it = 0;; it += chunk) {
        if (it > cap) return set_err(ctx, SHL_ENOCONV, "PCG did not stop within %lld iterations", cap);
        SHL_TRY(replay(ctx, s, &graph, chunk));
        SHL_CUDA(ctx, cudaMemcpyAsync(host_nactive, &st->nactive, sizeof(int), cudaMemcpyDeviceToHost, s));
        SHL_CUDA(ctx, cudaStreamSynchronize(s));
        if (*host_nactive == 0) break;
    }
    return SHL_OK;
}

// Full solve: x64 (18 N doubles, device) receives the displacements.
inline int run_solve(shl_ctx *ctx, int r, const Density &den, const shl_solve_opts *o, double *x64, bool warm,
                     cudaStream_t s, SolveOut *out) {
    const size_t N = (size_t)r * r * r;
    const size_t NV = 18 * N;
    HostPinned hp;
    SHL_TRY(host_pinned(ctx, &hp));
    ElemOp<double> op64;
    SHL_TRY(get_op(ctx, o->nu, r, &op64));
    // the FP32 + refinement mode forms its true residuals in double-float
    ElemOp<dfloat> opdf_v;
    const ElemOp<dfloat> *opdf = nullptr;
    if (o->precision == SHL_FP32_REFINE) {
        SHL_TRY(get_op(ctx, o->nu, r, &opdf_v));
        opdf = &opdf_v;
    }
    double *r64 = nullptr, *norms = nullptr;
    SHL_TRY(ws_get_t(ctx, "r64", NV, &r64));
    SHL_TRY(ws_get_t(ctx, "norms", 32, &norms));  // [0:6] |f|^2, [12:18] |f - K x|^2 (pinned system)
    if (!warm) SHL_CUDA(ctx, cudaMemsetAsync(x64, 0, NV * sizeof(double), s));
    // ||f||^2 of the pinned system (r64 = f afterwards)
    SHL_TRY(resid64(ctx, r, den, op64, nullptr, r64, 1, norms + 0, s, 0x3f, opdf));
    double fpin[6];
    SHL_CUDA(ctx, cudaMemcpyAsync(fpin, norms, 6 * sizeof(double), cudaMemcpyDeviceToHost, s));
    SHL_CUDA(ctx, cudaStreamSynchronize(s));
    const double tol = o->tol;
    const int maxit = o->max_iter > 0 ? o->max_iter : 100000;
    int total_it[6] = {0, 0, 0, 0, 0, 0};
    if (o->precision == SHL_FP64) {
        Bufs<double> b{x64, r64, nullptr, nullptr, nullptr};
        SHL_TRY(ws_get_t(ctx, "p64", NV, &b.p));
        SHL_TRY(ws_get_t(ctx, "q64", NV, &b.q));
        SHL_TRY(ws_get_t(ctx, "dinv64", N, &b.dinv));
        dinv_kernel<double><<<grid1d(N), kBlk, 0, s>>>(r, den.mask, den.rho, den.E, den.Ev, op64.diag, b.dinv);
        ++ctx->launches;
        PcgState *st = nullptr;
        SHL_TRY(ws_get_t(ctx, "pcg_state64", 1, &st));
        pcg_config_kernel<<<1, 32, 0, s>>>(st, tol * tol, maxit, 1);
        ++ctx->launches;
        SHL_CUDA(ctx, cudaMemcpyAsync(st->bnorm2, norms, 6 * sizeof(double), cudaMemcpyDeviceToDevice, s));
        if (warm) SHL_TRY(resid64(ctx, r, den, op64, x64, r64, 1, nullptr, s));
        // multigrid preconditioner in FP32 (when asked and the grid coarsens far enough)
        Mg mg;
        const bool use_mg = (o->precond == SHL_PRECOND_MG) && mg_plan(r, &mg);
        ElemOp<float> op32;
        float *r32 = nullptr, *z32 = nullptr;
        double *z64 = nullptr;
        if (use_mg) {
            SHL_TRY(get_op(ctx, o->nu, r, &op32));
            SHL_TRY(ws_get_t(ctx, "r32", NV, &r32));
            SHL_TRY(ws_get_t(ctx, "z32", NV, &z32));
            SHL_TRY(ws_get_t(ctx, "z64", NV, &z64));
            SHL_TRY(mg_setup(ctx, r, den, o, &mg, s));
        }
        const ApplyArgs<float> a32 = use_mg ? make_apply<float>(r, den, op32) : ApplyArgs<float>{};
        out->precond = use_mg ? SHL_PRECOND_MG : SHL_PRECOND_JACOBI;
        // CG stops on its recurrence residual, which drifts from f - K x in
        // finite precision; restart from the true residual until it meets tol.
        int want = 0x3f, restarts = 0;
        for (;; ++restarts) {
            if (use_mg)
                SHL_TRY(pcg_run_mg64(ctx, r, den, op64, b, st, want, s, hp.nactive, maxit, mg, a32, r32, z32, z64));
            else
                SHL_TRY(pcg_run<double>(ctx, r, den, op64, b, st, want, 0, s, hp.nactive, maxit));
            int its[6], nerr = 0;
            SHL_CUDA(ctx, cudaMemcpyAsync(its, st->iters, sizeof(its), cudaMemcpyDeviceToHost, s));
            SHL_CUDA(ctx, cudaMemcpyAsync(&nerr, &st->numeric_err, sizeof(int), cudaMemcpyDeviceToHost, s));
            SHL_TRY(resid64(ctx, r, den, op64, x64, r64, 1, norms + 12, s));
            SHL_CUDA(ctx, cudaMemcpyAsync(hp.v, norms + 12, 6 * sizeof(double), cudaMemcpyDeviceToHost, s));
            SHL_CUDA(ctx, cudaStreamSynchronize(s));
            for (int k = 0; k < 6; ++k)
                if ((want >> k) & 1) total_it[k] += its[k];
            if (nerr) {
                out->status = SHL_ENUMERIC;
                set_err(ctx, SHL_ENUMERIC, "FP64 PCG stopped: %s", numeric_err_text(nerr));
                break;
            }
            want = 0;
            for (int k = 0; k < 6; ++k)
                if (fpin[k] > 0.0 && hp.v[k] > tol * tol * fpin[k] && total_it[k] < maxit) want |= 1 << k;
            if (!want || restarts >= 20) break;
        }
        out->n_refine = restarts;
    } else if (o->precision == SHL_FP32_REFINE) {
        ElemOp<float> op32;
        SHL_TRY(get_op(ctx, o->nu, r, &op32));
        Bufs<float> b{};
        SHL_TRY(ws_get_t(ctx, "x32", NV, &b.x));
        SHL_TRY(ws_get_t(ctx, "r32", NV, &b.r));
        SHL_TRY(ws_get_t(ctx, "p32", NV, &b.p));
        SHL_TRY(ws_get_t(ctx, "q32", NV, &b.q));
        SHL_TRY(ws_get_t(ctx, "dinv32", N, &b.dinv));
        dinv_kernel<float><<<grid1d(N), kBlk, 0, s>>>(r, den.mask, den.rho, den.E, den.Ev, op64.diag, b.dinv);
        ++ctx->launches;
        PcgState *st = nullptr;
        SHL_TRY(ws_get_t(ctx, "pcg_state32", 1, &st));
        double *one = nullptr;
        SHL_TRY(ws_get_t(ctx, "refine_scale", 8, &one));
        const double h_one[8] = {1, 1, 1, 1, 1, 1, 1, 1};
        SHL_CUDA(ctx, cudaMemcpyAsync(one, h_one, sizeof(h_one), cudaMemcpyHostToDevice, s));
        const double delta = o->inner_tol > 0.0 ? o->inner_tol : 1e-4;
        // r64 = f - K x64 (pinned; already f, with |f|^2, for a cold start);
        // r32 = float(r64); x32 = 0
        if (warm)
            SHL_TRY(resid64(ctx, r, den, op64, x64, r64, 1, norms + 12, s, 0x3f, opdf));
        else
            SHL_CUDA(ctx, cudaMemcpyAsync(norms + 12, norms, 6 * sizeof(double), cudaMemcpyDeviceToDevice, s));
        refine_scatter_kernel<<<grid1d(N), kBlk, 0, s>>>(N, r64, one, 0x3f, b.r, b.x);
        ++ctx->launches;
        pcg_config_kernel<<<1, 32, 0, s>>>(st, tol * tol, maxit, 1);
        ++ctx->launches;
        SHL_CUDA(ctx, cudaMemcpyAsync(st->bnorm2, norms, 6 * sizeof(double), cudaMemcpyDeviceToDevice, s));
        SHL_CUDA(ctx, cudaMemcpyAsync(hp.v, norms + 12, 6 * sizeof(double), cudaMemcpyDeviceToHost, s));
        SHL_CUDA(ctx, cudaStreamSynchronize(s));
        double last_rr[6];
        for (int k = 0; k < 6; ++k) last_rr[k] = hp.v[k];
        // PCG with reliable updates (one pcg_run per interval between updates)
        const double *rr_true = norms + 12;
        int want = 0;
        for (int k = 0; k < 6; ++k)
            if (fpin[k] > 0.0 && last_rr[k] > tol * tol * fpin[k]) want |= 1 << k;
        int updates = 0;
        if (want) {
            const size_t gv = grid1d(N, kBlk, 148 * 4);
            double *partial = nullptr;
            SHL_TRY(ws_get_t(ctx, "pcg_partial", (size_t)gv * 12, &partial));
            // multigrid preconditioner (when the grid coarsens far enough)
            Mg mg;
            const bool use_mg = (o->precond == SHL_PRECOND_MG) && mg_plan(r, &mg);
            dfloat *xdf = nullptr;  // x64 as double-floats, written by the fold for the true residual
            SHL_TRY(ws_get_t(ctx, "resid_xdf", 18 * N, &xdf));
            float *z32 = nullptr;
            PcgState *vc_state = nullptr;  // gates the reliable update's V-cycle to the updated load cases
            if (use_mg) {
                SHL_TRY(ws_get_t(ctx, "z32", NV, &z32));
                SHL_TRY(ws_get_t(ctx, "mg_vc_state", 1, &vc_state));
                SHL_TRY(mg_setup(ctx, r, den, o, &mg, s));
            }
            out->precond = use_mg ? SHL_PRECOND_MG : SHL_PRECOND_JACOBI;
            VecArgs<float> va{N, b.x, b.r, b.p, b.q, b.dinv, st, partial, z32};
            ApplyArgs<float> a = make_apply<float>(r, den, op32);
            if (use_mg) SHL_TRY(mg_vcycle(ctx, &mg, a, b.r, z32, nullptr, s));
            pcg_init_kernel<float><<<gv, kBlk, 0, s>>>(va, want, 0);
            ++ctx->launches;
            a.p = b.p;
            a.q = b.q;
            a.pin = 1;
            a.dot = 1;
            a.defer = 1;  // p.q is reduced by the update kernel
            a.st = st;
            a.ticket = &st->ticket_apply;
            const int chunk = use_mg ? 8 : 32;
            // workspaces the iteration uses must exist before capture
            {
                const size_t nblk = (size_t)apply_partial_rows<float>(r, den);
                double *ap = nullptr;
                SHL_TRY(ws_get_t(ctx, "apply_partial", nblk * 6, &ap));
                a.partial = ap;
            }
            // one iteration: q = K p (+ p.q -> alpha); x, r update (+ r.r, and
            // the first fine pre-smoothing step z = w D^-1 r); V-cycle; last
            // fine post-smoothing step (+ r.z -> beta); p = z + beta p
            VecGeom vg = vec_geom<float>(N);
            if (o->active && vg.V > 1) SHL_TRY(active_chunk_list(ctx, r, den, &vg, s));
            FineJacobi fj{};
            if (use_mg) fj = FineJacobi{mg.lv[0].Dinv, mg.lv[0].omega, z32};
            auto iteration = [&]() -> int {
                SHL_TRY(launch_apply<float>(ctx, a, s));
                launch_vec_update<float>(ctx, va, vg, fj, use_mg, ApplyDot{a.partial, apply_partial_rows<float>(r, den)},
                                         s);
                if (use_mg) {
                    SHL_TRY(mg_vcycle(ctx, &mg, a, b.r, z32, st, s, kVcFirstFused | kVcLastExternal));
                    launch_vec_jacobi_rz(ctx, va, vg, fj, mg.lv[0].t, s);
                }
                launch_vec_direction<float>(ctx, va, vg, s);
                return SHL_OK;
            };
            IterGraph graph;
            SHL_TRY(capture_iteration(ctx, s, &graph, iteration,
                                      "pcg32_" + std::to_string(r) + (use_mg ? "_mg" : "_jacobi") +
                                          (den.Ev == 0.0 ? "_a" : "")));
            PcgState hst;
            for (long long it = 0;; it += chunk) {
                if (it > (long long)maxit + 2 * chunk)
                    return set_err(ctx, SHL_ENOCONV, "PCG did not stop within %d iterations", maxit);
                SHL_TRY(replay(ctx, s, &graph, chunk));
                SHL_CUDA(ctx, cudaMemcpyAsync(&hst, st, sizeof(PcgState), cudaMemcpyDeviceToHost, s));
                SHL_CUDA(ctx, cudaStreamSynchronize(s));
                if (hst.numeric_err) {
                    out->status = SHL_ENUMERIC;
                    int itmax = 0;
                    for (int k = 0; k < 6; ++k) itmax = std::max(itmax, hst.iters[k]);
                    set_err(ctx, SHL_ENUMERIC, "%s PCG stopped at iteration %d: %s",
                            use_mg ? "multigrid-preconditioned" : "Jacobi-preconditioned", itmax,
                            numeric_err_text(hst.numeric_err));
                    break;
                }
                // want: load cases not yet verified converged by their FP64 residual
                int mask = 0, restart = 0;
                for (int k = 0; k < 6; ++k)
                    if ((want >> k) & 1) {
                        const bool stopped = !hst.active[k];
                        if (stopped || hst.rr[k] <= delta * delta * last_rr[k]) mask |= 1 << k;
                        if (stopped) restart |= 1 << k;
                    }
                if (mask) {
                    ++updates;
                    // fold x32 into x64 (also as double-floats), the true residual left as double-floats
                    reliable_fold_kernel<<<grid1d(N), kBlk, 0, s>>>(N, b.x, x64, mask, xdf);
                    ++ctx->launches;
                    SHL_TRY(resid64(ctx, r, den, op64, x64, r64, 1, norms + 12, s, mask, opdf, xdf, true));
                    reliable_rebase_kernel<<<gv, kBlk, 0, s>>>(va, nullptr, reinterpret_cast<const dfloat *>(r64),
                                                               mask, restart, rr_true);
                    ++ctx->launches;
                    if (use_mg) {  // direction restarts from the preconditioned true residual
                        mg_mask_state_kernel<<<1, 32, 0, s>>>(vc_state, mask);
                        ++ctx->launches;
                        SHL_TRY(mg_vcycle(ctx, &mg, a, b.r, z32, vc_state, s));
                        pcg_restart_z_kernel<float><<<gv, kBlk, 0, s>>>(va, mask);
                        ++ctx->launches;
                    }
                    SHL_CUDA(ctx, cudaMemcpyAsync(&hst, st, sizeof(PcgState), cudaMemcpyDeviceToHost, s));
                    SHL_CUDA(ctx, cudaMemcpyAsync(hp.v, norms + 12, 6 * sizeof(double), cudaMemcpyDeviceToHost, s));
                    SHL_CUDA(ctx, cudaStreamSynchronize(s));
                    for (int k = 0; k < 6; ++k)
                        if ((mask >> k) & 1) {
                            last_rr[k] = hp.v[k];
                            if (!hst.active[k]) want &= ~(1 << k);  // converged (or out of iterations)
                        }
                }
                if (hst.nactive == 0 && !want) break;
            }
            for (int k = 0; k < 6; ++k) total_it[k] = hst.iters[k];
        }
        out->n_refine = updates;
    } else {
        return set_err(ctx, SHL_EINVAL, "unknown precision mode %d", o->precision);
    }
    for (int k = 0; k < 6; ++k) out->iters[k] = total_it[k];
    // true residual of the pinned system, FP64.  Both modes end with it
    // already in norms[12..17] for the final iterate (the FP64 restart loop
    // computes it every pass; in FP32 + refinement each load case stops at a
    // reliable update, after which its FP64 iterate no longer changes), so an
    // FP64 apply is spent here only after a numeric breakdown.
    if (out->status == SHL_ENUMERIC) SHL_TRY(resid64(ctx, r, den, op64, x64, r64, 1, norms + 12, s, 0x3f, opdf));
    double hn[24];
    SHL_CUDA(ctx, cudaMemcpyAsync(hn, norms, sizeof(hn), cudaMemcpyDeviceToHost, s));
    unsigned *aerr = nullptr, haerr = 0;
    SHL_TRY(ws_get_t(ctx, "apply_err", 1, &aerr));
    SHL_CUDA(ctx, cudaMemcpyAsync(&haerr, aerr, sizeof(unsigned), cudaMemcpyDeviceToHost, s));
    SHL_CUDA(ctx, cudaStreamSynchronize(s));
    if (haerr) {
        SHL_CUDA(ctx, cudaMemsetAsync(aerr, 0, sizeof(unsigned), s));
        return set_err(ctx, SHL_ECUDA, "stiffness apply: a bulk row copy did not complete in time (error bits %#x)",
                       haerr);
    }
    for (int k = 0; k < 6; ++k) {
        out->relres[k] = hn[k] > 0.0 ? std::sqrt(hn[12 + k] / hn[k]) : std::sqrt(hn[12 + k]);
        if (!std::isfinite(out->relres[k]))
            out->status = SHL_ENUMERIC;
        else if (out->status == SHL_OK && out->relres[k] > tol)
            out->status = SHL_ENOCONV;
    }
    return SHL_OK;
}

// C^H from the displacements u (FP64).  With df the element energies are
// summed in double-float arithmetic (the FP32 + refinement mode), else in FP64.
inline int run_chom(shl_ctx *ctx, int r, const Density &den, double nu, const double *u, double *C_dev,
                    cudaStream_t s, bool df = false) {
    const size_t N = (size_t)r * r * r;
    const int g = grid1d(N, kChomThreads, 148 * 8);
    const int gdf = (int)std::min<size_t>((N + kChomDfElems - 1) / kChomDfElems, 148 * 6);
    double *partial = nullptr;
    unsigned *ticket = nullptr;
    SHL_TRY(ws_get_t(ctx, "chom_partial", (size_t)std::max(g, gdf) * 21, &partial));
    SHL_TRY(ws_get_t(ctx, "chom_ticket", 1, &ticket));
    if (df) {
        ElemOp<dfloat> opd;
        SHL_TRY(get_op(ctx, nu, r, &opd));
        dfloat *udf = nullptr;
        SHL_TRY(ws_get_t(ctx, "resid_xdf", 18 * N, &udf));
        to_dfloat_kernel<<<grid1d(18 * N, kBlk, 148 * 8), kBlk, 0, s>>>(N, 0x3f, u, udf);
        ChomDfArgs a{};
        a.r = r;
        a.N = N;
        a.u = udf;
        a.mask = den.mask;
        a.rho = den.rho;
        a.E = den.E;
        a.Evoid = den.Ev;
        a.partial = partial;
        a.ticket = ticket;
        a.C = C_dev;
        a.op = opd;
        chom_df_kernel<<<gdf, kChomDfThreads, 0, s>>>(a);
        ctx->launches += 2;
        SHL_CUDA(ctx, cudaGetLastError());
        return SHL_OK;
    }
    ElemOp<double> op;
    SHL_TRY(get_op(ctx, nu, r, &op));
    ChomArgs a{};
    a.r = r;
    a.N = N;
    a.u = u;
    a.mask = den.mask;
    a.rho = den.rho;
    a.E = den.E;
    a.Evoid = den.Ev;
    a.partial = partial;
    a.ticket = ticket;
    a.C = C_dev;
    a.op = op;
    const size_t smem = sizeof(double) * 6 * 24 * kChomThreads;
    raise_smem_limit((const void *)chom_kernel, smem);
    chom_kernel<<<g, kChomThreads, smem, s>>>(a);
    ++ctx->launches;
    SHL_CUDA(ctx, cudaGetLastError());
    return SHL_OK;
}

inline int validate_solve_opts(shl_ctx *ctx, const shl_solve_opts *o) {
    if (!o) return set_err(ctx, SHL_EINVAL, "solve options are NULL");
    if (!(o->E > 0.0) || !(o->E_void >= 0.0) || !(o->E_void < o->E))
        return set_err(ctx, SHL_EINVAL, "moduli must satisfy 0 <= E_void < E");
    if (!(o->nu > -1.0 && o->nu < 0.5)) return set_err(ctx, SHL_EINVAL, "Poisson ratio %g outside (-1, 0.5)", o->nu);
    if (!(o->tol > 0.0 && o->tol < 1.0)) return set_err(ctx, SHL_EINVAL, "tol %g outside (0, 1)", o->tol);
    if (o->precision != SHL_FP64 && o->precision != SHL_FP32_REFINE)
        return set_err(ctx, SHL_EINVAL, "unknown precision %d", o->precision);
    if (o->density != SHL_MASK && o->density != SHL_SMOOTH)
        return set_err(ctx, SHL_EINVAL, "unknown density mode %d", o->density);
    if (o->precond != SHL_PRECOND_JACOBI && o->precond != SHL_PRECOND_MG)
        return set_err(ctx, SHL_EINVAL, "unknown preconditioner %d", o->precond);
    if (!(o->mg_omega <= 0.0 || o->mg_omega < 2.0))
        return set_err(ctx, SHL_EINVAL, "mg_omega (damping times lambda_max) must be < 2");
    if (o->mg_nu > 64 || o->mg_nu_coarse > 64)
        return set_err(ctx, SHL_EINVAL, "mg_nu %d / mg_nu_coarse %d above 64 sweeps", o->mg_nu, o->mg_nu_coarse);
    if (o->mg_gamma < 0 || o->mg_gamma > 2) return set_err(ctx, SHL_EINVAL, "mg_gamma %d not 0, 1 or 2", o->mg_gamma);
    if (o->active != 0 && o->active != 1) return set_err(ctx, SHL_EINVAL, "active must be 0 or 1, got %d", o->active);
    if (o->active && !(o->cull < 1.0)) return set_err(ctx, SHL_EINVAL, "cull threshold %g must be < 1", o->cull);
    return SHL_OK;
}

// Solve + C^H for a given density on stream s (caller validated the arguments
// and holds the context lock).  u_dev: displacements (in: initial guess when
// warm; out: solution), or null for a context workspace.
inline int solve_impl(shl_ctx *ctx, int r, const uint8_t *mask_dev, const double *rho_dev, const shl_solve_opts *o,
                      double *u_dev, bool warm, double *C_out, shl_stats *st, cudaStream_t s) {
    const size_t NV = (size_t)18 * r * r * r;
    double *x64 = u_dev;
    if (!x64) SHL_TRY(ws_get_t(ctx, "x64", NV, &x64));
    Density den{mask_dev, rho_dev, o->E, o->E_void};
    if (o->active) {
        // active set (Sec. 4.2.1): no ersatz floor, culled elements carry no
        // stiffness (a mask is its own active set); nodes left with a zero
        // diagonal get zero (block) inverses and so never change
        den.Ev = 0.0;
        if (rho_dev) {
            const size_t N = (size_t)r * r * r;
            double *rc = nullptr;
            SHL_TRY(ws_get_t(ctx, "rho_active", N, &rc));
            cull_rho_kernel<<<grid1d(N), kBlk, 0, s>>>(N, rho_dev, o->cull > 0.0 ? o->cull : 1e-3, rc);
            ++ctx->launches;
            den.rho = rc;
        }
    }
    SolveOut so;
    cudaEvent_t e0, e1, e2;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    cudaEventCreate(&e2);
    cudaEventRecord(e0, s);
    int rc = run_solve(ctx, r, den, o, x64, warm, s, &so);
    if ((rc == SHL_OK && so.status == SHL_ENUMERIC && so.precond == SHL_PRECOND_MG) ||
        (rc == SHL_ENUMERIC && o->precond == SHL_PRECOND_MG)) {
        // multigrid setup or the multigrid-preconditioned CG broke down:
        // solve again with point Jacobi
        shl_solve_opts oj = *o;
        oj.precond = SHL_PRECOND_JACOBI;
        so = SolveOut();
        rc = run_solve(ctx, r, den, &oj, x64, false, s, &so);
    }
    cudaEventRecord(e1, s);
    double *Cd = nullptr;
    if (rc == SHL_OK) rc = ws_get_t(ctx, "chom_out", 36, &Cd);
    if (rc == SHL_OK) rc = run_chom(ctx, r, den, o->nu, x64, Cd, s, o->precision == SHL_FP32_REFINE);
    cudaEventRecord(e2, s);
    if (rc == SHL_OK && C_out) cudaMemcpyAsync(C_out, Cd, 36 * sizeof(double), cudaMemcpyDeviceToHost, s);
    cudaStreamSynchronize(s);
    if (st) {
        for (int k = 0; k < 6; ++k) {
            st->iters[k] = so.iters[k];
            st->relres[k] = so.relres[k];
        }
        st->n_refine = so.n_refine;
        st->precond = so.precond;
        st->status = rc != SHL_OK ? rc : so.status;
        cudaEventElapsedTime(&st->ms_solve, e0, e1);
        cudaEventElapsedTime(&st->ms_chom, e1, e2);
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaEventDestroy(e2);
    if (rc != SHL_OK) return rc;
    if (so.status == SHL_ENUMERIC) return set_err(ctx, SHL_ENUMERIC, "solve broke down: %s", ctx->err.c_str());
    if (so.status == SHL_ENOCONV) return set_err(ctx, SHL_ENOCONV, "a load case did not reach tol");
    return SHL_OK;
}

// The whole path for one design on stream s (arguments validated, lock held).
inline int homogenize_impl(shl_ctx *ctx, const shl_design *d, int r, const shl_solve_opts *o, double *C_out,
                           shl_stats *st, cudaStream_t s, double *x64, bool warm) {
    uint8_t *mask = nullptr;
    double *rho = nullptr;
    const size_t N = (size_t)r * r * r;
    SHL_TRY(ws_get_t(ctx, "hom_mask", N, &mask));
    if (o->density == SHL_SMOOTH) SHL_TRY(ws_get_t(ctx, "hom_rho", N, &rho));
    if (st) std::memset(st, 0, sizeof(*st));
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    cudaEventRecord(e0, s);
    VoxOut v;
    int rc = run_voxelize(ctx, d, r, o->kappa, mask, rho, nullptr, s, &v);
    cudaEventRecord(e1, s);
    if (rc == SHL_OK)
        rc = solve_impl(ctx, r, o->density == SHL_SMOOTH ? nullptr : mask, rho, o, x64, warm, C_out, st, s);
    if (st) {
        cudaEventElapsedTime(&st->ms_field, e0, e1);
        st->t = v.t;
        st->margin = v.margin;
        st->n_solid = v.n_solid;
        st->n_ambiguous = v.n_amb;
        if (rc != SHL_OK && st->status == SHL_OK) st->status = rc;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return rc;
}

// Device workspace bytes a design of grid r needs (admission estimate).
inline size_t design_footprint(int r, const shl_solve_opts *o) {
    const size_t N = (size_t)r * r * r;
    size_t per = 144 + 144 + 8 + 1 + 8;  // x64, r64, distances, mask, dinv
    per += (o->precision == SHL_FP64) ? 144 + 144 : 4 * 72;
    if (o->density == SHL_SMOOTH) per += 8;
    return N * per + ((size_t)8 << 20);
}

// Gradient of an objective E(C^H, V) with dE/dC^H = dEdC (host, 36) and
// dE/dV = dEdV, V the mean smoothed occupancy, w.r.t. charge
// positions/magnitudes, iso-level, half-thickness and alpha (Eq. chain),
// through the smoothed density.  Arguments validated, lock held.
inline int grad_impl(shl_ctx *ctx, const shl_design *d, int r, const shl_solve_opts *o, const double *dEdC,
                     double dEdV, double *u_dev, double *C_out, double *g_pos, double *g_q, double *g_iso,
                     double *g_t, double *g_alpha, double *V_out, shl_stats *st, cudaStream_t s) {
    const size_t N = (size_t)r * r * r;
    const int nb = 2 * d->K + 1;
    double *F = nullptr, *gF = nullptr, *dd = nullptr, *rho = nullptr, *g = nullptr, *QR = nullptr, *Abar = nullptr,
           *Gd = nullptr, *gout = nullptr, *partial = nullptr;
    unsigned *ticket = nullptr;
    SHL_TRY(ws_get_t(ctx, "adj_F", N, &F));
    SHL_TRY(ws_get_t(ctx, "adj_gF", 3 * N, &gF));
    SHL_TRY(ws_get_t(ctx, "adj_d", N, &dd));
    SHL_TRY(ws_get_t(ctx, "adj_rho", N, &rho));
    SHL_TRY(ws_get_t(ctx, "adj_g", N, &g));
    SHL_TRY(ws_get_t(ctx, "adj_QR", (size_t)r * 2 * nb * nb, &QR));
    SHL_TRY(ws_get_t(ctx, "adj_Abar", (size_t)nb * nb * nb, &Abar));
    SHL_TRY(ws_get_t(ctx, "adj_small", 64, &Gd));
    gout = Gd + 40;
    if (st) std::memset(st, 0, sizeof(*st));
    // forward: distances, t (held fixed), smoothed density, F and grad F
    VoxOut v;
    SHL_TRY(run_voxelize(ctx, d, r, o->kappa, nullptr, rho, dd, s, &v));
    const double kappa = o->kappa > 0.0 ? o->kappa : std::log(9.0) * r;
    SHL_TRY(run_field(ctx, d, r, F, gF, nullptr, s));
    // six cell problems and C^H
    const size_t NV = 18 * N;
    double *x64 = u_dev;
    if (!x64) SHL_TRY(ws_get_t(ctx, "adj_x64", NV, &x64));
    int rc = solve_impl(ctx, r, nullptr, rho, o, x64, o->warm_start && u_dev, C_out, st, s);
    if (st) {
        st->t = v.t;
        st->margin = v.margin;
        st->n_solid = v.n_solid;
        st->n_ambiguous = v.n_amb;
    }
    if (rc != SHL_OK && rc != SHL_ENOCONV) return rc;
    // element sensitivities g_e = dE/drho_e
    SHL_CUDA(ctx, cudaMemcpyAsync(Gd, dEdC, 36 * sizeof(double), cudaMemcpyHostToDevice, s));
    {
        ElemOp<double> op;
        SHL_TRY(get_op(ctx, o->nu, r, &op));
        ChomArgs a{};
        a.r = r;
        a.N = N;
        a.u = x64;
        a.rho = rho;
        a.E = o->E;
        a.Evoid = o->E_void;
        a.G = Gd;
        a.g = g;
        a.op = op;
        const size_t smem = sizeof(double) * 6 * 24 * kChomThreads;
        raise_smem_limit((const void *)chom_kernel, smem);
        chom_kernel<<<grid1d(N, kChomThreads, 148 * 8), kChomThreads, smem, s>>>(a);
        ++ctx->launches;
    }
    // seeds for F, grad F; dE/dt, dE/dc
    const int gs = grid1d(N, kBlk, 148 * 4);
    SHL_TRY(ws_get_t(ctx, "adj_partial", (size_t)gs * 3, &partial));
    SHL_TRY(ws_get_t(ctx, "adj_ticket", 1, &ticket));
    SeedArgs sa{N, F, gF, rho, g, dEdV / (double)N, d->iso, kappa, partial, ticket, gout};
    adj_seed_kernel<<<gs, kBlk, 0, s>>>(sa);
    ++ctx->launches;
    // back through the separable field to the coefficient tensor and the charges
    const size_t smp = sizeof(double) * ((size_t)r * nb + (size_t)r * 3 * nb);
    raise_smem_limit((const void *)adj_plane_kernel, smp);
    adj_plane_kernel<<<r, 256, smp, s>>>(r, d->K, F, gF, QR);
    const size_t smc = sizeof(double) * (size_t)r * nb;
    raise_smem_limit((const void *)adj_coef_kernel, smc);
    adj_coef_kernel<<<1, 512, smc, s>>>(r, d->K, QR, Abar);
    Uploaded up;
    SHL_TRY(upload_design(ctx, d, s, &up, "grad"));
    double *gp = nullptr;
    const int na = (d->K + 1) * (d->K + 1) * (d->K + 1);
    SHL_TRY(ws_get_t(ctx, "adj_gcharges", (size_t)4 * d->n + na, &gp));
    adj_charge_kernel<<<(d->n + 127) / 128, 128, 0, s>>>(d->n, d->K, up.pos, up.q, up.alpha, Abar, gp, gp + 3 * d->n);
    ctx->launches += 3;
    if (g_alpha) {
        adj_alpha_kernel<<<1, 256, 0, s>>>(d->n, d->K, up.pos, up.q, Abar, gp + 4 * d->n);
        ++ctx->launches;
    }
    SHL_CUDA(ctx, cudaGetLastError());
    std::vector<double> hg((size_t)4 * d->n + na);
    double ho[3];
    SHL_CUDA(ctx, cudaMemcpyAsync(hg.data(), gp, hg.size() * sizeof(double), cudaMemcpyDeviceToHost, s));
    SHL_CUDA(ctx, cudaMemcpyAsync(ho, gout, 3 * sizeof(double), cudaMemcpyDeviceToHost, s));
    SHL_CUDA(ctx, cudaStreamSynchronize(s));
    if (g_pos) std::memcpy(g_pos, hg.data(), sizeof(double) * 3 * d->n);
    if (g_q) std::memcpy(g_q, hg.data() + 3 * d->n, sizeof(double) * d->n);
    if (g_alpha) std::memcpy(g_alpha, hg.data() + 4 * d->n, sizeof(double) * na);
    if (g_t) *g_t = ho[0];
    if (g_iso) *g_iso = ho[1];
    if (V_out) *V_out = ho[2];
    return rc;
}

}  // namespace shl

#include "serve.cuh"

namespace shl {
// serving slots count toward the owning context's telemetry
inline void serve_counters(shl_ctx *ctx, shl_counters *out) {
    auto *sv = static_cast<Server *>(ctx->serve);
    if (!sv) return;
    std::lock_guard<std::mutex> lk(sv->mu);
    for (auto *w : sv->slot_ctx) {
        out->kernel_launches += w->launches;
        out->workspace_bytes += ctx_ws_bytes(w);
    }
    out->workspace_bytes += sv->warm_bytes;
}
}  // namespace shl

// ===========================================================================
// C-ABI
// ===========================================================================
extern "C" {

void shl_default_solve_opts(shl_solve_opts *o) {
    if (!o) return;
    std::memset(o, 0, sizeof(*o));
    o->E = 1.0;
    o->nu = 0.3;
    o->E_void = 1e-6;
    o->tol = 1e-10;
    o->max_iter = 100000;
    o->precision = SHL_FP64;
    o->density = SHL_MASK;
    o->kappa = 0.0;
    o->inner_tol = 1e-4;
    o->precond = SHL_PRECOND_MG;
    o->mg_nu = 1;
    o->mg_nu_coarse = 0;  // 2 at r <= 32, else 3
    o->mg_gamma = 0;
    o->mg_omega = 1.6;
    o->active = 0;
    o->cull = 1e-3;
}

int shl_create(const shl_opts *opts, shl_ctx **out) {
    if (!out) return set_err(nullptr, SHL_EINVAL, "out is NULL");
    *out = nullptr;
    int dev = opts ? opts->device : 0;
    int ndev = 0;
    cudaError_t e = cudaGetDeviceCount(&ndev);
    if (e != cudaSuccess || ndev == 0) {
        cudaGetLastError();
        return set_err(nullptr, SHL_ECUDA, "no CUDA device: %s", cudaGetErrorString(e));
    }
    if (dev < 0 || dev >= ndev) return set_err(nullptr, SHL_EINVAL, "device %d out of range", dev);
    e = cudaSetDevice(dev);
    if (e != cudaSuccess) return set_err(nullptr, SHL_ECUDA, "cudaSetDevice: %s", cudaGetErrorString(e));
    shl_ctx *c = new shl_ctx();
    c->device = dev;
    if (opts) c->opts = *opts;
    e = cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
        delete c;
        return set_err(nullptr, SHL_ECUDA, "cudaStreamCreate: %s", cudaGetErrorString(e));
    }
    *out = c;
    return SHL_OK;
}

int shl_destroy(shl_ctx *ctx) {
    if (!ctx) return SHL_OK;
    cudaSetDevice(ctx->device);
    serve_stop(ctx);
    cudaStreamSynchronize(ctx->stream);
    aux_release(ctx);
    ws_free_all(ctx);
    cudaStreamDestroy(ctx->stream);
    delete ctx;
    return SHL_OK;
}

const char *shl_last_error(shl_ctx *ctx) { return ctx ? ctx->err.c_str() : global_err().msg.c_str(); }

int shl_field(shl_ctx *ctx, const shl_design *d, int32_t r, double *F_dev, double *gradF_dev, void *stream) {
    if (!ctx) return set_err(nullptr, SHL_EINVAL, "ctx is NULL");
    std::lock_guard<std::recursive_mutex> lk(ctx->mu);
    if (!d) return set_err(ctx, SHL_EINVAL, "design is NULL");
    shl_design dd = *d;
    if (!(dd.t > 0.0)) dd.t = 1.0;  // no shell needed for the field alone
    SHL_TRY(validate_design(ctx, &dd, r));
    if (!F_dev) return set_err(ctx, SHL_EINVAL, "F_dev is NULL");
    cudaSetDevice(ctx->device);
    return run_field(ctx, d, r, F_dev, gradF_dev, nullptr, pick_stream(ctx, stream));
}

int shl_voxelize(shl_ctx *ctx, const shl_design *d, int32_t r, double kappa, uint8_t *mask_dev, double *rho_dev,
                 double *d_dev, double *t_out, double *margin_out, int64_t *n_solid, int64_t *n_ambiguous,
                 void *stream) {
    if (!ctx) return set_err(nullptr, SHL_EINVAL, "ctx is NULL");
    std::lock_guard<std::recursive_mutex> lk(ctx->mu);
    SHL_TRY(validate_design(ctx, d, r));
    cudaSetDevice(ctx->device);
    VoxOut v;
    SHL_TRY(run_voxelize(ctx, d, r, kappa, mask_dev, rho_dev, d_dev, pick_stream(ctx, stream), &v));
    if (t_out) *t_out = v.t;
    if (margin_out) *margin_out = v.margin;
    if (n_solid) *n_solid = v.n_solid;
    if (n_ambiguous) *n_ambiguous = v.n_amb;
    return SHL_OK;
}

int shl_apply(shl_ctx *ctx, int32_t r, const uint8_t *mask_dev, const double *rho_dev, double E, double nu,
              double E_void, int32_t precision, int32_t nvec, const void *p_dev, void *q_dev, void *stream) {
    if (!ctx) return set_err(nullptr, SHL_EINVAL, "ctx is NULL");
    std::lock_guard<std::recursive_mutex> lk(ctx->mu);
    if (r < 1 || r > 1024) return set_err(ctx, SHL_EINVAL, "grid size r=%d out of range [1, 1024]", r);
    if (nvec < 1 || nvec > 6) return set_err(ctx, SHL_EINVAL, "nvec=%d out of range [1, 6]", nvec);
    if (!p_dev || !q_dev || (!mask_dev && !rho_dev)) return set_err(ctx, SHL_EINVAL, "NULL buffer");
    if (!(nu > -1.0 && nu < 0.5)) return set_err(ctx, SHL_EINVAL, "Poisson ratio %g outside (-1, 0.5)", nu);
    cudaSetDevice(ctx->device);
    Density den{mask_dev, rho_dev, E, E_void};
    cudaStream_t s = pick_stream(ctx, stream);
    if (precision == SHL_FP64) {
        ElemOp<double> op;
        SHL_TRY(get_op(ctx, nu, r, &op));
        ApplyArgs<double> a = make_apply<double>(r, den, op);
        a.nvec = nvec;
        a.p = static_cast<const double *>(p_dev);
        a.q = static_cast<double *>(q_dev);
        return launch_apply<double>(ctx, a, s);
    } else if (precision == SHL_FP32_REFINE) {
        ElemOp<float> op;
        SHL_TRY(get_op(ctx, nu, r, &op));
        ApplyArgs<float> a = make_apply<float>(r, den, op);
        a.nvec = nvec;
        a.p = static_cast<const float *>(p_dev);
        a.q = static_cast<float *>(q_dev);
        return launch_apply<float>(ctx, a, s);
    }
    return set_err(ctx, SHL_EINVAL, "unknown precision %d", precision);
}

int shl_rhs(shl_ctx *ctx, int32_t r, const uint8_t *mask_dev, const double *rho_dev, double E, double nu,
            double E_void, double *f_dev, void *stream) {
    if (!ctx) return set_err(nullptr, SHL_EINVAL, "ctx is NULL");
    std::lock_guard<std::recursive_mutex> lk(ctx->mu);
    if (r < 1 || r > 1024) return set_err(ctx, SHL_EINVAL, "grid size r=%d out of range [1, 1024]", r);
    if (!f_dev || (!mask_dev && !rho_dev)) return set_err(ctx, SHL_EINVAL, "NULL buffer");
    cudaSetDevice(ctx->device);
    ElemOp<double> op;
    SHL_TRY(get_op(ctx, nu, r, &op));
    const size_t N = (size_t)r * r * r;
    rhs_kernel<<<grid1d(N), kBlk, 0, pick_stream(ctx, stream)>>>(r, mask_dev, rho_dev, E, E_void, op, f_dev);
    ++ctx->launches;
    SHL_CUDA(ctx, cudaGetLastError());
    return SHL_OK;
}

int shl_chom(shl_ctx *ctx, int32_t r, const uint8_t *mask_dev, const double *rho_dev, double E, double nu,
             double E_void, const double *u_dev, double *C_out, void *stream) {
    if (!ctx) return set_err(nullptr, SHL_EINVAL, "ctx is NULL");
    std::lock_guard<std::recursive_mutex> lk(ctx->mu);
    if (r < 1 || r > 1024) return set_err(ctx, SHL_EINVAL, "grid size r=%d out of range [1, 1024]", r);
    if (!u_dev || !C_out || (!mask_dev && !rho_dev)) return set_err(ctx, SHL_EINVAL, "NULL buffer");
    cudaSetDevice(ctx->device);
    cudaStream_t s = pick_stream(ctx, stream);
    double *Cd = nullptr;
    SHL_TRY(ws_get_t(ctx, "chom_out", 36, &Cd));
    Density den{mask_dev, rho_dev, E, E_void};
    SHL_TRY(run_chom(ctx, r, den, nu, u_dev, Cd, s));
    SHL_CUDA(ctx, cudaMemcpyAsync(C_out, Cd, 36 * sizeof(double), cudaMemcpyDeviceToHost, s));
    SHL_CUDA(ctx, cudaStreamSynchronize(s));
    return SHL_OK;
}

int shl_solve(shl_ctx *ctx, int32_t r, const uint8_t *mask_dev, const double *rho_dev, const shl_solve_opts *o,
              double *u_dev, double *C_out, shl_stats *st, void *stream) {
    if (!ctx) return set_err(nullptr, SHL_EINVAL, "ctx is NULL");
    std::lock_guard<std::recursive_mutex> lk(ctx->mu);
    SHL_TRY(validate_solve_opts(ctx, o));
    if (r < 2 || r > 1024) return set_err(ctx, SHL_EINVAL, "grid size r=%d out of range [2, 1024]", r);
    if (!mask_dev && !rho_dev) return set_err(ctx, SHL_EINVAL, "no density given");
    cudaSetDevice(ctx->device);
    if (st) std::memset(st, 0, sizeof(*st));
    return solve_impl(ctx, r, mask_dev, rho_dev, o, u_dev, o->warm_start && u_dev, C_out, st, pick_stream(ctx, stream));
}

int shl_homogenize(shl_ctx *ctx, const shl_design *d, int32_t r, const shl_solve_opts *o, double *C_out,
                   shl_stats *st, void *stream) {
    if (!ctx) return set_err(nullptr, SHL_EINVAL, "ctx is NULL");
    std::lock_guard<std::recursive_mutex> lk(ctx->mu);
    SHL_TRY(validate_solve_opts(ctx, o));
    SHL_TRY(validate_design(ctx, d, r));
    if (!C_out) return set_err(ctx, SHL_EINVAL, "C_out is NULL");
    cudaSetDevice(ctx->device);
    return homogenize_impl(ctx, d, r, o, C_out, st, pick_stream(ctx, stream), nullptr, false);
}

int shl_grad(shl_ctx *ctx, const shl_design *d, int32_t r, const shl_solve_opts *o, const double *dE_dC,
             double dE_dV, double *u_dev, double *C_out, double *g_pos, double *g_q, double *g_iso, double *g_t,
             double *g_alpha, double *V_out, shl_stats *st, void *stream) {
    if (!ctx) return set_err(nullptr, SHL_EINVAL, "ctx is NULL");
    std::lock_guard<std::recursive_mutex> lk(ctx->mu);
    SHL_TRY(validate_solve_opts(ctx, o));
    SHL_TRY(validate_design(ctx, d, r));
    if (o->density != SHL_SMOOTH)
        return set_err(ctx, SHL_EINVAL, "shl_grad needs the smooth density (the binary mask has no derivative)");
    if (o->active)
        return set_err(ctx, SHL_EINVAL, "shl_grad differentiates the ersatz-void problem; active = 1 is forward only");
    if (!dE_dC) return set_err(ctx, SHL_EINVAL, "dE_dC is NULL");
    for (int i = 0; i < 36; ++i)
        if (!std::isfinite(dE_dC[i])) return set_err(ctx, SHL_EINVAL, "non-finite dE_dC");
    if (!std::isfinite(dE_dV)) return set_err(ctx, SHL_EINVAL, "non-finite dE_dV");
    cudaSetDevice(ctx->device);
    return grad_impl(ctx, d, r, o, dE_dC, dE_dV, u_dev, C_out, g_pos, g_q, g_iso, g_t, g_alpha, V_out, st,
                     pick_stream(ctx, stream));
}

// The designs of a batch run concurrently on the serving slots (each a
// private context with its own stream and workspaces), so that one design's
// latency-bound phases (small coarse-grid kernels, host reads of convergence
// flags) overlap with the others' bandwidth-bound applies.
int shl_homogenize_batch(shl_ctx *ctx, int32_t n, const shl_design *d, const int32_t *r, const shl_solve_opts *o,
                         double *C_out, shl_stats *st, void *stream) {
    if (!ctx) return set_err(nullptr, SHL_EINVAL, "ctx is NULL");
    if (n < 0 || (n > 0 && (!d || !r || !C_out))) return set_err(ctx, SHL_EINVAL, "bad batch arguments");
    if (n == 0) return SHL_OK;
    SHL_TRY(validate_solve_opts(ctx, o));
    for (int i = 0; i < n; ++i) SHL_TRY(validate_design(ctx, d + i, r[i]));
    if (n == 1) return shl_homogenize(ctx, d, r[0], o, C_out, st, stream);
    cudaSetDevice(ctx->device);
    cudaStream_t cs = pick_stream(ctx, stream);
    Server *sv = nullptr;
    {
        std::lock_guard<std::recursive_mutex> lk(ctx->mu);
        SHL_TRY(serve_start(ctx, &sv));
    }
    for (int i = 0; i < n; ++i)
        if (design_footprint(r[i], o) > sv->budget)
            return set_err(ctx, SHL_EINVAL, "batch: design %d footprint exceeds the HBM budget %zu", i, sv->budget);
    cudaEvent_t entry = nullptr;
    SHL_CUDA(ctx, cudaEventCreateWithFlags(&entry, cudaEventDisableTiming));
    std::vector<cudaEvent_t> fin(n, nullptr);
    std::vector<uint64_t> tk(n, 0);
    int err = cudaEventRecord(entry, cs) == cudaSuccess ? SHL_OK : set_err(ctx, SHL_ECUDA, "batch: event record failed");
    int submitted = 0;
    for (int i = 0; i < n && err == SHL_OK; ++i) {
        if (cudaEventCreateWithFlags(&fin[i], cudaEventDisableTiming) != cudaSuccess) {
            err = set_err(ctx, SHL_ECUDA, "batch: event create failed");
            break;
        }
        shl_request req{};
        req.design = d[i];
        req.r = r[i];
        req.opts = *o;
        req.session = -1;
        err = serve_enqueue(ctx, &req, entry, fin[i], &tk[i]);
        if (err == SHL_OK) ++submitted;
    }
    int worst = SHL_OK;
    for (int i = 0; i < submitted; ++i) {
        shl_result res{};
        const int rc = serve_take(ctx, tk[i], &res, true);
        if (rc != SHL_OK) {
            if (err == SHL_OK) err = rc;
            continue;
        }
        std::memcpy(C_out + 36 * i, res.C, sizeof(res.C));
        if (st) st[i] = res.stats;
        const int s = res.stats.status;
        if (s == SHL_ENOCONV && worst == SHL_OK) worst = s;
        if (s != SHL_OK && s != SHL_ENOCONV && err == SHL_OK)
            err = set_err(ctx, s, "batch: design %d failed: %s", i, ctx->err.c_str());
        if (cudaStreamWaitEvent(cs, fin[i], 0) != cudaSuccess && err == SHL_OK)
            err = set_err(ctx, SHL_ECUDA, "batch: stream wait failed");
    }
    for (auto e : fin)
        if (e) cudaEventDestroy(e);
    cudaEventDestroy(entry);
    return err != SHL_OK ? err : worst;
}

int shl_probe_peaks(shl_ctx *ctx, shl_peaks *out) {
    if (!ctx || !out) return set_err(ctx, SHL_EINVAL, "NULL argument");
    std::lock_guard<std::recursive_mutex> lk(ctx->mu);
    cudaSetDevice(ctx->device);
    cudaStream_t s = ctx->stream;
    int nsm = 0;
    SHL_CUDA(ctx, cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, ctx->device));
    const int threads = 512, blocks = nsm * 4;
    float *buf = nullptr;
    SHL_TRY(ws_get_t(ctx, "probe_out", (size_t)threads * blocks, &buf));
    cudaEvent_t e0, e1;
    SHL_CUDA(ctx, cudaEventCreate(&e0));
    SHL_CUDA(ctx, cudaEventCreate(&e1));
    // flop/s = threads x blocks x iters x chains x (2 per FMA, 4 per packed FMA) / seconds
    auto timed = [&](int kind, int iters, double flops_per_fma) -> double {
        for (int rep = 0; rep < 2; ++rep) {  // the first launch warms up, the second is timed
            cudaEventRecord(e0, s);
            if (kind == 0) probe_ffma_kernel<<<blocks, threads, 0, s>>>(iters, 0.999f, 1e-3f, buf);
            if (kind == 1) probe_ffma2_kernel<<<blocks, threads, 0, s>>>(iters, 0.999f, 1e-3f, buf);
            if (kind == 2) probe_dfma_kernel<<<blocks, threads, 0, s>>>(iters, 0.999, 1e-3, buf);
            cudaEventRecord(e1, s);
        }
        ctx->launches += 2;
        cudaEventSynchronize(e1);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        return (double)threads * blocks * iters * kProbeChains * flops_per_fma / (ms * 1e-3) / 1e9;
    };
    out->fp32_fma_gflops = timed(0, 4096, 2.0);
    out->fp32x2_fma_gflops = timed(1, 4096, 4.0);
    out->fp64_fma_gflops = timed(2, 256, 2.0);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    SHL_CUDA(ctx, cudaGetLastError());
    return SHL_OK;
}

int shl_probe_wait_timeout(shl_ctx *ctx, uint32_t polls, int32_t *timed_out) {
    if (!ctx || !timed_out) return set_err(ctx, SHL_EINVAL, "NULL argument");
    if (polls < 1 || polls > (1u << 20)) return set_err(ctx, SHL_EINVAL, "polls %u outside [1, 2^20]", polls);
    std::lock_guard<std::recursive_mutex> lk(ctx->mu);
    cudaSetDevice(ctx->device);
    cudaStream_t s = ctx->stream;
    unsigned *err = nullptr;
    SHL_TRY(ws_get_t(ctx, "probe_err", 1, &err));
    SHL_CUDA(ctx, cudaMemsetAsync(err, 0, sizeof(unsigned), s));
    probe_wait_timeout_kernel<<<1, 32, 0, s>>>(polls, err);
    ++ctx->launches;
    SHL_CUDA(ctx, cudaGetLastError());
    unsigned h = 0;
    SHL_CUDA(ctx, cudaMemcpyAsync(&h, err, sizeof(unsigned), cudaMemcpyDeviceToHost, s));
    SHL_CUDA(ctx, cudaStreamSynchronize(s));
    *timed_out = (h & kApplyErrWaitTimeout) ? 1 : 0;
    return SHL_OK;
}

int shl_get_counters(shl_ctx *ctx, shl_counters *out) {
    if (!ctx || !out) return set_err(ctx, SHL_EINVAL, "NULL argument");
    std::lock_guard<std::recursive_mutex> lk(ctx->mu);
    out->kernel_launches = ctx->launches;
    uint64_t b = 0;
    for (auto &kv : ctx->ws.slots) b += kv.second.second;
    out->workspace_bytes = b;
    serve_counters(ctx, out);
    return SHL_OK;
}

}  // extern "C"

// ===========================================================================
// Allocation-free C^H reduction (shl_chom_noalloc)
//
// For callers that must not allocate device memory: code that runs inside
// another framework's memory pool or a real-time loop where cudaMalloc can
// stall or is forbidden.  The reduction's scratch (last-block ticket and
// per-block partial sums) lives in the file-scope array below instead of a
// context workspace; the caller passes only inputs and the 36-double output.
// ===========================================================================
namespace shl {

constexpr int kNoAllocMaxBlocks = 148 * 8;           // grid cap of the C^H kernel
constexpr size_t kNoAllocScratchBytes = 256 * 1024;  // held by every GPU that loads the library
constexpr int kNoAllocMaxR = 512;
static_assert(256 + sizeof(double) * 21 * kNoAllocMaxBlocks <= kNoAllocScratchBytes, "scratch too small");

// [0, 256): reduction ticket; [256, ...): per-block partial sums (21 doubles each).
static __device__ __align__(256) unsigned char g_chom_scratch[kNoAllocScratchBytes];

// Device address of g_chom_scratch, looked up once per device.  In host code
// the array's name is only a host-side stand-in, so kernels must be given this
// address instead.
static std::mutex g_noalloc_mu;
static unsigned char *g_noalloc_ptr[64];

static int noalloc_scratch(int dev, unsigned char **out) {
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (dev < 0 || dev >= 64) return set_err(nullptr, SHL_EINVAL, "device ordinal %d out of range [0, 64)", dev);
    if (!g_noalloc_ptr[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_chom_scratch);
        if (e != cudaSuccess || !p)
            return set_err(nullptr, SHL_ECUDA, "cudaGetSymbolAddress(scratch) failed: %s", cudaGetErrorString(e));
        g_noalloc_ptr[dev] = static_cast<unsigned char *>(p);
    }
    *out = g_noalloc_ptr[dev];
    return SHL_OK;
}

}  // namespace shl

extern "C" int shl_chom_noalloc(int32_t r, const uint8_t *mask_dev, const double *rho_dev, double E, double nu,
                                double E_void, const double *u_dev, double *C_dev, void *stream) {
    if (r < 1 || r > kNoAllocMaxR)
        return set_err(nullptr, SHL_EINVAL, "shl_chom_noalloc: grid size r=%d outside [1, %d]", r, kNoAllocMaxR);
    if (!u_dev || !C_dev || (!mask_dev && !rho_dev))
        return set_err(nullptr, SHL_EINVAL, "shl_chom_noalloc: NULL buffer");
    if (!(nu > -1.0 && nu < 0.5)) return set_err(nullptr, SHL_EINVAL, "Poisson ratio %g outside (-1, 0.5)", nu);
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return set_err(nullptr, SHL_ECUDA, "cudaGetDevice: %s", cudaGetErrorString(e));
    // the kernel runs on the current device: buffers of another device (or
    // host memory) would be read and written through the wrong address space
    const void *bufs[4] = {u_dev, C_dev, mask_dev, rho_dev};
    const char *names[4] = {"u_dev", "C_dev", "mask_dev", "rho_dev"};
    for (int i = 0; i < 4; ++i) {
        if (!bufs[i]) continue;
        cudaPointerAttributes at{};
        e = cudaPointerGetAttributes(&at, bufs[i]);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return set_err(nullptr, SHL_EINVAL, "shl_chom_noalloc: %s is not a CUDA pointer (%s)", names[i],
                           cudaGetErrorString(e));
        }
        if (at.type != cudaMemoryTypeDevice && at.type != cudaMemoryTypeManaged)
            return set_err(nullptr, SHL_EINVAL, "shl_chom_noalloc: %s is not device memory", names[i]);
        if (at.device != dev)
            return set_err(nullptr, SHL_EINVAL, "shl_chom_noalloc: %s is on device %d, the current device is %d",
                           names[i], at.device, dev);
    }
    unsigned char *scratch = nullptr;
    SHL_TRY(noalloc_scratch(dev, &scratch));
    ElemOp<double> op;
    SHL_TRY(get_op(nullptr, nu, r, &op));
    const size_t N = (size_t)r * r * r;
    const int g = grid1d(N, kChomThreads, kNoAllocMaxBlocks);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    ChomArgs a{};
    a.r = r;
    a.N = N;
    a.u = u_dev;
    a.mask = mask_dev;
    a.rho = rho_dev;
    a.E = E;
    a.Evoid = E_void;
    a.ticket = reinterpret_cast<unsigned *>(scratch);
    a.partial = reinterpret_cast<double *>(scratch + 256);
    a.C = C_dev;
    a.op = op;
    // the ticket must start at zero; the partials are fully overwritten
    SHL_CUDA(nullptr, cudaMemsetAsync(a.ticket, 0, sizeof(unsigned), s));
    const size_t smem = sizeof(double) * 6 * 24 * kChomThreads;
    raise_smem_limit((const void *)chom_kernel, smem);
    chom_kernel<<<g, kChomThreads, smem, s>>>(a);
    SHL_CUDA(nullptr, cudaGetLastError());
    return SHL_OK;
}
