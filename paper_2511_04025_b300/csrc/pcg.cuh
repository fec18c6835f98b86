// pcg.cuh -- batched 6-RHS Jacobi-preconditioned conjugate gradients with
// device-resident scalars, per-load-case convergence and skip (Sec. 4.2.2:
// all six right-hand sides in the same kernels, per-RHS residual tracking,
// converged RHS skip their updates), plus the precision-refinement helpers.
#pragma once

#include "apply.cuh"

namespace shl {

template <typename T>
struct VecArgs {
    size_t N;
    T *x, *r, *p;
    const T *q;
    const T *dinv;  // point-Jacobi inverse diagonal (Jacobi mode)
    PcgState *st;
    double *partial;
    const T *z;     // preconditioned residual M^-1 r (multigrid mode; null for Jacobi)
};

// x += alpha p ; r -= alpha q ; z = D^-1 r ; partial (r.z, r.r)
// Last block: convergence test, beta, active flags.
template <typename T>
__global__ void pcg_update_kernel(VecArgs<T> a) {
    PcgState *st = a.st;
    if (st->nactive == 0) return;
    bool act[6];
    T al[6];
#pragma unroll
    for (int k = 0; k < 6; ++k) {
        act[k] = st->active[k] != 0;
        al[k] = (T)st->alpha[k];
    }
    DotAcc<T> dacc[12];
    const size_t N = a.N;
    // the vectors never alias: lets the loads of all planes be issued together
    T *__restrict__ x = a.x;
    T *__restrict__ rv_ = a.r;
    const T *__restrict__ p = a.p;
    const T *__restrict__ q = a.q;
    const T *__restrict__ dinv = a.dinv;
    const bool zmode = a.z != nullptr;
    for (size_t n = blockIdx.x * (size_t)blockDim.x + threadIdx.x; n < N; n += (size_t)gridDim.x * blockDim.x) {
        const T di = zmode ? T(0) : dinv[n];
#pragma unroll
        for (int k = 0; k < 6; ++k) {
            if (!act[k]) continue;
#pragma unroll
            for (int i = 0; i < 3; ++i) {
                const size_t o = (size_t)(3 * k + i) * N + n;
                const T pv = p[o], qv = q[o];
                x[o] += al[k] * pv;
                const T rv = rv_[o] - al[k] * qv;
                rv_[o] = rv;
                if (!zmode) dacc[k].add(rv * (di * rv));
                dacc[6 + k].add(rv * rv);
            }
        }
    }
    double acc[12];
#pragma unroll
    for (int k = 0; k < 12; ++k) acc[k] = dacc[k].get();
    const unsigned nb = gridDim.x;
    block_reduce_store<12>(acc, a.partial, blockIdx.x);
    if (!last_block_ticket(&st->ticket_update, nb)) return;
    __shared__ double tot[12];
    sum_partials_ordered<12>(a.partial, nb, tot);
    if (threadIdx.x == 0) {
        int na = 0;
        for (int k = 0; k < 6; ++k) {
            if (!act[k]) continue;
            st->iters[k] += 1;
            const double rz = tot[k], rr = tot[6 + k];
            st->rr[k] = rr;
            if (!isfinite(rz) || !isfinite(rr)) {
                st->numeric_err = kNumErrResid;
                st->active[k] = 0;
            } else if (rr <= st->tol2 * st->bnorm2[k]) {
                st->active[k] = 0;
            } else if (st->iters[k] >= st->maxit) {
                st->active[k] = 0;
            } else if (!a.z) {
                st->beta[k] = rz / st->rz[k];
                st->rz[k] = rz;
            }
        }
        for (int k = 0; k < 6; ++k) na += st->active[k];
        st->nactive = na;
    }
}

// Multigrid mode: rz = r . z after the V-cycle; beta = rz_new / rz_old.
template <typename T>
__global__ void pcg_rz_kernel(VecArgs<T> a) {
    PcgState *st = a.st;
    if (st->nactive == 0) return;
    bool act[6];
#pragma unroll
    for (int k = 0; k < 6; ++k) act[k] = st->active[k] != 0;
    DotAcc<T> dacc[6];
    const size_t N = a.N;
    for (size_t n = blockIdx.x * (size_t)blockDim.x + threadIdx.x; n < N; n += (size_t)gridDim.x * blockDim.x) {
#pragma unroll
        for (int k = 0; k < 6; ++k) {
            if (!act[k]) continue;
#pragma unroll
            for (int i = 0; i < 3; ++i) {
                const size_t o = (size_t)(3 * k + i) * N + n;
                dacc[k].add(__ldg(a.r + o) * __ldg(a.z + o));
            }
        }
    }
    double acc[6];
#pragma unroll
    for (int k = 0; k < 6; ++k) acc[k] = dacc[k].get();
    block_reduce_store<6>(acc, a.partial, blockIdx.x);
    if (!last_block_ticket(&st->ticket_aux, gridDim.x)) return;
    __shared__ double tot[6];
    sum_partials_ordered<6>(a.partial, gridDim.x, tot);
    if (threadIdx.x == 0) {
        for (int k = 0; k < 6; ++k) {
            if (!act[k]) continue;
            if (!isfinite(tot[k]) || !(tot[k] > 0.0)) {
                st->numeric_err = kNumErrRz;
                st->active[k] = 0;
                continue;
            }
            st->beta[k] = tot[k] / st->rz[k];
            st->rz[k] = tot[k];
        }
        int na = 0;
        for (int k = 0; k < 6; ++k) na += st->active[k];
        st->nactive = na;
    }
}

// Multigrid mode, (re)start of the direction for the load cases in mask:
// p = z, rz = r . z.
template <typename T>
__global__ void pcg_restart_z_kernel(VecArgs<T> a, int mask) {
    PcgState *st = a.st;
    DotAcc<T> dacc[6];
    const size_t N = a.N;
    for (size_t n = blockIdx.x * (size_t)blockDim.x + threadIdx.x; n < N; n += (size_t)gridDim.x * blockDim.x) {
#pragma unroll
        for (int k = 0; k < 6; ++k) {
            if (!((mask >> k) & 1)) continue;
#pragma unroll
            for (int i = 0; i < 3; ++i) {
                const size_t o = (size_t)(3 * k + i) * N + n;
                const T zv = a.z[o];
                a.p[o] = zv;
                dacc[k].add(a.r[o] * zv);
            }
        }
    }
    double acc[6];
#pragma unroll
    for (int k = 0; k < 6; ++k) acc[k] = dacc[k].get();
    block_reduce_store<6>(acc, a.partial, blockIdx.x);
    if (!last_block_ticket(&st->ticket_aux, gridDim.x)) return;
    __shared__ double tot[6];
    sum_partials_ordered<6>(a.partial, gridDim.x, tot);
    if (threadIdx.x == 0)
        for (int k = 0; k < 6; ++k)
            if ((mask >> k) & 1) st->rz[k] = tot[k];
}

// p = D^-1 r + beta p
template <typename T>
__global__ void pcg_direction_kernel(VecArgs<T> a) {
    PcgState *st = a.st;
    if (st->nactive == 0) return;
    bool act[6];
    T be[6];
#pragma unroll
    for (int k = 0; k < 6; ++k) {
        act[k] = st->active[k] != 0;
        be[k] = (T)st->beta[k];
    }
    const size_t N = a.N;
    T *__restrict__ p = a.p;
    const T *__restrict__ r = a.r;
    const T *__restrict__ z = a.z;
    const T *__restrict__ dinv = a.dinv;
    for (size_t n = blockIdx.x * (size_t)blockDim.x + threadIdx.x; n < N; n += (size_t)gridDim.x * blockDim.x) {
        const T di = z ? T(0) : dinv[n];
#pragma unroll
        for (int k = 0; k < 6; ++k) {
            if (!act[k]) continue;
#pragma unroll
            for (int i = 0; i < 3; ++i) {
                const size_t o = (size_t)(3 * k + i) * N + n;
                p[o] = (z ? z[o] : di * r[o]) + be[k] * p[o];
            }
        }
    }
}

// Start of a solve: p = z = D^-1 r, rz = r.z, rr = r.r, active = rr > tol2 bnorm2.
// want_mask selects the load cases to solve (others stay inactive).
template <typename T>
__global__ void pcg_init_kernel(VecArgs<T> a, int want_mask, int set_bnorm) {
    PcgState *st = a.st;
    DotAcc<T> dacc[12];
    const size_t N = a.N;
    for (size_t n = blockIdx.x * (size_t)blockDim.x + threadIdx.x; n < N; n += (size_t)gridDim.x * blockDim.x) {
        const T di = a.z ? T(0) : a.dinv[n];
#pragma unroll
        for (int k = 0; k < 6; ++k) {
            if (!((want_mask >> k) & 1)) continue;
#pragma unroll
            for (int i = 0; i < 3; ++i) {
                const size_t o = (size_t)(3 * k + i) * N + n;
                const T rv = a.r[o];
                const T z = a.z ? a.z[o] : di * rv;
                a.p[o] = z;
                dacc[k].add(rv * z);
                dacc[6 + k].add(rv * rv);
            }
        }
    }
    double acc[12];
#pragma unroll
    for (int k = 0; k < 12; ++k) acc[k] = dacc[k].get();
    const unsigned nb = gridDim.x;
    block_reduce_store<12>(acc, a.partial, blockIdx.x);
    if (!last_block_ticket(&st->ticket_aux, nb)) return;
    __shared__ double tot[12];
    sum_partials_ordered<12>(a.partial, nb, tot);
    if (threadIdx.x == 0) {
        int na = 0;
        for (int k = 0; k < 6; ++k) {
            st->iters[k] = 0;
            st->alpha[k] = st->beta[k] = 0.0;
            st->rz[k] = tot[k];
            st->rr[k] = tot[6 + k];
            if (set_bnorm) st->bnorm2[k] = tot[6 + k];
            const bool want = (want_mask >> k) & 1;
            st->active[k] = want && (tot[6 + k] > st->tol2 * st->bnorm2[k]) && st->bnorm2[k] > 0.0;
            if (want && !isfinite(tot[6 + k])) {
                st->numeric_err = kNumErrInit;
                st->active[k] = 0;
            }
            na += st->active[k];
        }
        st->nactive = na;
    }
}

// ---- FP64 CG with the FP32 multigrid preconditioner ------------------------
// out = float(in) / out = double(in) on the 18 planes of the active load
// cases (all six when st is null): the residual goes to the FP32 V-cycle and
// its result comes back, while the CG recurrences stay FP64.
__global__ void cvt_f64_f32_kernel(size_t N, const PcgState *st, const double *__restrict__ in,
                                   float *__restrict__ out) {
    pdl_enter();
    if (st && st->nactive == 0) return;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < 18 * N; i += (size_t)gridDim.x * blockDim.x) {
        if (st && !st->active[i / (3 * N)]) continue;
        out[i] = (float)in[i];
    }
}
__global__ void cvt_f32_f64_kernel(size_t N, const PcgState *st, const float *__restrict__ in,
                                   double *__restrict__ out) {
    pdl_enter();
    if (st && st->nactive == 0) return;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < 18 * N; i += (size_t)gridDim.x * blockDim.x) {
        if (st && !st->active[i / (3 * N)]) continue;
        out[i] = (double)in[i];
    }
}

// ---- mixed precision: reliable updates -------------------------------------
//
// The FP32 PCG keeps its Krylov direction; every time its recurrence
// residual has fallen by a factor delta (or claims convergence) the FP32
// correction is folded into the FP64 iterate, the true residual f - K x64 is
// recomputed in FP64, and the FP32 residual is replaced by it.  The search
// direction p = z + beta p_prev is moved to the new residual,
// p += D^-1 (r_new - r_old), so the next step is the CG step from the true
// residual along the same conjugate direction.

// x64 += x32 ; x32 = 0 for the load cases in mask
// x64 += x32, x32 = 0 for the load cases in mask; with xdf, also the new x64
// as double-floats (the operand of the true-residual apply that follows).
__global__ void reliable_fold_kernel(size_t N, float *x32, double *x64, int mask, dfloat *xdf) {
    for (size_t n = blockIdx.x * (size_t)blockDim.x + threadIdx.x; n < N; n += (size_t)gridDim.x * blockDim.x) {
        for (int k = 0; k < 6; ++k) {
            if (!((mask >> k) & 1)) continue;
            for (int i = 0; i < 3; ++i) {
                const size_t o = (size_t)(3 * k + i) * N + n;
                const double v = x64[o] + (double)x32[o];
                x64[o] = v;
                x32[o] = 0.0f;
                if (xdf) xdf[o] = dfloat(v);
            }
        }
    }
}

// r_new = float(r64); p += D^-1 (r_new - r) (or p = D^-1 r_new for the load
// cases in restart, whose last direction update was skipped because their
// FP32 residual claimed convergence); r = r_new; rz, rr for mask.
// Last block: a load case stays active unless its true FP64 residual
// (rr_true, squared) meets tol2 * bnorm2 or its iteration budget is spent.
// The true residual comes as doubles (r64) or, straight from the
// double-float apply, as double-floats (rdf; rounded to FP32 as their exact
// sum would be).
__global__ void reliable_rebase_kernel(VecArgs<float> a, const double *r64, const dfloat *rdf, int mask,
                                       int restart, const double *rr_true) {
    PcgState *st = a.st;
    DotAcc<float> dacc[12];
    const size_t N = a.N;
    for (size_t n = blockIdx.x * (size_t)blockDim.x + threadIdx.x; n < N; n += (size_t)gridDim.x * blockDim.x) {
        const float di = a.z ? 0.0f : a.dinv[n];
#pragma unroll
        for (int k = 0; k < 6; ++k) {
            if (!((mask >> k) & 1)) continue;
#pragma unroll
            for (int i = 0; i < 3; ++i) {
                const size_t o = (size_t)(3 * k + i) * N + n;
                const float rn = rdf ? __fadd_rn(rdf[o].hi, rdf[o].lo) : (float)r64[o];
                if (!a.z) {
                    if ((restart >> k) & 1)
                        a.p[o] = di * rn;
                    else
                        a.p[o] += di * (rn - a.r[o]);
                }
                a.r[o] = rn;
                dacc[k].add(rn * (di * rn));
                dacc[6 + k].add(rn * rn);
            }
        }
    }
    double acc[12];
#pragma unroll
    for (int k = 0; k < 12; ++k) acc[k] = dacc[k].get();
    const unsigned nb = gridDim.x;
    block_reduce_store<12>(acc, a.partial, blockIdx.x);
    if (!last_block_ticket(&st->ticket_aux, nb)) return;
    __shared__ double tot[12];
    sum_partials_ordered<12>(a.partial, nb, tot);
    if (threadIdx.x == 0) {
        int na = 0;
        for (int k = 0; k < 6; ++k) {
            if ((mask >> k) & 1) {
                st->rz[k] = tot[k];
                st->rr[k] = tot[6 + k];
                if (!isfinite(rr_true[k]) || !isfinite(tot[k])) {
                    st->numeric_err = kNumErrRestart;
                    st->active[k] = 0;
                } else {
                    st->active[k] = (rr_true[k] > st->tol2 * st->bnorm2[k]) && (st->iters[k] < st->maxit);
                }
            }
            na += st->active[k];
        }
        st->nactive = na;
    }
}

// ---- refinement helpers ----------------------------------------------------

// b32 = r64 / s_k for the load cases in mask (s_k = ||r64_k||), x32 = 0.
__global__ void refine_scatter_kernel(size_t N, const double *r64, const double *scale, int mask, float *b32,
                                      float *x32) {
    for (size_t n = blockIdx.x * (size_t)blockDim.x + threadIdx.x; n < N; n += (size_t)gridDim.x * blockDim.x) {
        for (int k = 0; k < 6; ++k) {
            if (!((mask >> k) & 1)) continue;
            const double inv = 1.0 / scale[k];
            for (int i = 0; i < 3; ++i) {
                const size_t o = (size_t)(3 * k + i) * N + n;
                b32[o] = (float)(r64[o] * inv);
                x32[o] = 0.0f;
            }
        }
    }
}

// x64 += s_k x32
__global__ void refine_gather_kernel(size_t N, const float *x32, const double *scale, int mask, double *x64) {
    for (size_t n = blockIdx.x * (size_t)blockDim.x + threadIdx.x; n < N; n += (size_t)gridDim.x * blockDim.x) {
        for (int k = 0; k < 6; ++k) {
            if (!((mask >> k) & 1)) continue;
            for (int i = 0; i < 3; ++i) {
                const size_t o = (size_t)(3 * k + i) * N + n;
                x64[o] += scale[k] * (double)x32[o];
            }
        }
    }
}

}  // namespace shl
