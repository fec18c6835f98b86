// mg.cuh -- geometric multigrid V-cycle preconditioner for the batched 6-RHS
// PCG (Sec. 4.2: multigrid on the voxel hierarchy, 2x2x2 coarsening, one
// Dirichlet node on the coarsest level solved directly; here on the dense
// periodic grid).
//
// Levels l = 0 (fine, r) .. L (coarsest), r_{l+1} = r_l / 2 while r_l is
// even and >= 6.  Prolongation P is trilinear interpolation, restriction
// R = P^T.  Coarse operators are Galerkin, A_{l+1} = P^T A_l P, stored as
// 27-point stencils of 3x3 blocks (S[I][delta][i][j], delta = (dz+1)*9 +
// (dy+1)*3 + (dx+1)):
//   level 1 from the fine elements: a coarse element's matrix is
//     sum_c E_c P_c^T Khat P_c over its 8 children c, with the 8 child
//     matrices M_c = P_c^T K_unit P_c precomputed (sum_c M_c = 2 K_unit: the
//     Galerkin operator of a uniform material is the rediscretised one);
//   level l+1 from level l: S'[I][d] = sum_{a,b} w(a) w(a + b - 2 d) S[2I+a][b],
//     w(v) = prod_dim max(0, 1 - |v|/2).
// Smoother: damped 3x3 block Jacobi, nu sweeps before and after (symmetric,
// so the V-cycle is a symmetric preconditioner).  Fine level: the matrix-free
// apply with node 0 pinned (its block-Jacobi inverse is zero, so the pinned
// DOFs never move).  Coarsest level: the stencil assembled densely on the
// host, coarse node 0 pinned, inverted in FP64, applied as a dense matvec.
#pragma once

#include "apply.cuh"

namespace shl {

constexpr int kMgMaxLevels = 10;
constexpr int kMgMaxCoarse = 216;  // nodes of the coarsest level (dense inverse on the host)


// Trilinear weight of a fine-node offset v (in fine cells) from a coarse node.
__host__ __device__ inline float tri_w(int vx, int vy, int vz) {
    const int ax = vx < 0 ? -vx : vx, ay = vy < 0 ? -vy : vy, az = vz < 0 ? -vz : vz;
    if (ax > 1 || ay > 1 || az > 1) return 0.0f;
    return (ax ? 0.5f : 1.0f) * (ay ? 0.5f : 1.0f) * (az ? 0.5f : 1.0f);
}

// Host: the 8 child matrices M_c (binary corner order, DOF 3*b+i), unit element.
inline double build_child_matrices(double nu, float Mc[8][24][24]) {
    double Ku[24][24];
    unit_hex8_stiffness(nu, Ku);
    double sum[24][24] = {};
    for (int c = 0; c < 8; ++c) {
        double P[8][8];  // P[b][B]: weight of coarse corner B at child corner b
        for (int b = 0; b < 8; ++b)
            for (int B = 0; B < 8; ++B) {
                double w = 1.0;
                for (int d = 0; d < 3; ++d) {
                    const double s = 0.5 * (((c >> d) & 1) + ((b >> d) & 1));
                    w *= ((B >> d) & 1) ? s : 1.0 - s;
                }
                P[b][B] = w;
            }
        for (int A = 0; A < 8; ++A)
            for (int i = 0; i < 3; ++i)
                for (int B = 0; B < 8; ++B)
                    for (int j = 0; j < 3; ++j) {
                        double s = 0.0;
                        for (int b = 0; b < 8; ++b)
                            for (int b2 = 0; b2 < 8; ++b2) s += P[b][A] * Ku[3 * b + i][3 * b2 + j] * P[b2][B];
                        Mc[c][3 * A + i][3 * B + j] = (float)s;
                        sum[3 * A + i][3 * B + j] += s;
                    }
    }
    double err = 0.0, mx = 0.0;
    for (int m = 0; m < 24; ++m)
        for (int n = 0; n < 24; ++n) {
            err = std::fmax(err, std::fabs(sum[m][n] - 2.0 * Ku[m][n]));
            mx = std::fmax(mx, std::fabs(Ku[m][n]));
        }
    return err / mx;
}

__device__ inline int wrap_l(int v, int r) { return v < 0 ? v + r : (v >= r ? v - r : v); }

// Kernels of the V-cycle run inside the PCG loop: they stop early once every
// load case has converged (uniform across the grid).
__device__ inline bool mg_done(const PcgState *st) { return st && st->nactive == 0; }

// Level 1 stencil from the fine elements.  Thread = (coarse node I, offset delta).
// Mc: the 8 child matrices P_c^T K_unit P_c (unit modulus, unit element),
// [8][24][24] floats in device memory (per context, uploaded at setup).
__global__ void mg_galerkin_fine_kernel(int rc, const uint8_t *mask, const double *rho, float E, float Ev, float h,
                                        const float *__restrict__ Mc, float *S) {
    const size_t Nc = (size_t)rc * rc * rc;
    const int rf = 2 * rc;
    for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < Nc * 27; t += (size_t)gridDim.x * blockDim.x) {
        const size_t I = t / 27;
        const int dl = (int)(t % 27);
        const int dx = dl % 3 - 1, dy = (dl / 3) % 3 - 1, dz = dl / 9 - 1;
        const int ix = I % rc, iy = (I / rc) % rc, iz = I / ((size_t)rc * rc);
        float acc[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
        for (int A = 0; A < 8; ++A) {
            const int ax = A & 1, ay = (A >> 1) & 1, az = A >> 2;
            const int bx = ax + dx, by = ay + dy, bz = az + dz;
            if (bx < 0 || bx > 1 || by < 0 || by > 1 || bz < 0 || bz > 1) continue;
            const int B = bx + 2 * by + 4 * bz;
            const int X = wrap_l(ix - ax, rc), Y = wrap_l(iy - ay, rc), Z = wrap_l(iz - az, rc);
            for (int c = 0; c < 8; ++c) {
                const size_t e = ((size_t)(2 * Z + (c >> 2)) * rf + (2 * Y + ((c >> 1) & 1))) * rf + (2 * X + (c & 1));
                const float Ee = rho ? (float)(Ev + rho[e] * (E - Ev)) : (mask[e] ? E : Ev);
#pragma unroll
                for (int i = 0; i < 3; ++i)
#pragma unroll
                    for (int j = 0; j < 3; ++j) acc[3 * i + j] += Ee * __ldg(Mc + (c * 24 + 3 * A + i) * 24 + 3 * B + j);
            }
        }
#pragma unroll
        for (int m = 0; m < 9; ++m) S[(size_t)(dl * 9 + m) * Nc + I] = h * acc[m];
    }
}

// Level l+1 stencil from level l (Galerkin with trilinear P).  Thread = (I, delta).
__global__ void mg_galerkin_coarse_kernel(int rc, const float *__restrict__ Sf, float *__restrict__ Sc) {
    const size_t Nc = (size_t)rc * rc * rc;
    const int rf = 2 * rc;
    const size_t Nf = (size_t)rf * rf * rf;
    for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < Nc * 27; t += (size_t)gridDim.x * blockDim.x) {
        const size_t I = t / 27;
        const int dl = (int)(t % 27);
        const int dx = dl % 3 - 1, dy = (dl / 3) % 3 - 1, dz = dl / 9 - 1;
        const int ix = I % rc, iy = (I / rc) % rc, iz = I / ((size_t)rc * rc);
        float acc[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
        for (int az = -1; az <= 1; ++az)
            for (int ay = -1; ay <= 1; ++ay)
                for (int ax = -1; ax <= 1; ++ax) {
                    const float wa = tri_w(ax, ay, az);
                    const size_t fi =
                        ((size_t)wrap_l(2 * iz + az, rf) * rf + wrap_l(2 * iy + ay, rf)) * rf + wrap_l(2 * ix + ax, rf);
                    for (int bz = -1; bz <= 1; ++bz)
                        for (int by = -1; by <= 1; ++by)
                            for (int bx = -1; bx <= 1; ++bx) {
                                const float wb = tri_w(ax + bx - 2 * dx, ay + by - 2 * dy, az + bz - 2 * dz);
                                if (wb == 0.0f) continue;
                                const float w = wa * wb;
                                const int bl = (bz + 1) * 9 + (by + 1) * 3 + (bx + 1);
#pragma unroll
                                for (int m = 0; m < 9; ++m) acc[m] += w * Sf[(size_t)(bl * 9 + m) * Nf + fi];
                            }
                }
#pragma unroll
        for (int m = 0; m < 9; ++m) Sc[(size_t)(dl * 9 + m) * Nc + I] = acc[m];
    }
}

__device__ inline void inv3(const double a[9], double o[9]) {
    const double c00 = a[4] * a[8] - a[5] * a[7], c01 = a[5] * a[6] - a[3] * a[8], c02 = a[3] * a[7] - a[4] * a[6];
    const double det = a[0] * c00 + a[1] * c01 + a[2] * c02;
    const double id = det != 0.0 ? 1.0 / det : 0.0;
    o[0] = c00 * id;
    o[1] = (a[2] * a[7] - a[1] * a[8]) * id;
    o[2] = (a[1] * a[5] - a[2] * a[4]) * id;
    o[3] = c01 * id;
    o[4] = (a[0] * a[8] - a[2] * a[6]) * id;
    o[5] = (a[2] * a[3] - a[0] * a[5]) * id;
    o[6] = c02 * id;
    o[7] = (a[1] * a[6] - a[0] * a[7]) * id;
    o[8] = (a[0] * a[4] - a[1] * a[3]) * id;
}

// Block-Jacobi inverse of a stencil level (center block).
__global__ void mg_dinv_stencil_kernel(size_t N, const float *S, float *Dinv) {
    for (size_t n = blockIdx.x * (size_t)blockDim.x + threadIdx.x; n < N; n += (size_t)gridDim.x * blockDim.x) {
        double a[9], o[9];
        for (int m = 0; m < 9; ++m) a[m] = S[(size_t)(13 * 9 + m) * N + n];
        inv3(a, o);
        for (int m = 0; m < 9; ++m) Dinv[(size_t)m * N + n] = (float)o[m];
    }
}

// Block-Jacobi inverse at the fine level: sum over the 8 incident elements of
// E_e Khat's corner-diagonal block; node 0 (pinned) gets a zero inverse.
struct CornerBlocks {
    float K[8][9];  // Khat[(a,i),(a,j)] for corner a
};

__global__ void mg_dinv_fine_kernel(int r, const uint8_t *mask, const double *rho, float E, float Ev, CornerBlocks cb,
                                    float *Dinv) {
    const size_t N = (size_t)r * r * r;
    for (size_t n = blockIdx.x * (size_t)blockDim.x + threadIdx.x; n < N; n += (size_t)gridDim.x * blockDim.x) {
        const int ix = n % r, iy = (n / r) % r, iz = n / ((size_t)r * r);
        double a[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0}, o[9];
        for (int b = 0; b < 8; ++b) {
            const size_t e = ((size_t)wrap_l(iz - (b >> 2), r) * r + wrap_l(iy - ((b >> 1) & 1), r)) * r +
                             wrap_l(ix - (b & 1), r);
            const double Ee = rho ? Ev + rho[e] * (E - Ev) : (mask[e] ? E : Ev);
            for (int m = 0; m < 9; ++m) a[m] += Ee * cb.K[b][m];
        }
        inv3(a, o);
        for (int m = 0; m < 9; ++m) Dinv[(size_t)m * N + n] = n == 0 ? 0.0f : (float)o[m];
    }
}

// Smoother pieces (18 SoA planes).  first: x = w D^-1 b;  update: x += w D^-1 (b - t).
__global__ void mg_jacobi_kernel(size_t N, const float *__restrict__ b, const float *__restrict__ t,
                                 const float *__restrict__ Dinv, float w, float *__restrict__ x, int first,
                                 const PcgState *st) {
    if (mg_done(st)) return;
    for (size_t n = blockIdx.x * (size_t)blockDim.x + threadIdx.x; n < N; n += (size_t)gridDim.x * blockDim.x) {
        float D[9];
#pragma unroll
        for (int m = 0; m < 9; ++m) D[m] = Dinv[(size_t)m * N + n];
#pragma unroll
        for (int k = 0; k < 6; ++k) {
            float rv[3];
#pragma unroll
            for (int i = 0; i < 3; ++i) {
                const size_t o = (size_t)(3 * k + i) * N + n;
                rv[i] = first ? b[o] : b[o] - t[o];
            }
#pragma unroll
            for (int i = 0; i < 3; ++i) {
                const size_t o = (size_t)(3 * k + i) * N + n;
                const float dx = w * (D[3 * i] * rv[0] + D[3 * i + 1] * rv[1] + D[3 * i + 2] * rv[2]);
                x[o] = first ? dx : x[o] + dx;
            }
        }
    }
}

// 27-point 3x3-block stencil (periodic) with a fused epilogue:
//   mode 0: out = S x
//   mode 1: out = b - S x                      (residual)
//   mode 2: out = x + w D^-1 (b - S x)         (one damped block-Jacobi sweep)
__global__ void mg_stencil_kernel(int r, const float *__restrict__ S, const float *__restrict__ x,
                                  const float *__restrict__ b, const float *__restrict__ Dinv, float w, int mode,
                                  float *__restrict__ out, const PcgState *st) {
    if (mg_done(st)) return;
    const size_t N = (size_t)r * r * r;
    for (size_t n = blockIdx.x * (size_t)blockDim.x + threadIdx.x; n < N; n += (size_t)gridDim.x * blockDim.x) {
        const int ix = n % r, iy = (n / r) % r, iz = n / ((size_t)r * r);
        float acc[18];
#pragma unroll
        for (int m = 0; m < 18; ++m) acc[m] = 0.0f;
        for (int dl = 0; dl < 27; ++dl) {
            const int dx = dl % 3 - 1, dy = (dl / 3) % 3 - 1, dz = dl / 9 - 1;
            const size_t j = ((size_t)wrap_l(iz + dz, r) * r + wrap_l(iy + dy, r)) * r + wrap_l(ix + dx, r);
            float B[9];
#pragma unroll
            for (int m = 0; m < 9; ++m) B[m] = S[(size_t)(dl * 9 + m) * N + n];
#pragma unroll
            for (int k = 0; k < 6; ++k) {
                const float x0 = x[(size_t)(3 * k) * N + j], x1 = x[(size_t)(3 * k + 1) * N + j],
                            x2 = x[(size_t)(3 * k + 2) * N + j];
#pragma unroll
                for (int i = 0; i < 3; ++i) acc[3 * k + i] += B[3 * i] * x0 + B[3 * i + 1] * x1 + B[3 * i + 2] * x2;
            }
        }
        if (mode == 0) {
#pragma unroll
            for (int m = 0; m < 18; ++m) out[(size_t)m * N + n] = acc[m];
        } else if (mode == 1) {
#pragma unroll
            for (int m = 0; m < 18; ++m) out[(size_t)m * N + n] = b[(size_t)m * N + n] - acc[m];
        } else {
            float D[9];
#pragma unroll
            for (int m = 0; m < 9; ++m) D[m] = Dinv[(size_t)m * N + n];
#pragma unroll
            for (int k = 0; k < 6; ++k) {
                float rv[3];
#pragma unroll
                for (int i = 0; i < 3; ++i) rv[i] = b[(size_t)(3 * k + i) * N + n] - acc[3 * k + i];
#pragma unroll
                for (int i = 0; i < 3; ++i) {
                    const size_t o = (size_t)(3 * k + i) * N + n;
                    out[o] = x[o] + w * (D[3 * i] * rv[0] + D[3 * i + 1] * rv[1] + D[3 * i + 2] * rv[2]);
                }
            }
        }
    }
}

// bc = R (bf - tf): coarse I gathers w(a) (bf - tf)[2I + a]; tf may be null
// (bf is then the residual itself).
__global__ void mg_restrict_kernel(int rc, const float *__restrict__ bf, const float *__restrict__ tf,
                                   float *__restrict__ bc, const PcgState *st) {
    if (mg_done(st)) return;
    const size_t Nc = (size_t)rc * rc * rc;
    const int rf = 2 * rc;
    const size_t Nf = (size_t)rf * rf * rf;
    for (size_t I = blockIdx.x * (size_t)blockDim.x + threadIdx.x; I < Nc; I += (size_t)gridDim.x * blockDim.x) {
        const int ix = I % rc, iy = (I / rc) % rc, iz = I / ((size_t)rc * rc);
        float acc[18];
#pragma unroll
        for (int m = 0; m < 18; ++m) acc[m] = 0.0f;
        for (int az = -1; az <= 1; ++az)
            for (int ay = -1; ay <= 1; ++ay)
                for (int ax = -1; ax <= 1; ++ax) {
                    const float w = tri_w(ax, ay, az);
                    const size_t f =
                        ((size_t)wrap_l(2 * iz + az, rf) * rf + wrap_l(2 * iy + ay, rf)) * rf + wrap_l(2 * ix + ax, rf);
                    if (tf) {
#pragma unroll
                        for (int m = 0; m < 18; ++m) acc[m] += w * (bf[(size_t)m * Nf + f] - tf[(size_t)m * Nf + f]);
                    } else {
#pragma unroll
                        for (int m = 0; m < 18; ++m) acc[m] += w * bf[(size_t)m * Nf + f];
                    }
                }
#pragma unroll
        for (int m = 0; m < 18; ++m) bc[(size_t)m * Nc + I] = acc[m];
    }
}

// xf += P xc (trilinear), fine node i from the coarse nodes around it; the
// fine node 0 (pinned at level 0) is left untouched when pin0 is set.
__global__ void mg_prolong_kernel(int rc, const float *__restrict__ xc, float *__restrict__ xf, int pin0,
                                  const PcgState *st) {
    if (mg_done(st)) return;
    const int rf = 2 * rc;
    const size_t Nf = (size_t)rf * rf * rf, Nc = (size_t)rc * rc * rc;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < Nf; i += (size_t)gridDim.x * blockDim.x) {
        if (pin0 && i == 0) continue;
        const int fx = i % rf, fy = (i / rf) % rf, fz = i / ((size_t)rf * rf);
        const int cx0 = fx >> 1, cy0 = fy >> 1, cz0 = fz >> 1;
        const int nx = (fx & 1) + 1, ny = (fy & 1) + 1, nz = (fz & 1) + 1;
        const float wx = (fx & 1) ? 0.5f : 1.0f, wy = (fy & 1) ? 0.5f : 1.0f, wz = (fz & 1) ? 0.5f : 1.0f;
        float acc[18];
#pragma unroll
        for (int m = 0; m < 18; ++m) acc[m] = 0.0f;
        for (int kz = 0; kz < nz; ++kz)
            for (int ky = 0; ky < ny; ++ky)
                for (int kx = 0; kx < nx; ++kx) {
                    const size_t I = ((size_t)wrap_l(cz0 + kz, rc) * rc + wrap_l(cy0 + ky, rc)) * rc + wrap_l(cx0 + kx, rc);
                    const float w = wx * wy * wz;
#pragma unroll
                    for (int m = 0; m < 18; ++m) acc[m] += w * xc[(size_t)m * Nc + I];
                }
#pragma unroll
        for (int m = 0; m < 18; ++m) xf[(size_t)m * Nf + i] += acc[m];
    }
}

// ---- lambda_max(D^-1 A) by power iteration (sets the damping per level) ----
// Uses the first three planes (one load case).
__global__ void mg_power_seed_kernel(size_t N, float *x) {
    for (size_t n = blockIdx.x * (size_t)blockDim.x + threadIdx.x; n < 18 * N; n += (size_t)gridDim.x * blockDim.x) {
        if (n >= 3 * N) {
            x[n] = 0.0f;
            continue;
        }
        unsigned h = (unsigned)n * 2654435761u + 0x9e3779b9u;
        h ^= h >> 15;
        h *= 2246822519u;
        h ^= h >> 13;
        x[n] = (float)(h & 0xffffff) / 8388608.0f - 1.0f;
    }
}

// y = D^-1 t on planes 0..2 and ||y||^2 (deterministic last-block reduction).
__global__ void mg_power_dinv_kernel(size_t N, const float *t, const float *Dinv, float *y, double *partial,
                                     unsigned *ticket, double *out) {
    double acc[1] = {0.0};
    for (size_t n = blockIdx.x * (size_t)blockDim.x + threadIdx.x; n < N; n += (size_t)gridDim.x * blockDim.x) {
        float D[9];
#pragma unroll
        for (int m = 0; m < 9; ++m) D[m] = Dinv[(size_t)m * N + n];
        const float r0 = t[n], r1 = t[N + n], r2 = t[2 * N + n];
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            const float v = D[3 * i] * r0 + D[3 * i + 1] * r1 + D[3 * i + 2] * r2;
            y[(size_t)i * N + n] = v;
            acc[0] += (double)v * v;
        }
    }
    block_reduce_store<1>(acc, partial, blockIdx.x);
    if (!last_block_ticket(ticket, gridDim.x)) return;
    __shared__ double tot[1];
    sum_partials_ordered<1>(partial, gridDim.x, tot);
    if (threadIdx.x == 0) out[0] = tot[0];
}

// x = y / ||y|| on planes 0..2
__global__ void mg_power_scale_kernel(size_t N, const float *y, const double *nrm2, float *x) {
    const float inv = (float)(1.0 / sqrt(nrm2[0] > 0.0 ? nrm2[0] : 1.0));
    for (size_t n = blockIdx.x * (size_t)blockDim.x + threadIdx.x; n < 3 * N; n += (size_t)gridDim.x * blockDim.x)
        x[n] = y[n] * inv;
}

// x = Ainv b on the coarsest level (dense, 3N x 3N, applied per load case).
__global__ void mg_dense_solve_kernel(int n3, const float *__restrict__ Ainv, const float *__restrict__ b,
                                      float *__restrict__ x, const PcgState *st) {
    if (mg_done(st)) return;
    const int N = n3 / 3;
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < 6 * n3; t += gridDim.x * blockDim.x) {
        const int k = t / n3, row = t % n3;
        float s = 0.0f;
        for (int col = 0; col < n3; ++col) {
            const int cn = col / 3, ci = col % 3;
            s += Ainv[(size_t)row * n3 + col] * b[(size_t)(3 * k + ci) * N + cn];
        }
        x[(size_t)(3 * k + row % 3) * N + row / 3] = s;
    }
}

}  // namespace shl
