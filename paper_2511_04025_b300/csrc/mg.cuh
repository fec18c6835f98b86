// mg.cuh -- geometric multigrid V-cycle preconditioner for the batched 6-RHS
// PCG (Sec. 4.2: multigrid on the voxel hierarchy, 2x2x2 coarsening, one
// Dirichlet node on the coarsest level solved directly; here on the dense
// periodic grid).
//
// Levels l = 0 (fine, r) .. L (coarsest), r_{l+1} = r_l / 2 while r_l is
// even and >= 6.  Prolongation P is trilinear interpolation, restriction
// R = P^T.  Coarse operators are Galerkin, A_{l+1} = P^T A_l P, stored as
// 27-point stencils of 3x3 blocks, node-major (S[I][delta][i][j], delta =
// (dz+1)*9 + (dy+1)*3 + (dx+1); one node's 243 entries are contiguous):
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
// host, coarse node 0 pinned, regularised by a small multiple of the
// all-solid stiffness, factored by Cholesky in FP64 and applied as
// Y^T (Y b) with the FP32 inverse factor Y = L^-1.
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

// Node activity of the active set (Sec. 4.2.1), per level: a fine node is
// active when one of its 8 elements carries stiffness, a coarse node when one
// of the fine nodes 2I + a (a in {-1, 0, 1}^3) of its prolongation support is.
// An inactive node's stencil row and block inverse are exactly zero on every
// level (every product that forms them sums zeros), so the kernels below can
// skip it without changing a result.
__global__ void mg_node_active_fine_kernel(int r, const uint8_t *mask, const double *rho, double E, double Ev,
                                           uint8_t *act) {
    const size_t N = (size_t)r * r * r;
    for (size_t n = blockIdx.x * (size_t)blockDim.x + threadIdx.x; n < N; n += (size_t)gridDim.x * blockDim.x) {
        const int ix = n % r, iy = (n / r) % r, iz = n / ((size_t)r * r);
        bool any = false;
        for (int b = 0; b < 8 && !any; ++b) {
            const size_t e = ((size_t)wrap_l(iz - (b >> 2), r) * r + wrap_l(iy - ((b >> 1) & 1), r)) * r +
                             wrap_l(ix - (b & 1), r);
            any = (rho ? Ev + rho[e] * (E - Ev) : (mask[e] ? E : Ev)) != 0.0;
        }
        act[n] = any ? 1 : 0;
    }
}
__global__ void mg_node_active_coarse_kernel(int rc, const uint8_t *__restrict__ act_f, uint8_t *__restrict__ act_c) {
    const size_t Nc = (size_t)rc * rc * rc;
    const int rf = 2 * rc;
    for (size_t I = blockIdx.x * (size_t)blockDim.x + threadIdx.x; I < Nc; I += (size_t)gridDim.x * blockDim.x) {
        const int ix = I % rc, iy = (I / rc) % rc, iz = I / ((size_t)rc * rc);
        bool any = false;
        for (int a = 0; a < 27 && !any; ++a)
            any = act_f[((size_t)wrap_l(2 * iz + a / 9 - 1, rf) * rf + wrap_l(2 * iy + (a / 3) % 3 - 1, rf)) * rf +
                        wrap_l(2 * ix + a % 3 - 1, rf)] != 0;
        act_c[I] = any ? 1 : 0;
    }
}
// blk[b] = 1 when one of the nodes 32 b .. 32 b + 31 is active (the node
// groups of mg_stencil_nc_kernel)
__global__ void mg_block_active_kernel(size_t N, const uint8_t *__restrict__ act, uint8_t *__restrict__ blk) {
    const size_t nb = (N + 31) / 32;
    for (size_t b = blockIdx.x * (size_t)blockDim.x + threadIdx.x; b < nb; b += (size_t)gridDim.x * blockDim.x) {
        bool any = false;
        for (size_t n = 32 * b; n < min(N, 32 * b + 32) && !any; ++n) any = act[n] != 0;
        blk[b] = any ? 1 : 0;
    }
}

// Level 1 stencil from the fine elements.  Thread = (coarse node I, offset delta).
// Mc: the 8 child matrices P_c^T K_unit P_c (unit modulus, unit element),
// [8][24][24] floats in device memory (per context, uploaded at setup).
__global__ void mg_galerkin_fine_kernel(int rc, const uint8_t *mask, const double *rho, float E, float Ev, float h,
                                        const float *__restrict__ Mc, float *S, const uint8_t *act_c) {
    const size_t Nc = (size_t)rc * rc * rc;
    const int rf = 2 * rc;
    for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < Nc * 27; t += (size_t)gridDim.x * blockDim.x) {
        const size_t I = t / 27;
        const int dl = (int)(t % 27);
        const int dx = dl % 3 - 1, dy = (dl / 3) % 3 - 1, dz = dl / 9 - 1;
        const int ix = I % rc, iy = (I / rc) % rc, iz = I / ((size_t)rc * rc);
        float acc[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
        if (act_c && !act_c[I]) {  // inactive coarse node (active set): every child culled, a zero row
#pragma unroll
            for (int m = 0; m < 9; ++m) S[(I * 27 + dl) * 9 + m] = 0.0f;
            continue;
        }
        for (int A = 0; A < 8; ++A) {
            const int ax = A & 1, ay = (A >> 1) & 1, az = A >> 2;
            const int bx = ax + dx, by = ay + dy, bz = az + dz;
            if (bx < 0 || bx > 1 || by < 0 || by > 1 || bz < 0 || bz > 1) continue;
            const int B = bx + 2 * by + 4 * bz;
            const int X = wrap_l(ix - ax, rc), Y = wrap_l(iy - ay, rc), Z = wrap_l(iz - az, rc);
            for (int c = 0; c < 8; ++c) {
                const size_t e = ((size_t)(2 * Z + (c >> 2)) * rf + (2 * Y + ((c >> 1) & 1))) * rf + (2 * X + (c & 1));
                const float Ee = rho ? (float)(Ev + rho[e] * (E - Ev)) : (mask[e] ? E : Ev);
                if (Ee == 0.0f) continue;  // culled child (active set): adds exact zeros
#pragma unroll
                for (int i = 0; i < 3; ++i)
#pragma unroll
                    for (int j = 0; j < 3; ++j) acc[3 * i + j] += Ee * __ldg(Mc + (c * 24 + 3 * A + i) * 24 + 3 * B + j);
            }
        }
#pragma unroll
        for (int m = 0; m < 9; ++m) S[(I * 27 + dl) * 9 + m] = h * acc[m];
    }
}

// Level l+1 stencil from level l (Galerkin with trilinear P):
//   Sc(I, delta) = sum_a sum_b w(a) w(a + b - 2 delta) Sf(2I + a, b).
// Block = one coarse node I: the stencils of the 27 fine nodes 2I + a of its
// prolongation support (27 x 243 floats) are staged in shared memory once,
// and thread (delta, entry m) sums its entry from there over (a, b) in the
// same order as a thread per block would (the rounding of these sums decides
// whether a mode held only by the ersatz void stays resolvable on the
// coarsest level, so it is kept fixed).
// ACT (the active set): skip inactive coarse nodes and inactive fine neighbours.
constexpr int kGalerkinThreads = 256;  // 243 entries of a coarse node's stencil
template <bool ACT>
__global__ void __launch_bounds__(kGalerkinThreads)
    mg_galerkin_coarse_kernel(int rc, const float *__restrict__ Sf, float *__restrict__ Sc,
                              const uint8_t *__restrict__ act_f, const uint8_t *__restrict__ act_c) {
    __shared__ float sf[27 * 243];
    __shared__ uint8_t sact[27];
    const size_t Nc = (size_t)rc * rc * rc;
    const int rf = 2 * rc;
    for (size_t I = blockIdx.x; I < Nc; I += gridDim.x) {  // uniform per block
        const int ix = I % rc, iy = (I / rc) % rc, iz = I / ((size_t)rc * rc);
        if (ACT && !act_c[I]) {  // inactive coarse node (active set): a zero row
            for (int t = threadIdx.x; t < 243; t += blockDim.x) Sc[I * 243 + t] = 0.0f;
            continue;
        }
        auto fine = [&](int a) -> size_t {  // fine node 2I + a, a = (az + 1) 9 + (ay + 1) 3 + (ax + 1)
            return ((size_t)wrap_l(2 * iz + a / 9 - 1, rf) * rf + wrap_l(2 * iy + (a / 3) % 3 - 1, rf)) * rf +
                   wrap_l(2 * ix + a % 3 - 1, rf);
        };
        __syncthreads();  // the previous node's reads of sf are done
        for (int k = threadIdx.x; k < 27 * 243; k += blockDim.x) {
            const int a = k / 243;
            const size_t fi = fine(a);
            sf[k] = (ACT && !act_f[fi]) ? 0.0f : __ldg(Sf + fi * 243 + (k - a * 243));
        }
        if (threadIdx.x < 27) sact[threadIdx.x] = ACT ? act_f[fine(threadIdx.x)] : 1;
        __syncthreads();
        if (threadIdx.x < 243) {
            const int t = threadIdx.x, m = t % 9, dl = t / 9;
            const int dx = dl % 3 - 1, dy = (dl / 3) % 3 - 1, dz = dl / 9 - 1;
            float acc = 0.0f;
            for (int az = -1; az <= 1; ++az)
                for (int ay = -1; ay <= 1; ++ay)
                    for (int ax = -1; ax <= 1; ++ax) {
                        const float wa = tri_w(ax, ay, az);
                        const int a = (az + 1) * 9 + (ay + 1) * 3 + (ax + 1);
                        if (ACT && !sact[a]) continue;  // an inactive fine node's row is zero
                        for (int bz = -1; bz <= 1; ++bz)
                            for (int by = -1; by <= 1; ++by)
                                for (int bx = -1; bx <= 1; ++bx) {
                                    const float wb = tri_w(ax + bx - 2 * dx, ay + by - 2 * dy, az + bz - 2 * dz);
                                    if (wb == 0.0f) continue;
                                    const int bl = (bz + 1) * 9 + (by + 1) * 3 + (bx + 1);
                                    acc += (wa * wb) * sf[a * 243 + bl * 9 + m];
                                }
                    }
            Sc[I * 243 + t] = acc;
        }
    }
}

__host__ __device__ inline void inv3(const double a[9], double o[9]) {
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

// Regularisation of the coarsest operator: + kMgCoarseReg E A_hom, A_hom the
// all-solid stiffness on the coarsest grid.  Above the FP32 rounding of the
// Galerkin sums there (~1e-5 of the largest entries), far below the stiffness
// of any load-bearing mode.
constexpr double kMgCoarseReg = 1e-4;

// Eigenvalue floor of the coarse block inverses, relative to the block's
// largest |eigenvalue|: keeps D^-1 SPD after FP32 storage (condition <= 1e5).
constexpr double kMgBlockFloor = 1e-5;

// SPD inverse of a symmetric 3x3 block given with FP32 rounding.  The block
// is symmetrised, diagonalised by cyclic Jacobi rotations, and its
// eigenvalues are raised to kMgBlockFloor |lambda|_max before inverting: a
// node tied to the solid along one direction only has a nearly singular
// Galerkin block that FP32 rounding can make indefinite.  (LDL^T pivots are
// no substitute: all three can clear the floor while the smallest eigenvalue
// does not.)  A zero block gives a zero inverse.
__host__ __device__ inline void spd_inv3(const double a_in[9], double o[9]) {
    double A[3][3];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) A[i][j] = 0.5 * (a_in[3 * i + j] + a_in[3 * j + i]);
    const double tr = fabs(A[0][0]) + fabs(A[1][1]) + fabs(A[2][2]) + fabs(A[0][1]) + fabs(A[0][2]) + fabs(A[1][2]);
    double V[3][3] = {{1, 0, 0}, {0, 1, 0}, {0, 0, 1}};
    for (int sweep = 0; sweep < 10; ++sweep) {
        const double off = fabs(A[0][1]) + fabs(A[0][2]) + fabs(A[1][2]);
        if (!(off > 1e-15 * tr)) break;
        for (int pq = 0; pq < 3; ++pq) {
            const int p = pq == 2 ? 1 : 0, q = pq == 0 ? 1 : 2;
            if (A[p][q] == 0.0) continue;
            const double th = (A[q][q] - A[p][p]) / (2.0 * A[p][q]);
            const double t = (th >= 0.0 ? 1.0 : -1.0) / (fabs(th) + sqrt(th * th + 1.0));
            const double c = 1.0 / sqrt(t * t + 1.0), sn = t * c;
            for (int k = 0; k < 3; ++k) {  // A <- A J (columns p, q)
                const double akp = A[k][p], akq = A[k][q];
                A[k][p] = c * akp - sn * akq;
                A[k][q] = sn * akp + c * akq;
            }
            for (int k = 0; k < 3; ++k) {  // A <- J^T A (rows p, q)
                const double apk = A[p][k], aqk = A[q][k];
                A[p][k] = c * apk - sn * aqk;
                A[q][k] = sn * apk + c * aqk;
            }
            for (int k = 0; k < 3; ++k) {  // V <- V J
                const double vkp = V[k][p], vkq = V[k][q];
                V[k][p] = c * vkp - sn * vkq;
                V[k][q] = sn * vkp + c * vkq;
            }
        }
    }
    double lmax = 0.0;
    for (int i = 0; i < 3; ++i) lmax = fmax(lmax, fabs(A[i][i]));
    double il[3];
    for (int i = 0; i < 3; ++i) il[i] = lmax > 0.0 ? 1.0 / fmax(A[i][i], kMgBlockFloor * lmax) : 0.0;
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j)
            o[3 * i + j] = V[i][0] * il[0] * V[j][0] + V[i][1] * il[1] * V[j][1] + V[i][2] * il[2] * V[j][2];
}

// Block-Jacobi inverse of a stencil level (center block), SPD by construction.
__global__ void mg_dinv_stencil_kernel(size_t N, const float *S, float *Dinv, const uint8_t *act) {
    for (size_t n = blockIdx.x * (size_t)blockDim.x + threadIdx.x; n < N; n += (size_t)gridDim.x * blockDim.x) {
        if (act && !act[n]) {  // inactive node (active set): zero block, zero inverse
            for (int m = 0; m < 9; ++m) Dinv[(size_t)m * N + n] = 0.0f;
            continue;
        }
        double a[9], o[9];
        for (int m = 0; m < 9; ++m) a[m] = S[(n * 27 + 13) * 9 + m];
        spd_inv3(a, o);
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
        bool any = false;
        for (int b = 0; b < 8; ++b) {
            const size_t e = ((size_t)wrap_l(iz - (b >> 2), r) * r + wrap_l(iy - ((b >> 1) & 1), r)) * r +
                             wrap_l(ix - (b & 1), r);
            const double Ee = rho ? Ev + rho[e] * (E - Ev) : (mask[e] ? E : Ev);
            if (Ee == 0.0) continue;  // culled element (active set): adds exact zeros
            any = true;
            for (int m = 0; m < 9; ++m) a[m] += Ee * cb.K[b][m];
        }
        // a node with no active element has a zero block, whose inverse is zero
        if (any) inv3(a, o);
        for (int m = 0; m < 9; ++m) Dinv[(size_t)m * N + n] = (n == 0 || !any) ? 0.0f : (float)o[m];
    }
}

// Smoother pieces (18 SoA planes).  first: x = w D^-1 b;  update: x += w D^-1 (b - t).
__global__ void mg_jacobi_kernel(size_t N, const float *__restrict__ b, const float *__restrict__ t,
                                 const float *__restrict__ Dinv, float w, float *__restrict__ x, int first,
                                 const PcgState *st) {
    pdl_enter();
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

// Warp reduce-scatter of 18 per-lane values: after five halving steps
// (offsets 16, 8, 4, 2, 1; 9 + 5 + 3 + 2 + 1 shuffles) each lane holds the
// warp-wide sum of at most one of the 18 values; rs_id(lane) says which (-1:
// none).  Every step keeps the first ceil(n/2) positions in the lower lane of
// a pair and the rest (padded with zeros) in the upper one.
template <int N, int O>
__device__ __forceinline__ void rs_step(const float (&v)[N], float (&w)[(N + 1) / 2], bool up) {
    constexpr int M = (N + 1) / 2;
#pragma unroll
    for (int q = 0; q < M; ++q) {
        const float lo = v[q];
        const float hi = (M + q < N) ? v[(M + q < N) ? M + q : 0] : 0.0f;
        const float send = up ? lo : hi;
        const float keep = up ? hi : lo;
        w[q] = keep + __shfl_xor_sync(0xffffffffu, send, O);
    }
}

__device__ __forceinline__ float reduce_scatter18(const float (&v)[18], int lane) {
    float a9[9], a5[5], a3[3], a2[2], a1[1];
    rs_step<18, 16>(v, a9, lane & 16);
    rs_step<9, 8>(a9, a5, lane & 8);
    rs_step<5, 4>(a5, a3, lane & 4);
    rs_step<3, 2>(a3, a2, lane & 2);
    rs_step<2, 1>(a2, a1, lane & 1);
    return a1[0];
}

__device__ __forceinline__ int rs_id(int lane) {
    int lo = 0, cnt = 18, n = 18;
    for (int o = 16; o > 0; o >>= 1) {
        const int m = (n + 1) / 2;
        if (lane & o) {
            lo += m;
            cnt = cnt > m ? cnt - m : 0;
        } else {
            cnt = cnt < m ? cnt : m;
        }
        n = m;
    }
    return cnt > 0 ? lo : -1;
}

// 27-point 3x3-block stencil (periodic) with a fused epilogue.  One warp per
// node: lane dl < 27 takes the offset dl (its 9 stencil entries are part of
// the node's contiguous 243, so the warp's loads are coalesced) and all six
// load cases; a reduce-scatter sums the 27 contributions, leaving output
// component rs_id(lane) (load case id / 3) in that lane.  Every load of a node
// is issued at once: the coarse levels are small, so latency, not bandwidth,
// bounds them.
//   mode 0: out = S x
//   mode 1: out = b - S x                      (residual)
//   mode 2: out = x + w D^-1 (b - S x)         (one damped block-Jacobi sweep)
// Load cases that have converged (st->active) are skipped.
__global__ void __launch_bounds__(256) mg_stencil_kernel(int r, const float *__restrict__ S,
                                                         const float *__restrict__ x, const float *__restrict__ b,
                                                         const float *__restrict__ Dinv, float w, int mode,
                                                         float *__restrict__ out, const PcgState *st) {
    pdl_enter();
    if (mg_done(st)) return;
    const unsigned N = (unsigned)r * r * r;
    const int lane = threadIdx.x & 31;
    const unsigned nwarps = (gridDim.x * blockDim.x) >> 5;
    bool act[6];
#pragma unroll
    for (int k = 0; k < 6; ++k) act[k] = !st || st->active[k] != 0;
    const bool live = lane < 27;
    const int dl = live ? lane : 13;
    const int dx = dl % 3 - 1, dy = (dl / 3) % 3 - 1, dz = dl / 9 - 1;
    // the output component this lane ends with, its load case, and the lanes
    // holding the three components of that load case (for the 3x3 Jacobi block)
    const int myid = rs_id(lane);
    const int mk = myid >= 0 ? myid / 3 : 0, mi = myid >= 0 ? myid - 3 * mk : 0;
    int src[3] = {0, 0, 0};
    bool myact = false;
#pragma unroll
    for (int m = 0; m < 18; ++m) {
        const int owner = __ffs(__ballot_sync(0xffffffffu, myid == m)) - 1;
        if (m / 3 == mk) src[m % 3] = owner;
    }
#pragma unroll
    for (int k = 0; k < 6; ++k)
        if (k == mk) myact = act[k] && myid >= 0;
    for (unsigned n = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; n < N; n += nwarps) {
        const int ix = (int)(n % (unsigned)r), iy = (int)((n / (unsigned)r) % (unsigned)r),
                  iz = (int)(n / ((unsigned)r * r));
        const unsigned j = ((unsigned)wrap_l(iz + dz, r) * r + (unsigned)wrap_l(iy + dy, r)) * r + wrap_l(ix + dx, r);
        float B[9];
        const float *Sn = S + ((size_t)n * 27 + dl) * 9;
#pragma unroll
        for (int m = 0; m < 9; ++m) B[m] = live ? __ldg(Sn + m) : 0.0f;
        float acc[18];
#pragma unroll
        for (int k = 0; k < 6; ++k) {
            float x0 = 0.0f, x1 = 0.0f, x2 = 0.0f;
            if (act[k] && live) {
                x0 = x[(size_t)(3 * k) * N + j];
                x1 = x[(size_t)(3 * k + 1) * N + j];
                x2 = x[(size_t)(3 * k + 2) * N + j];
            }
#pragma unroll
            for (int i = 0; i < 3; ++i) acc[3 * k + i] = B[3 * i] * x0 + B[3 * i + 1] * x1 + B[3 * i + 2] * x2;
        }
        const float own = reduce_scatter18(acc, lane);
        const size_t o = (size_t)(myid >= 0 ? myid : 0) * N + n;
        if (mode == 0) {
            if (myact) out[o] = own;
        } else if (mode == 1) {
            if (myact) out[o] = b[o] - own;
        } else {
            const float res = myact ? b[o] - own : 0.0f;
            const float r0 = __shfl_sync(0xffffffffu, res, src[0]), r1 = __shfl_sync(0xffffffffu, res, src[1]),
                        r2 = __shfl_sync(0xffffffffu, res, src[2]);
            if (myact) {
                const float d0 = __ldg(Dinv + (size_t)(3 * mi) * N + n), d1 = __ldg(Dinv + (size_t)(3 * mi + 1) * N + n),
                            d2 = __ldg(Dinv + (size_t)(3 * mi + 2) * N + n);
                out[o] = x[o] + w * (d0 * r0 + d1 * r1 + d2 * r2);
            }
        }
    }
}

// The same stencil, one thread per (node, load case).  A block takes 32
// consecutive nodes and the six load cases (warp w = load case w): it first
// copies the 32 nodes' stencils (contiguous, 31 KB) into shared memory at a
// node pitch of 244 floats, so that every node's record starts on 16 bytes,
// then each thread accumulates its three output components over the 27
// offsets, reading its node's blocks four offsets (36 floats, nine 16-byte
// loads) at a time (pitch 244: the eight lanes of a 16-byte load phase hit
// distinct bank groups), with three coalesced loads of x per offset.  The
// sums are formed in the same order as with one block at a time.
constexpr int kStencilNodes = 32, kStencilPitch = 244;
// ACT (the active set): node groups whose blk byte is 0 take the short path.
template <bool ACT>
__global__ void __launch_bounds__(6 * kStencilNodes) mg_stencil_nc_kernel(int r, const float *__restrict__ S,
                                                                        const float *__restrict__ x,
                                                                        const float *__restrict__ b,
                                                                        const float *__restrict__ Dinv, float w,
                                                                        int mode, float *__restrict__ out,
                                                                        const PcgState *st,
                                                                        const uint8_t *__restrict__ blk) {
    __shared__ __align__(16) float sS[kStencilNodes * kStencilPitch];
    pdl_enter();
    if (mg_done(st)) return;
    const unsigned N = (unsigned)r * r * r;
    const unsigned n0 = blockIdx.x * kStencilNodes;
    const unsigned nn = min((unsigned)kStencilNodes, N - n0);
    if (ACT && !blk[blockIdx.x]) {
        // 32 inactive nodes (active set): zero rows and zero block inverses,
        // so A x = 0 there and the pass reduces to mode 0: 0, 1: b, 2: x
        const int k = threadIdx.x / kStencilNodes, lane = threadIdx.x % kStencilNodes;
        if ((unsigned)lane >= nn || (st && !st->active[k])) return;
        const size_t o = (size_t)(3 * k) * N + n0 + lane;
#pragma unroll
        for (int c = 0; c < 3; ++c)
            out[o + (size_t)c * N] = mode == 0 ? 0.0f : (mode == 1 ? b[o + (size_t)c * N] : x[o + (size_t)c * N]);
        return;
    }
    {
        // 16-byte loads (n0 * 243 floats is a multiple of 4: n0 is a multiple of 32), scattered to the pitch
        const unsigned cnt = nn * 243;
        const float *src = S + (size_t)n0 * 243;
        const float4 *src4 = reinterpret_cast<const float4 *>(src);
        for (unsigned i4 = threadIdx.x; i4 < cnt / 4; i4 += blockDim.x) {
            const float4 v = __ldg(src4 + i4);
            const unsigned i = 4 * i4;
            sS[i + i / 243] = v.x;
            sS[i + 1 + (i + 1) / 243] = v.y;
            sS[i + 2 + (i + 2) / 243] = v.z;
            sS[i + 3 + (i + 3) / 243] = v.w;
        }
        for (unsigned i = (cnt / 4) * 4 + threadIdx.x; i < cnt; i += blockDim.x) sS[i + i / 243] = __ldg(src + i);
    }
    __syncthreads();
    const int k = threadIdx.x / kStencilNodes, lane = threadIdx.x % kStencilNodes;
    if ((unsigned)lane >= nn) return;
    if (st && !st->active[k]) return;
    const unsigned n = n0 + lane;
    const int ix = (int)(n % (unsigned)r), iy = (int)((n / (unsigned)r) % (unsigned)r), iz = (int)(n / ((unsigned)r * r));
    const float *x0p = x + (size_t)(3 * k) * N, *x1p = x0p + N, *x2p = x1p + N;
    unsigned xo[3], yo[3], zo[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        xo[d] = (unsigned)wrap_l(ix + d - 1, r);
        yo[d] = (unsigned)wrap_l(iy + d - 1, r) * (unsigned)r;
        zo[d] = (unsigned)wrap_l(iz + d - 1, r) * (unsigned)r * (unsigned)r;
    }
    const float4 *B4 = reinterpret_cast<const float4 *>(sS + lane * kStencilPitch);
    float a0 = 0.0f, a1 = 0.0f, a2 = 0.0f;
#pragma unroll
    for (int g = 0; g < 7; ++g) {  // offsets 4g .. 4g + 3 (the last group has three)
        constexpr int kMaxQ = 9;
        float bv[4 * kMaxQ];
        const int nq = g < 6 ? 9 : 7;
#pragma unroll
        for (int qi = 0; qi < kMaxQ; ++qi)
            if (qi < nq) {
                const float4 v = B4[g * 9 + qi];
                bv[4 * qi] = v.x, bv[4 * qi + 1] = v.y, bv[4 * qi + 2] = v.z, bv[4 * qi + 3] = v.w;
            }
#pragma unroll
        for (int o = 0; o < 4; ++o) {
            const int dl = 4 * g + o;
            if (dl < 27) {
                const unsigned j = zo[dl / 9] + yo[(dl / 3) % 3] + xo[dl % 3];
                const float v0 = __ldg(x0p + j), v1 = __ldg(x1p + j), v2 = __ldg(x2p + j);
                const float *Bd = bv + o * 9;
                a0 += Bd[0] * v0 + Bd[1] * v1 + Bd[2] * v2;
                a1 += Bd[3] * v0 + Bd[4] * v1 + Bd[5] * v2;
                a2 += Bd[6] * v0 + Bd[7] * v1 + Bd[8] * v2;
            }
        }
    }
    const size_t o = (size_t)(3 * k) * N + n;
    if (mode == 0) {
        out[o] = a0;
        out[o + N] = a1;
        out[o + 2 * (size_t)N] = a2;
        return;
    }
    const float r0 = b[o] - a0, r1 = b[o + N] - a1, r2 = b[o + 2 * (size_t)N] - a2;
    if (mode == 1) {
        out[o] = r0;
        out[o + N] = r1;
        out[o + 2 * (size_t)N] = r2;
        return;
    }
    float D[9];
#pragma unroll
    for (int m = 0; m < 9; ++m) D[m] = __ldg(Dinv + (size_t)m * N + n);
    out[o] = x[o] + w * (D[0] * r0 + D[1] * r1 + D[2] * r2);
    out[o + N] = x[o + N] + w * (D[3] * r0 + D[4] * r1 + D[5] * r2);
    out[o + 2 * (size_t)N] = x[o + 2 * (size_t)N] + w * (D[6] * r0 + D[7] * r1 + D[8] * r2);
}

// One fine plane restricted to coarse node (ix, iy, iz): the weights w(a) of
// the 27 fine neighbours 2I + a (1 on the node, 1/2 per odd offset).  Each of
// the 9 fine rows is read as one 8-byte pair (2ix, 2ix + 1); the left
// neighbour 2ix - 1 is the previous lane's right value when that lane holds
// ix - 1 of the same row.  Every lane of the warp must call it (shuffles).
__device__ __forceinline__ float restrict_plane(const float *__restrict__ bm, const float *__restrict__ tm, int ix,
                                                const unsigned (&zo)[3], const unsigned (&yo)[3], int rf,
                                                bool left_in_warp) {
    float acc = 0.0f;
#pragma unroll
    for (int az = 0; az < 3; ++az)
#pragma unroll
        for (int ay = 0; ay < 3; ++ay) {
            const unsigned row = zo[az] + yo[ay];
            float2 c = *reinterpret_cast<const float2 *>(bm + row + 2 * ix);
            if (tm) {
                const float2 t = *reinterpret_cast<const float2 *>(tm + row + 2 * ix);
                c.x -= t.x;
                c.y -= t.y;
            }
            float left = __shfl_up_sync(0xffffffffu, c.y, 1);
            if (!left_in_warp) {
                const unsigned xl = (unsigned)wrap_l(2 * ix - 1, rf);
                left = tm ? bm[row + xl] - tm[row + xl] : bm[row + xl];
            }
            const float rowsum = c.x + 0.5f * (left + c.y);
            acc += (az == 1 ? 1.0f : 0.5f) * (ay == 1 ? 1.0f : 0.5f) * rowsum;
        }
    return acc;
}

// bc = R (bf - tf): coarse node I gathers w(a) (bf - tf)[2I + a] over its 27
// fine neighbours; tf may be null (bf is then the residual itself).  Grid:
// x over coarse nodes (one per thread), y over the 18 planes.  Converged load
// cases are skipped.
__global__ void __launch_bounds__(256) mg_restrict_kernel(int rc, const float *__restrict__ bf,
                                                          const float *__restrict__ tf, float *__restrict__ bc,
                                                          const PcgState *st, const uint8_t *__restrict__ act_c) {
    pdl_enter();
    if (mg_done(st)) return;
    const int m = blockIdx.y;
    if (st && !st->active[m / 3]) return;
    const unsigned Nc = (unsigned)rc * rc * rc;
    const int rf = 2 * rc;
    const unsigned rrf = (unsigned)rf * rf;
    const size_t Nf = (size_t)rrf * rf;
    const float *bm = bf + (size_t)m * Nf;
    const float *tm = tf ? tf + (size_t)m * Nf : nullptr;
    const int lane = threadIdx.x & 31;
    // every lane runs the same number of iterations (the shuffles need the whole warp)
    const unsigned stride = gridDim.x * blockDim.x;
    const unsigned iters = (Nc + stride - 1) / stride;
    for (unsigned it = 0; it < iters; ++it) {
        const unsigned I = it * stride + blockIdx.x * blockDim.x + threadIdx.x;
        const bool valid = I < Nc;
        const unsigned Iv = valid ? I : 0;
        // a warp of inactive coarse nodes (active set) restricts zeros
        if (act_c && __all_sync(0xffffffffu, !valid || !act_c[Iv])) {
            if (valid) bc[(size_t)m * Nc + I] = 0.0f;
            continue;
        }
        const int ix = (int)(Iv % (unsigned)rc), iy = (int)((Iv / (unsigned)rc) % (unsigned)rc),
                  iz = (int)(Iv / ((unsigned)rc * rc));
        const unsigned zo[3] = {(unsigned)wrap_l(2 * iz - 1, rf) * rrf, (unsigned)(2 * iz) * rrf,
                                (unsigned)wrap_l(2 * iz + 1, rf) * rrf};
        const unsigned yo[3] = {(unsigned)wrap_l(2 * iy - 1, rf) * rf, (unsigned)(2 * iy) * rf,
                                (unsigned)wrap_l(2 * iy + 1, rf) * rf};
        const float acc = restrict_plane(bm, tm, ix, zo, yo, rf, lane > 0 && ix > 0);
        if (valid) bc[(size_t)m * Nc + I] = acc;
    }
}

// The same restriction for the three planes of load case k = grid y, followed
// by the coarse level's first damped block-Jacobi step from a zero iterate,
// xc = w Dc^-1 bc: the down-leg of the V-cycle needs no separate Jacobi launch
// on a coarse level that is smoothed.
__global__ void __launch_bounds__(256) mg_restrict_jacobi_kernel(int rc, const float *__restrict__ bf,
                                                                 const float *__restrict__ tf, float *__restrict__ bc,
                                                                 const float *__restrict__ Dc, float w,
                                                                 float *__restrict__ xc, const PcgState *st,
                                                                 const uint8_t *__restrict__ act_c) {
    pdl_enter();
    if (mg_done(st)) return;
    const int k = blockIdx.y;
    if (st && !st->active[k]) return;
    const unsigned Nc = (unsigned)rc * rc * rc;
    const int rf = 2 * rc;
    const unsigned rrf = (unsigned)rf * rf;
    const size_t Nf = (size_t)rrf * rf;
    const int lane = threadIdx.x & 31;
    const unsigned stride = gridDim.x * blockDim.x;
    const unsigned iters = (Nc + stride - 1) / stride;
    for (unsigned it = 0; it < iters; ++it) {
        const unsigned I = it * stride + blockIdx.x * blockDim.x + threadIdx.x;
        const bool valid = I < Nc;
        const unsigned Iv = valid ? I : 0;
        // a warp of inactive coarse nodes (active set): zero restriction, zero
        // block inverses, so b and x are zero there
        if (act_c && __all_sync(0xffffffffu, !valid || !act_c[Iv])) {
            if (valid)
#pragma unroll
                for (int i = 0; i < 3; ++i) {
                    const size_t o = (size_t)(3 * k + i) * Nc + I;
                    bc[o] = 0.0f;
                    xc[o] = 0.0f;
                }
            continue;
        }
        const int ix = (int)(Iv % (unsigned)rc), iy = (int)((Iv / (unsigned)rc) % (unsigned)rc),
                  iz = (int)(Iv / ((unsigned)rc * rc));
        const unsigned zo[3] = {(unsigned)wrap_l(2 * iz - 1, rf) * rrf, (unsigned)(2 * iz) * rrf,
                                (unsigned)wrap_l(2 * iz + 1, rf) * rrf};
        const unsigned yo[3] = {(unsigned)wrap_l(2 * iy - 1, rf) * rf, (unsigned)(2 * iy) * rf,
                                (unsigned)wrap_l(2 * iy + 1, rf) * rf};
        float b3[3];
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            const size_t m = (size_t)(3 * k + i);
            b3[i] = restrict_plane(bf + m * Nf, tf ? tf + m * Nf : nullptr, ix, zo, yo, rf, lane > 0 && ix > 0);
        }
        if (valid) {
#pragma unroll
            for (int i = 0; i < 3; ++i) {
                const size_t o = (size_t)(3 * k + i) * Nc + I;
                bc[o] = b3[i];
                xc[o] = w * (Dc[(size_t)(3 * i) * Nc + I] * b3[0] + Dc[(size_t)(3 * i + 1) * Nc + I] * b3[1] +
                             Dc[(size_t)(3 * i + 2) * Nc + I] * b3[2]);
            }
        }
    }
}

// xf += P xc (trilinear).  One thread per (plane m = grid y, coarse node C):
// it loads the 8 coarse values of the cell [C, C + 1]^3 once and updates the
// 8 fine nodes 2C + (a, b, c), a, b, c in {0, 1} (odd fine coordinates average
// their two coarse neighbours), two x-neighbours per 8-byte access.
// Converged load cases are skipped; with pin0 the fine node 0 (pinned) is
// left unchanged.
__global__ void __launch_bounds__(256) mg_prolong_kernel(int rc, const float *__restrict__ xc,
                                                         float *__restrict__ xf, int pin0, const PcgState *st,
                                                         const uint8_t *__restrict__ act_c) {
    pdl_enter();
    if (mg_done(st)) return;
    const int m = blockIdx.y;
    if (st && !st->active[m / 3]) return;
    const int rf = 2 * rc;
    const unsigned rrc = (unsigned)rc * rc, Nc = rrc * rc, rrf = (unsigned)rf * rf;
    const float *xm = xc + (size_t)m * Nc;
    float *xo = xf + (size_t)m * rrf * rf;
    for (unsigned I = blockIdx.x * blockDim.x + threadIdx.x; I < Nc; I += gridDim.x * blockDim.x) {
        const int cx = (int)(I % (unsigned)rc), cy = (int)((I / (unsigned)rc) % (unsigned)rc), cz = (int)(I / rrc);
        const unsigned x1 = (unsigned)wrap_l(cx + 1, rc), y0 = (unsigned)cy * rc, y1 = (unsigned)wrap_l(cy + 1, rc) * rc,
                       z0 = (unsigned)cz * rrc, z1 = (unsigned)wrap_l(cz + 1, rc) * rrc;
        // a coarse cell whose 8 corners are inactive (active set) holds x = 0: nothing to add
        if (act_c && !(act_c[z0 + y0 + cx] | act_c[z0 + y0 + x1] | act_c[z0 + y1 + cx] | act_c[z0 + y1 + x1] |
                       act_c[z1 + y0 + cx] | act_c[z1 + y0 + x1] | act_c[z1 + y1 + cx] | act_c[z1 + y1 + x1]))
            continue;
        float e[2][2][2];  // [c][b][x]: the cell's values combined along z and y
#pragma unroll
        for (int xi = 0; xi < 2; ++xi) {
            const unsigned xx = xi ? x1 : (unsigned)cx;
            const float v00 = xm[z0 + y0 + xx], v01 = xm[z0 + y1 + xx], v10 = xm[z1 + y0 + xx], v11 = xm[z1 + y1 + xx];
            e[0][0][xi] = v00;
            e[0][1][xi] = 0.5f * (v00 + v01);
            e[1][0][xi] = 0.5f * (v00 + v10);
            e[1][1][xi] = 0.25f * ((v00 + v01) + (v10 + v11));
        }
#pragma unroll
        for (int c = 0; c < 2; ++c)
#pragma unroll
            for (int b = 0; b < 2; ++b) {
                float2 *f = reinterpret_cast<float2 *>(xo + ((size_t)(2 * cz + c) * rf + (2 * cy + b)) * rf + 2 * cx);
                float2 v = *f;
                if (!(pin0 && I == 0 && c == 0 && b == 0)) v.x += e[c][b][0];
                v.y += 0.5f * (e[c][b][0] + e[c][b][1]);
                *f = v;
            }
    }
}

// ---- lambda_max(D^-1 A) by power iteration (sets the damping per level) ----
// Uses the first three planes (one load case).
__global__ void mg_power_seed_kernel(size_t N, float *x) {
    for (size_t n = blockIdx.x * (size_t)blockDim.x + threadIdx.x; n < 3 * N; n += (size_t)gridDim.x * blockDim.x) {
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
// State of the power iteration: one vector (load case 0), so the coarse
// stencil passes skip the other five.
__global__ void mg_power_state_kernel(PcgState *st) {
    if (threadIdx.x == 0) {
        for (int k = 0; k < 6; ++k) st->active[k] = k == 0;
        st->nactive = 1;
    }
}

// State that gates a V-cycle to the load cases in mask (bit k): the reliable
// update preconditions only the residuals it has just replaced.
__global__ void mg_mask_state_kernel(PcgState *st, int mask) {
    if (threadIdx.x == 0) {
        int na = 0;
        for (int k = 0; k < 6; ++k) {
            st->active[k] = (mask >> k) & 1;
            na += st->active[k];
        }
        st->nactive = na;
    }
}

__global__ void mg_power_scale_kernel(size_t N, const float *y, const double *nrm2, float *x) {
    const float inv = (float)(1.0 / sqrt(nrm2[0] > 0.0 ? nrm2[0] : 1.0));
    for (size_t n = blockIdx.x * (size_t)blockDim.x + threadIdx.x; n < 3 * N; n += (size_t)gridDim.x * blockDim.x)
        x[n] = y[n] * inv;
}

// x = Y^T (Y b) on the coarsest level, Y = L^-1 the inverse Cholesky factor
// of the pinned coarse operator (FP32, lower triangular, the rows and columns
// of node 0 zero).  Y^T Y is positive semi-definite whatever the rounding of
// Y, so the coarse correction cannot make the V-cycle indefinite (an explicit
// FP32 inverse of a badly conditioned coarse operator can).  Two launches,
// w = Y b then x = Y^T w (YT = Y^T row-major), each one warp per (load case,
// row), lanes split the columns of a coalesced row, fixed shuffle tree.
__global__ void mg_dense_y_kernel(int n3, const float *__restrict__ Y, const float *__restrict__ b,
                                  float *__restrict__ w, const PcgState *st) {
    pdl_enter();
    if (mg_done(st)) return;
    const int N = n3 / 3;
    const int lane = threadIdx.x & 31;
    const int nw = (gridDim.x * blockDim.x) >> 5;
    for (int wi = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; wi < 6 * n3; wi += nw) {
        const int k = wi / n3, row = wi - k * n3;
        if (st && !st->active[k]) continue;  // warp-uniform
        const float *bk = b + (size_t)3 * k * N;
        float s = 0.0f;
        for (int col = lane; col <= row; col += 32) s += Y[(size_t)row * n3 + col] * bk[(size_t)(col % 3) * N + col / 3];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (lane == 0) w[wi] = s;
    }
}

__global__ void mg_dense_yt_kernel(int n3, const float *__restrict__ YT, const float *__restrict__ w,
                                   float *__restrict__ x, const PcgState *st) {
    pdl_enter();
    if (mg_done(st)) return;
    const int N = n3 / 3;
    const int lane = threadIdx.x & 31;
    const int nw = (gridDim.x * blockDim.x) >> 5;
    for (int wi = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; wi < 6 * n3; wi += nw) {
        const int k = wi / n3, row = wi - k * n3;
        if (st && !st->active[k]) continue;  // warp-uniform
        const float *wk = w + (size_t)k * n3;
        float s = 0.0f;
        for (int col = (row & ~31) + lane; col < n3; col += 32)
            if (col >= row) s += YT[(size_t)row * n3 + col] * wk[col];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (lane == 0) x[(size_t)(3 * k + row % 3) * N + row / 3] = s;
    }
}

}  // namespace shl
