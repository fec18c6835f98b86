// adjoint.cuh -- hand-written adjoint of C^H through the smoothed density
// (Eq. chain).  For an objective E(C^H) with G = dE/dC^H:
//   g_e    = dE/drho_e = (E - E_void) sum_ij G_ij w_i^T Khat w_j, w = chi + u
//            (chom_kernel in sensitivity mode; the cell problems are
//            self-adjoint, so no adjoint solve is needed)
//   seeds  dE/dd_e = -g_e kappa beta (1 - beta), dE/dt = sum_e g_e kappa beta (1 - beta)
//          Fbar = dE/dd sgn(F - c) / |grad F|,  gFbar = -dE/dd |F - c| grad F / |grad F|^3,
//          dE/dc = -sum_e Fbar
//   field  the separable expansion F = sum_abc A_abc phi_a phi_b phi_c is
//          contracted backwards: per line over x, per plane over y, then over
//          z gives Abar = dE/dA; per charge, A's definition gives
//          dE/dq_j, dE/dx_j (and dE/dalpha_hkl) in O((2K+1)^3).
#pragma once

#include "field.cuh"

namespace shl {

struct SeedArgs {
    size_t N;
    double *F;    // in: F, out: Fbar
    double *gF;   // in: grad F (x,y,z per voxel), out: gFbar
    const double *rho;  // beta_e
    const double *g;    // dE/drho_e through C^H
    double gV;          // dE/dV / N: V = (1/N) sum_e rho_e adds this to every dE/drho_e
    double iso, kappa;
    double *partial;    // [nblocks][3]
    unsigned *ticket;
    double *out;        // [0] dE/dt, [1] dE/dc, [2] V
};

__global__ void adj_seed_kernel(SeedArgs a) {
    double acc[3] = {0.0, 0.0, 0.0};
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < a.N; e += (size_t)gridDim.x * blockDim.x) {
        const double b = a.rho[e];
        const double db = a.kappa * b * (1.0 - b);
        const double ge = a.g[e] + a.gV;
        acc[2] += b;
        acc[0] += ge * db;
        const double dEdd = -ge * db;
        const double F = a.F[e] - a.iso;
        const double gx = a.gF[3 * e], gy = a.gF[3 * e + 1], gz = a.gF[3 * e + 2];
        const double gn2 = gx * gx + gy * gy + gz * gz;
        double fb = 0.0, cg = 0.0;
        if (gn2 > 0.0) {
            const double gn = sqrt(gn2);
            fb = dEdd * (F > 0.0 ? 1.0 : (F < 0.0 ? -1.0 : 0.0)) / gn;
            cg = -dEdd * fabs(F) / (gn2 * gn);
        }
        acc[1] -= fb;
        a.F[e] = fb;
        a.gF[3 * e] = cg * gx;
        a.gF[3 * e + 1] = cg * gy;
        a.gF[3 * e + 2] = cg * gz;
    }
    block_reduce_store<3>(acc, a.partial, blockIdx.x);
    if (!last_block_ticket(a.ticket, gridDim.x)) return;
    __shared__ double tot[3];
    sum_partials_ordered<3>(a.partial, gridDim.x, tot);
    if (threadIdx.x == 0) {
        a.out[0] = tot[0];
        a.out[1] = tot[1];
        a.out[2] = tot[2] / (double)a.N;
    }
}

// One block per z-plane: Q_ab(z) = sum_y [S0_a(y) phi_b(y) + S1_a(y) phi'_b(y)],
// R_ab(z) = sum_y S2_a(y) phi_b(y), with the line sums
// S0_a = sum_x Fbar phi_a(x) + gFbar_x phi'_a(x), S1_a = sum_x gFbar_y phi_a(x),
// S2_a = sum_x gFbar_z phi_a(x).  out: [z][2][nb*nb].
__global__ void adj_plane_kernel(int r, int K, const double *__restrict__ Fb, const double *__restrict__ gFb,
                                 double *__restrict__ out) {
    extern __shared__ double sm[];
    const int nb = 2 * K + 1;
    const int iz = blockIdx.x;
    double *phi = sm;                 // [r][nb]
    double *S = phi + (size_t)r * nb;  // [r][3][nb]
    for (int i = threadIdx.x; i < r; i += blockDim.x) basis_eval((i + 0.5) / r, K, phi + (size_t)i * nb);
    __syncthreads();
    for (int t = threadIdx.x; t < r * nb; t += blockDim.x) {
        const int iy = t / nb, aa = t % nb;
        double s0 = 0.0, s1 = 0.0, s2 = 0.0;
        const size_t row = ((size_t)iz * r + iy) * r;
        for (int ix = 0; ix < r; ++ix) {
            const double *px = phi + (size_t)ix * nb;
            const double p = px[aa], dp = basis_deriv(px, aa, K);
            const size_t e = row + ix;
            s0 += Fb[e] * p + gFb[3 * e] * dp;
            s1 += gFb[3 * e + 1] * p;
            s2 += gFb[3 * e + 2] * p;
        }
        S[((size_t)iy * 3 + 0) * nb + aa] = s0;
        S[((size_t)iy * 3 + 1) * nb + aa] = s1;
        S[((size_t)iy * 3 + 2) * nb + aa] = s2;
    }
    __syncthreads();
    for (int t = threadIdx.x; t < nb * nb; t += blockDim.x) {
        const int aa = t / nb, bb = t % nb;
        double q = 0.0, rr = 0.0;
        for (int iy = 0; iy < r; ++iy) {
            const double *py = phi + (size_t)iy * nb;
            const double p = py[bb], dp = basis_deriv(py, bb, K);
            q += S[((size_t)iy * 3 + 0) * nb + aa] * p + S[((size_t)iy * 3 + 1) * nb + aa] * dp;
            rr += S[((size_t)iy * 3 + 2) * nb + aa] * p;
        }
        out[((size_t)iz * 2 + 0) * nb * nb + t] = q;
        out[((size_t)iz * 2 + 1) * nb * nb + t] = rr;
    }
}

// Abar_abc = sum_z Q_ab(z) phi_c(z) + R_ab(z) phi'_c(z); one block.
__global__ void adj_coef_kernel(int r, int K, const double *__restrict__ QR, double *__restrict__ Abar) {
    extern __shared__ double phi[];  // [r][nb]
    const int nb = 2 * K + 1;
    for (int i = threadIdx.x; i < r; i += blockDim.x) basis_eval((i + 0.5) / r, K, phi + (size_t)i * nb);
    __syncthreads();
    for (int t = threadIdx.x; t < nb * nb * nb; t += blockDim.x) {
        const int ab = t / nb, cc = t % nb;
        double s = 0.0;
        for (int iz = 0; iz < r; ++iz) {
            const double *pz = phi + (size_t)iz * nb;
            s += QR[((size_t)iz * 2 + 0) * nb * nb + ab] * pz[cc] +
                 QR[((size_t)iz * 2 + 1) * nb * nb + ab] * basis_deriv(pz, cc, K);
        }
        Abar[t] = s;
    }
}

__device__ inline double mode_coef(int a, int b, int c, int K, const double *alpha) {
    const int h = basis_freq(a, K), k = basis_freq(b, K), l = basis_freq(c, K);
    if (h + k + l == 0) return 0.0;
    const double al = alpha ? alpha[(h * (K + 1) + k) * (K + 1) + l] : 1.0;
    return al * mode_weight(h, k, l) / (double)(h * h + k * k + l * l);
}

// Per charge j: g_q = sum coef Abar phi phi phi, g_pos = q_j sum coef Abar (phi' phi phi, ...).
__global__ void adj_charge_kernel(int n, int K, const double *__restrict__ pos, const double *__restrict__ q,
                                  const double *__restrict__ alpha, const double *__restrict__ Abar,
                                  double *__restrict__ g_pos, double *__restrict__ g_q) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    const int nb = 2 * K + 1;
    double ph[3][kMaxBasis], dph[3][kMaxBasis];
    for (int d = 0; d < 3; ++d) {
        basis_eval(pos[3 * j + d], K, ph[d]);
        for (int a = 0; a < nb; ++a) dph[d][a] = basis_deriv(ph[d], a, K);
    }
    double gq = 0.0, gx = 0.0, gy = 0.0, gz = 0.0;
    for (int a = 0; a < nb; ++a)
        for (int b = 0; b < nb; ++b)
            for (int c = 0; c < nb; ++c) {
                const double w = mode_coef(a, b, c, K, alpha) * Abar[(a * nb + b) * nb + c];
                if (w == 0.0) continue;
                gq += w * ph[0][a] * ph[1][b] * ph[2][c];
                gx += w * dph[0][a] * ph[1][b] * ph[2][c];
                gy += w * ph[0][a] * dph[1][b] * ph[2][c];
                gz += w * ph[0][a] * ph[1][b] * dph[2][c];
            }
    g_q[j] = gq;
    g_pos[3 * j] = q[j] * gx;
    g_pos[3 * j + 1] = q[j] * gy;
    g_pos[3 * j + 2] = q[j] * gz;
}

// dE/dalpha_hkl = w_hkl/|n|^2 sum over the (a,b,c) of frequency (h,k,l) of
// Abar_abc sum_j q_j phi_a phi_b phi_c; one block, thread per (h,k,l).
__global__ void adj_alpha_kernel(int n, int K, const double *__restrict__ pos, const double *__restrict__ q,
                                 const double *__restrict__ Abar, double *__restrict__ g_alpha) {
    const int K1 = K + 1, nb = 2 * K + 1;
    for (int t = threadIdx.x; t < K1 * K1 * K1; t += blockDim.x) {
        const int h = t / (K1 * K1), k = (t / K1) % K1, l = t % K1;
        double s = 0.0;
        if (h + k + l > 0) {
            const int as[2] = {h, h ? K + h : -1}, bs[2] = {k, k ? K + k : -1}, cs[2] = {l, l ? K + l : -1};
            for (int j = 0; j < n; ++j) {
                double ph[3][kMaxBasis];
                for (int d = 0; d < 3; ++d) basis_eval(pos[3 * j + d], K, ph[d]);
                for (int ia = 0; ia < 2; ++ia)
                    for (int ib = 0; ib < 2; ++ib)
                        for (int ic = 0; ic < 2; ++ic) {
                            const int a = as[ia], b = bs[ib], c = cs[ic];
                            if (a < 0 || b < 0 || c < 0) continue;
                            s += q[j] * ph[0][a] * ph[1][b] * ph[2][c] * Abar[(a * nb + b) * nb + c];
                        }
            }
            s *= mode_weight(h, k, l) / (double)(h * h + k * k + l * l);
        }
        g_alpha[t] = s;
    }
}

}  // namespace shl
