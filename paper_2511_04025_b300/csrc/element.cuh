// element.cuh -- the hex8 voxel element operator of libshl.
//
// Sec. 4.1: every voxel shares one stiffness K_0 (E = 1), scaled per element,
// K_e = E_e Khat.  Khat is the 8-node trilinear hexahedron on [0,h]^3 with
// 2x2x2 Gauss integration (exact for this element), so Khat = h * K_unit.
//
// Kernel form.  Inside a kernel the element's nodes use binary order
// b = cx + 2 cy + 4 cz and the displacement is held per component as v[i][b].
// The Walsh-Hadamard transform over the 8 corners, H_mb = (-1)^popcount(m&b),
// diagonalises the cube's three reflections.  A reflection about the element
// centre along axis d flips corner bit d and the sign of component d, so the
// transformed DOF (m, i) has character chi = m XOR e_i under the reflection
// group (Z_2)^3.  Khat commutes with the group, hence
//     G = (1/64) H Khat H^T   (H = H8 (x) I3)
// is block diagonal: 8 characters x one 3x3 block coupling
// (chi^e_0, x), (chi^e_1, y), (chi^e_2, z).  An element apply y = Khat v is
// then y = H (G (H v)): 2 x 3 eight-point butterflies (72 add/sub) and eight
// 3x3 blocks (72 FMA) instead of a dense 24x24 product (576 FMA).
#pragma once

#include "common.cuh"

namespace shl {

// Operator constants for one grid size r and Poisson ratio nu (E = 1).
template <typename T>
struct ElemOp {
    T G[8][3][3];       // h * unit-cube blocks, G[chi][i][j]
    T chihat[6][3][8];  // H chi^k (element-local test displacement, side h), [k][i][m]
    T kchi[6][3][8];    // Khat chi^k in binary node order, [k][i][b]
    T diag;             // Khat[(b,i),(b,i)] (same for every b, i)
};

// ---------------------------------------------------------------------------
// Host construction
// ---------------------------------------------------------------------------

// Unit-cube hex8 stiffness, E = 1, binary node order, DOF 3*b + i.
inline void unit_hex8_stiffness(double nu, double K[24][24]) {
    const double lam = nu / ((1.0 + nu) * (1.0 - 2.0 * nu));
    const double mu = 1.0 / (2.0 * (1.0 + nu));
    const double gq[2] = {0.5 - 0.5 / std::sqrt(3.0), 0.5 + 0.5 / std::sqrt(3.0)};
    std::memset(K, 0, sizeof(double) * 576);
    for (int g = 0; g < 8; ++g) {
        const double p[3] = {gq[g & 1], gq[(g >> 1) & 1], gq[(g >> 2) & 1]};
        double dN[8][3];  // dN_b / dx_d
        for (int b = 0; b < 8; ++b) {
            for (int d = 0; d < 3; ++d) {
                double prod = ((b >> d) & 1) ? 1.0 : -1.0;
                for (int e = 0; e < 3; ++e)
                    if (e != d) prod *= ((b >> e) & 1) ? p[e] : 1.0 - p[e];
                dN[b][d] = prod;
            }
        }
        // bilinear form: lam div u div v + mu (grad u : grad v + grad u : grad v^T)
        for (int a = 0; a < 8; ++a)
            for (int i = 0; i < 3; ++i)
                for (int b = 0; b < 8; ++b)
                    for (int j = 0; j < 3; ++j) {
                        double v = lam * dN[a][i] * dN[b][j] + mu * dN[a][j] * dN[b][i];
                        if (i == j) v += mu * (dN[a][0] * dN[b][0] + dN[a][1] * dN[b][1] + dN[a][2] * dN[b][2]);
                        K[3 * a + i][3 * b + j] += v / 8.0;  // Gauss weight on the unit cube
                    }
    }
}

// Unit Voigt strain k (11,22,33,23,13,12; engineering shear) as a tensor.
inline void voigt_unit_strain(int k, double eps[3][3]) {
    std::memset(eps, 0, sizeof(double) * 9);
    static const int a[6] = {0, 1, 2, 1, 0, 0}, b[6] = {0, 1, 2, 2, 2, 1};
    if (k < 3)
        eps[k][k] = 1.0;
    else
        eps[a[k]][b[k]] = eps[b[k]][a[k]] = 0.5;
}

// Non-zero pattern of the transformed blocks G[c][i][j] of the isotropic
// hex8 element (the same for every Poisson ratio; at nu = 0 some entries
// vanish as well): row i of block c as a bit mask over j.  45 of the 72
// block entries; the rows of the three translation modes are zero (a rigid
// translation carries no force).  build_elem_op checks it.
__host__ __device__ constexpr bool g_nz(int c, int i, int j) {
    constexpr unsigned char rows[8][3] = {{7, 7, 7}, {0, 6, 6}, {5, 0, 5}, {3, 3, 4},
                                          {3, 3, 0}, {5, 2, 5}, {1, 6, 6}, {7, 7, 7}};
    return (rows[c][i] >> j) & 1;
}
__host__ __device__ constexpr bool g_row_nz(int c, int i) { return g_nz(c, i, 0) || g_nz(c, i, 1) || g_nz(c, i, 2); }

// Builds the operator; returns the largest entry of G outside its block and
// non-zero pattern relative to max |G| (round-off level when the structure
// holds).
template <typename T>
inline double build_elem_op(double nu, int r, ElemOp<T> *op) {
    double Ku[24][24];
    unit_hex8_stiffness(nu, Ku);
    const double h = 1.0 / r;
    double H[8][8];
    for (int m = 0; m < 8; ++m)
        for (int b = 0; b < 8; ++b) H[m][b] = (__builtin_popcount(m & b) & 1) ? -1.0 : 1.0;
    double Gf[24][24];
    double gmax = 0.0;
    for (int m = 0; m < 8; ++m)
        for (int i = 0; i < 3; ++i)
            for (int n = 0; n < 8; ++n)
                for (int j = 0; j < 3; ++j) {
                    double s = 0.0;
                    for (int a = 0; a < 8; ++a)
                        for (int b = 0; b < 8; ++b) s += H[m][a] * Ku[3 * a + i][3 * b + j] * H[n][b];
                    Gf[3 * m + i][3 * n + j] = s / 64.0;
                    gmax = std::fmax(gmax, std::fabs(s / 64.0));
                }
    double off = 0.0;
    for (int m = 0; m < 8; ++m)
        for (int i = 0; i < 3; ++i)
            for (int n = 0; n < 8; ++n)
                for (int j = 0; j < 3; ++j) {
                    const int cb = m ^ (1 << i);  // block of row (m, i)
                    const bool in_block = cb == (n ^ (1 << j));
                    if (!in_block || !g_nz(cb, i, j)) off = std::fmax(off, std::fabs(Gf[3 * m + i][3 * n + j]));
                }
    for (int c = 0; c < 8; ++c)
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) op->G[c][i][j] = (T)(h * Gf[3 * (c ^ (1 << i)) + i][3 * (c ^ (1 << j)) + j]);
    // test displacements chi^k on [0,h]^3 and their transforms / loads
    for (int k = 0; k < 6; ++k) {
        double eps[3][3];
        voigt_unit_strain(k, eps);
        double chi[8][3];
        for (int b = 0; b < 8; ++b)
            for (int i = 0; i < 3; ++i) {
                double s = 0.0;
                for (int d = 0; d < 3; ++d) s += eps[i][d] * h * ((b >> d) & 1);
                chi[b][i] = s;
            }
        for (int i = 0; i < 3; ++i)
            for (int m = 0; m < 8; ++m) {
                double s = 0.0;
                for (int b = 0; b < 8; ++b) s += H[m][b] * chi[b][i];
                op->chihat[k][i][m] = (T)s;
            }
        for (int b = 0; b < 8; ++b)
            for (int i = 0; i < 3; ++i) {
                double s = 0.0;
                for (int a = 0; a < 8; ++a)
                    for (int j = 0; j < 3; ++j) s += h * Ku[3 * b + i][3 * a + j] * chi[a][j];
                op->kchi[k][i][b] = (T)s;
            }
    }
    op->diag = (T)(h * Ku[0][0]);
    return off / gmax;
}

// ---------------------------------------------------------------------------
// Device side
// ---------------------------------------------------------------------------

// In-place 8-point Walsh-Hadamard butterfly, natural order.
template <typename T>
__device__ __forceinline__ void wht8(T (&v)[8]) {
#pragma unroll
    for (int s = 1; s < 8; s <<= 1)
#pragma unroll
        for (int b = 0; b < 8; ++b)
            if (!(b & s)) {
                const T a = v[b], c = v[b | s];
                v[b] = a + c;
                v[b | s] = a - c;
            }
}

// y = scale * G u in the transformed basis (u, y: [component][mode]); only
// the entries of the non-zero pattern are multiplied (45 of 72).
template <typename T>
__device__ __forceinline__ void block_apply(const ElemOp<T> &op, const T (&u)[3][8], T (&y)[3][8], T scale) {
#pragma unroll
    for (int c = 0; c < 8; ++c) {
        const T a[3] = {u[0][c ^ 1], u[1][c ^ 2], u[2][c ^ 4]};
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            if (!g_row_nz(c, i)) {
                y[i][c ^ (1 << i)] = T(0);
                continue;
            }
            T s = T(0);
            bool first = true;
#pragma unroll
            for (int j = 0; j < 3; ++j)
                if (g_nz(c, i, j)) {
                    s = first ? op.G[c][i][j] * a[j] : s + op.G[c][i][j] * a[j];
                    first = false;
                }
            y[i][c ^ (1 << i)] = scale * s;
        }
    }
}

}  // namespace shl
