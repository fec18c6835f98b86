/*
 * shl_oracle.c -- plain FP64 CPU oracle for periodic elastic homogenisation of
 * charge-parametrised shells (arXiv 2511.04025).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, obviously-correct
 * reference against which the CUDA library is checked.  Only the test suite,
 * the smoke check and the benchmark's CPU-baseline leg load it.  It shares no
 * code, header or constant with the CUDA path.
 *
 * Everything is IEEE double, built without fast-math and without FMA
 * contraction.  OpenMP only splits independent outputs (points, rows,
 * elements) across threads; every reduction is summed in a fixed order, so
 * results do not depend on the thread count (except shlo_field_vjp, whose
 * per-thread partial sums make its last bits depend on it).
 *
 * Conventions (shared with the CUDA library by definition, not by code):
 *   - unit cell [0,1)^3, r voxels per axis, h = 1/r;
 *   - element e = (iz*r + iy)*r + ix owns local nodes
 *       (0,0,0),(1,0,0),(1,1,0),(0,1,0),(0,0,1),(1,0,1),(1,1,1),(0,1,1)
 *     offset from grid node (ix,iy,iz), wrapped periodically;
 *   - node n = (iz*r + iy)*r + ix sits at (ix/r, iy/r, iz/r);
 *   - oracle node vectors are AoS: v[(k*N + n)*3 + i], load case k, DOF i;
 *   - Voigt order 11,22,33,23,13,12 with engineering shear strains.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define SHLO_PI 3.14159265358979323846264338327950288

/* ------------------------------------------------------------------------- */
/* Field (Sec. 3.1, Eq. charge-field; weights w_hkl from Eq. inf-series).    */
/* ------------------------------------------------------------------------- */

/* w_hkl: 1/2 if exactly one index is zero, 1/4 if two are zero (Eq.
 * inf-series); 1 when none is zero (each |h|,|k|,|l| term of the full
 * lattice sum then has 8 sign images, against 4 and 2 for one and two zero
 * indices, so the relative weights are 1 : 1/2 : 1/4). */
static double shlo_weight(int h, int k, int l) {
    int zeros = (h == 0) + (k == 0) + (l == 0);
    if (zeros == 0) return 1.0;
    if (zeros == 1) return 0.5;
    if (zeros == 2) return 0.25;
    return 0.0; /* B_000 = 0 (truncated series) */
}

/*
 * F(p) = sum_{h,k,l=0..K} alpha_hkl w_hkl sum_j q_j B_hkl(p, p_j)
 * B_hkl = cos(2 pi h (x-xj)) cos(2 pi k (y-yj)) cos(2 pi l (z-zj)) / (h^2+k^2+l^2)
 * and its analytic gradient.  alpha is indexed [h][k][l] with (K+1)^3 entries
 * (NULL means all ones).  pts is npts x 3; F is npts; gF is npts x 3 or NULL.
 * Each 1-D cosine/sine factor is one libm call per (point, charge, axis,
 * order); B_hkl is their product.
 */
int shlo_field(int nc, const double *pos, const double *q, const double *alpha, int K,
               long npts, const double *pts, double *F, double *gF) {
    if (nc < 0 || K < 1 || K > 15 || npts < 0) return 1;
    const int K1 = K + 1;
    int st = 0;
#pragma omp parallel
    {
        /* per point: the 1-D factors cos/sin(2 pi n (x_d - x_{j,d})), n = 0..K */
        double *cs = (double *)malloc(sizeof(double) * (nc > 0 ? nc : 1) * 3 * K1);
        double *sn = (double *)malloc(sizeof(double) * (nc > 0 ? nc : 1) * 3 * K1);
        if (!cs || !sn) st = 2;
#pragma omp for schedule(static)
        for (long p = 0; p < npts; ++p) {
            if (!cs || !sn) continue;
            for (int j = 0; j < nc; ++j)
                for (int d = 0; d < 3; ++d)
                    for (int n = 0; n <= K; ++n) {
                        const double a = 2.0 * SHLO_PI * n * (pts[3 * p + d] - pos[3 * j + d]);
                        cs[(j * 3 + d) * K1 + n] = cos(a);
                        sn[(j * 3 + d) * K1 + n] = sin(a);
                    }
            double f = 0.0, gx = 0.0, gy = 0.0, gz = 0.0;
            for (int h = 0; h <= K; ++h)
                for (int k = 0; k <= K; ++k)
                    for (int l = 0; l <= K; ++l) {
                        if (h == 0 && k == 0 && l == 0) continue;
                        const double a = alpha ? alpha[(h * K1 + k) * K1 + l] : 1.0;
                        const double coef = a * shlo_weight(h, k, l) / (double)(h * h + k * k + l * l);
                        double sf = 0.0, sgx = 0.0, sgy = 0.0, sgz = 0.0;
                        for (int j = 0; j < nc; ++j) {
                            const double cx = cs[(j * 3 + 0) * K1 + h], sx = sn[(j * 3 + 0) * K1 + h];
                            const double cy = cs[(j * 3 + 1) * K1 + k], sy = sn[(j * 3 + 1) * K1 + k];
                            const double cz = cs[(j * 3 + 2) * K1 + l], sz = sn[(j * 3 + 2) * K1 + l];
                            sf += q[j] * (cx * cy * cz);
                            sgx += q[j] * (-2.0 * SHLO_PI * h * sx * cy * cz);
                            sgy += q[j] * (-2.0 * SHLO_PI * k * cx * sy * cz);
                            sgz += q[j] * (-2.0 * SHLO_PI * l * cx * cy * sz);
                        }
                        f += coef * sf;
                        gx += coef * sgx;
                        gy += coef * sgy;
                        gz += coef * sgz;
                    }
            F[p] = f;
            if (gF) {
                gF[3 * p] = gx;
                gF[3 * p + 1] = gy;
                gF[3 * p + 2] = gz;
            }
        }
        free(cs);
        free(sn);
    }
    return st;
}

/*
 * Per-charge parameter derivatives of F and grad F at one point, for the
 * chain rule of Eq. chain:
 *   dF/dq_j, dF/dx_j (3), d(gradF)/dq_j (3), d(gradF)/dx_j (3x3, row = grad
 *   component, column = charge coordinate).
 * Output per charge j (16 doubles): [dF/dq, dF/dxj(3), dG/dq(3), dG/dxj(9)].
 * dF/dx_j = -(dF/dx restricted to charge j), d gradF/dx_j = -(Hessian
 * restricted to charge j), both by the chain rule on (x - x_j).
 */
int shlo_field_param_derivs(int nc, const double *pos, const double *q, const double *alpha, int K,
                            const double *pt, double *out) {
    if (nc < 0 || K < 1 || K > 15) return 1;
    const int K1 = K + 1;
    for (int j = 0; j < nc; ++j) {
        double b = 0.0, g[3] = {0, 0, 0}, H[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
        for (int h = 0; h <= K; ++h)
            for (int k = 0; k <= K; ++k)
                for (int l = 0; l <= K; ++l) {
                    if (h == 0 && k == 0 && l == 0) continue;
                    const double a = alpha ? alpha[(h * K1 + k) * K1 + l] : 1.0;
                    const double coef = a * shlo_weight(h, k, l) / (double)(h * h + k * k + l * l);
                    const double wx = 2.0 * SHLO_PI * h, wy = 2.0 * SHLO_PI * k, wz = 2.0 * SHLO_PI * l;
                    const double ax = wx * (pt[0] - pos[3 * j]);
                    const double ay = wy * (pt[1] - pos[3 * j + 1]);
                    const double az = wz * (pt[2] - pos[3 * j + 2]);
                    const double cx = cos(ax), cy = cos(ay), cz = cos(az);
                    const double sx = sin(ax), sy = sin(ay), sz = sin(az);
                    b += coef * cx * cy * cz;
                    g[0] += coef * (-wx * sx * cy * cz);
                    g[1] += coef * (-wy * cx * sy * cz);
                    g[2] += coef * (-wz * cx * cy * sz);
                    H[0] += coef * (-wx * wx * cx * cy * cz);
                    H[1] += coef * (wx * wy * sx * sy * cz);
                    H[2] += coef * (wx * wz * sx * cy * sz);
                    H[4] += coef * (-wy * wy * cx * cy * cz);
                    H[5] += coef * (wy * wz * cx * sy * sz);
                    H[8] += coef * (-wz * wz * cx * cy * cz);
                }
        H[3] = H[1];
        H[6] = H[2];
        H[7] = H[5];
        double *o = out + 16 * j;
        o[0] = b;                                  /* dF/dq_j            */
        for (int i = 0; i < 3; ++i) o[1 + i] = -q[j] * g[i]; /* dF/dx_j */
        for (int i = 0; i < 3; ++i) o[4 + i] = g[i];         /* dG/dq_j */
        for (int i = 0; i < 9; ++i) o[7 + i] = -q[j] * H[i]; /* dG_i/dx_j,m */
    }
    return 0;
}

/* ------------------------------------------------------------------------- */
/* Element stiffness K0 (Sec. 4.1: one stiffness shared by all voxels).      */
/* ------------------------------------------------------------------------- */

static const int shlo_corner[8][3] = {{0, 0, 0}, {1, 0, 0}, {1, 1, 0}, {0, 1, 0},
                                      {0, 0, 1}, {1, 0, 1}, {1, 1, 1}, {0, 1, 1}};

/* Isotropic elasticity matrix, Voigt order 11,22,33,23,13,12, engineering shear. */
static void shlo_D(double E, double nu, double D[6][6]) {
    const double lam = E * nu / ((1.0 + nu) * (1.0 - 2.0 * nu));
    const double mu = E / (2.0 * (1.0 + nu));
    memset(D, 0, sizeof(double) * 36);
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) D[i][j] = lam + (i == j ? 2.0 * mu : 0.0);
    D[3][3] = D[4][4] = D[5][5] = mu;
}

/*
 * 24x24 stiffness of the 8-node trilinear hexahedron on the cube [0,h]^3,
 * DOF 3*a+i (local node a, displacement component i), integrated with the
 * 2x2x2 Gauss rule (exact for this element):
 *   K = sum_gp B^T D B * |J| w_gp.
 */
int shlo_element_stiffness(double E, double nu, double h, double *Ke) {
    if (!(h > 0.0)) return 1;
    double D[6][6];
    shlo_D(E, nu, D);
    const double g = 0.5 / sqrt(3.0);
    const double gp[2] = {0.5 - g, 0.5 + g}; /* Gauss points on [0,1] */
    memset(Ke, 0, sizeof(double) * 24 * 24);
    for (int gi = 0; gi < 8; ++gi) {
        const double xi[3] = {gp[gi & 1], gp[(gi >> 1) & 1], gp[(gi >> 2) & 1]};
        /* shape-function derivatives dN_a/dx_d on [0,h]^3 */
        double dN[8][3];
        for (int a = 0; a < 8; ++a) {
            double f[3], df[3];
            for (int d = 0; d < 3; ++d) {
                f[d] = shlo_corner[a][d] ? xi[d] : 1.0 - xi[d];
                df[d] = shlo_corner[a][d] ? 1.0 : -1.0;
            }
            dN[a][0] = df[0] * f[1] * f[2] / h;
            dN[a][1] = f[0] * df[1] * f[2] / h;
            dN[a][2] = f[0] * f[1] * df[2] / h;
        }
        double B[6][24];
        memset(B, 0, sizeof(B));
        for (int a = 0; a < 8; ++a) {
            B[0][3 * a + 0] = dN[a][0];
            B[1][3 * a + 1] = dN[a][1];
            B[2][3 * a + 2] = dN[a][2];
            B[3][3 * a + 1] = dN[a][2];
            B[3][3 * a + 2] = dN[a][1];
            B[4][3 * a + 0] = dN[a][2];
            B[4][3 * a + 2] = dN[a][0];
            B[5][3 * a + 0] = dN[a][1];
            B[5][3 * a + 1] = dN[a][0];
        }
        const double w = h * h * h / 8.0; /* |J| times Gauss weight */
        for (int m = 0; m < 24; ++m)
            for (int n = 0; n < 24; ++n) {
                double s = 0.0;
                for (int p = 0; p < 6; ++p)
                    for (int qq = 0; qq < 6; ++qq) s += B[p][m] * D[p][qq] * B[qq][n];
                Ke[m * 24 + n] += s * w;
            }
    }
    return 0;
}

/* Test displacement chi^k at the element's local nodes (Eq. inv-design):
 * chi_i = sum_j eps^(k)_ij X_j, X_a = h * corner(a), unit Voigt strain k. */
static void shlo_chi(int k, double h, double chi[24]) {
    double eps[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
    switch (k) {
    case 0: eps[0][0] = 1.0; break;
    case 1: eps[1][1] = 1.0; break;
    case 2: eps[2][2] = 1.0; break;
    case 3: eps[1][2] = eps[2][1] = 0.5; break;
    case 4: eps[0][2] = eps[2][0] = 0.5; break;
    case 5: eps[0][1] = eps[1][0] = 0.5; break;
    }
    for (int a = 0; a < 8; ++a)
        for (int i = 0; i < 3; ++i) {
            double s = 0.0;
            for (int j = 0; j < 3; ++j) s += eps[i][j] * h * shlo_corner[a][j];
            chi[3 * a + i] = s;
        }
}

int shlo_test_displacement(int k, double h, double *chi) {
    if (k < 0 || k > 5) return 1;
    shlo_chi(k, h, chi);
    return 0;
}

/* ------------------------------------------------------------------------- */
/* Assembled periodic stiffness (block CSR of 3x3 blocks).                   */
/* ------------------------------------------------------------------------- */

typedef struct {
    int r;
    long nn;      /* nodes = r^3 */
    long *rowptr; /* nn+1 */
    long *col;    /* block columns */
    double *val;  /* 9 per block, row-major */
} shlo_bsr;

static long shlo_node(int r, long ix, long iy, long iz) {
    ix = ((ix % r) + r) % r;
    iy = ((iy % r) + r) % r;
    iz = ((iz % r) + r) % r;
    return (iz * r + iy) * r + ix;
}

static int shlo_cmp_long(const void *a, const void *b) {
    long x = *(const long *)a, y = *(const long *)b;
    return (x > y) - (x < y);
}

/* E_e = E_void + rho_e (E - E_void) (ersatz void floor, binary or smooth rho). */
static double shlo_modulus(double rho, double E, double Evoid) { return Evoid + rho * (E - Evoid); }

/*
 * K = sum_e E_e * Khat scattered with periodic node wrap, where Khat is the
 * unit-modulus element stiffness on [0,h]^3.  Built row by row (each row
 * gathers from its 8 incident elements), duplicate columns (r <= 2) merged.
 */
static int shlo_assemble(int r, const double *rho, double E, double nu, double Evoid, shlo_bsr *A) {
    const long N = (long)r * r * r;
    double Ke[576];
    shlo_element_stiffness(1.0, nu, 1.0 / r, Ke);
    A->r = r;
    A->nn = N;
    A->rowptr = (long *)malloc(sizeof(long) * (N + 1));
    if (!A->rowptr) return 2;
    /* distinct neighbour count per row (27 for r >= 3) */
    int nb = (r >= 3) ? 27 : (r == 2 ? 8 : 1);
    A->col = (long *)malloc(sizeof(long) * N * nb);
    A->val = (double *)calloc((size_t)N * nb * 9, sizeof(double));
    if (!A->col || !A->val) return 2;
    for (long n = 0; n <= N; ++n) A->rowptr[n] = n * nb;
#pragma omp parallel for schedule(static)
    for (long n = 0; n < N; ++n) {
        const long ix = n % r, iy = (n / r) % r, iz = n / ((long)r * r);
        long nbrs[27];
        int m = 0;
        for (int dz = -1; dz <= 1; ++dz)
            for (int dy = -1; dy <= 1; ++dy)
                for (int dx = -1; dx <= 1; ++dx) nbrs[m++] = shlo_node(r, ix + dx, iy + dy, iz + dz);
        qsort(nbrs, 27, sizeof(long), shlo_cmp_long);
        int u = 0;
        for (int i = 0; i < 27; ++i)
            if (u == 0 || nbrs[i] != nbrs[u - 1]) nbrs[u++] = nbrs[i];
        long *cols = A->col + A->rowptr[n];
        double *vals = A->val + 9 * A->rowptr[n];
        for (int i = 0; i < u; ++i) cols[i] = nbrs[i];
        /* elements incident to node n: node n is local corner a of element
         * (ix - cx, iy - cy, iz - cz) */
        for (int a = 0; a < 8; ++a) {
            const long ex = ix - shlo_corner[a][0], ey = iy - shlo_corner[a][1], ez = iz - shlo_corner[a][2];
            const long e = shlo_node(r, ex, ey, ez);
            const double Ee = shlo_modulus(rho[e], E, Evoid);
            for (int b = 0; b < 8; ++b) {
                const long nb_node = shlo_node(r, ex + shlo_corner[b][0], ey + shlo_corner[b][1], ez + shlo_corner[b][2]);
                int slot = -1;
                for (int i = 0; i < u; ++i)
                    if (cols[i] == nb_node) slot = i;
                for (int i = 0; i < 3; ++i)
                    for (int j = 0; j < 3; ++j) vals[9 * slot + 3 * i + j] += Ee * Ke[(3 * a + i) * 24 + 3 * b + j];
            }
        }
    }
    return 0;
}

static void shlo_free(shlo_bsr *A) {
    free(A->rowptr);
    free(A->col);
    free(A->val);
}

/* y = A x for nvec node vectors (AoS per vector). */
static void shlo_spmv(const shlo_bsr *A, int nvec, const double *x, double *y) {
    const long N = A->nn;
#pragma omp parallel for schedule(static)
    for (long n = 0; n < N; ++n) {
        for (int v = 0; v < nvec; ++v) {
            double s[3] = {0, 0, 0};
            for (long b = A->rowptr[n]; b < A->rowptr[n + 1]; ++b) {
                const double *blk = A->val + 9 * b;
                const double *xv = x + ((long)v * N + A->col[b]) * 3;
                for (int i = 0; i < 3; ++i) s[i] += blk[3 * i] * xv[0] + blk[3 * i + 1] * xv[1] + blk[3 * i + 2] * xv[2];
            }
            for (int i = 0; i < 3; ++i) y[((long)v * N + n) * 3 + i] = s[i];
        }
    }
}

/* Fixed-order dot product over len entries (chunked, chunks summed in order). */
static double shlo_dot(long len, const double *a, const double *b) {
    const long CH = 4096;
    const long nch = (len + CH - 1) / CH;
    double *part = (double *)malloc(sizeof(double) * (nch > 0 ? nch : 1));
#pragma omp parallel for schedule(static)
    for (long c = 0; c < nch; ++c) {
        double s = 0.0;
        const long hi = (c + 1) * CH < len ? (c + 1) * CH : len;
        for (long i = c * CH; i < hi; ++i) s += a[i] * b[i];
        part[c] = s;
    }
    double s = 0.0;
    for (long c = 0; c < nch; ++c) s += part[c];
    free(part);
    return s;
}

int shlo_apply(int r, const double *rho, double E, double nu, double Evoid, int nvec, const double *x, double *y) {
    if (r < 1 || nvec < 0) return 1;
    shlo_bsr A;
    int st = shlo_assemble(r, rho, E, nu, Evoid, &A);
    if (st) return st;
    shlo_spmv(&A, nvec, x, y);
    shlo_free(&A);
    return 0;
}

/* f^(k) = - sum_e K_e chi^k (Eq. inv-design, load of cell problem k). */
int shlo_rhs(int r, const double *rho, double E, double nu, double Evoid, double *f) {
    if (r < 1) return 1;
    const long N = (long)r * r * r;
    double Ke[576], Kchi[6][24];
    const double h = 1.0 / r;
    shlo_element_stiffness(1.0, nu, h, Ke);
    for (int k = 0; k < 6; ++k) {
        double chi[24];
        shlo_chi(k, h, chi);
        for (int m = 0; m < 24; ++m) {
            double s = 0.0;
            for (int n = 0; n < 24; ++n) s += Ke[m * 24 + n] * chi[n];
            Kchi[k][m] = s;
        }
    }
#pragma omp parallel for schedule(static)
    for (long n = 0; n < N; ++n) {
        const long ix = n % r, iy = (n / r) % r, iz = n / ((long)r * r);
        for (int k = 0; k < 6; ++k) {
            double s[3] = {0, 0, 0};
            for (int a = 0; a < 8; ++a) {
                const long e = shlo_node(r, ix - shlo_corner[a][0], iy - shlo_corner[a][1], iz - shlo_corner[a][2]);
                const double Ee = shlo_modulus(rho[e], E, Evoid);
                for (int i = 0; i < 3; ++i) s[i] -= Ee * Kchi[k][3 * a + i];
            }
            for (int i = 0; i < 3; ++i) f[((long)k * N + n) * 3 + i] = s[i];
        }
    }
    return 0;
}

/*
 * Solve K u^(k) = f^(k), k = 1..6, with node pin_node pinned (its three DOFs
 * removed: zero rows/columns, unit diagonal, zero load), by Jacobi-
 * preconditioned CG in FP64.  A node whose diagonal block is zero (every
 * incident element has zero stiffness: outside the active set of Sec. 4.2.1)
 * is removed the same way, so its displacement stays 0.  All six load cases
 * share each SpMV; each has its own CG scalars and stops once
 * ||f - K u||_2 / ||f||_2 <= tol (the recurrence residual).  relres returns
 * the true residual of the pinned system after the solve; iters the
 * iterations each case used.  Returns 0, or 3 if some case hit maxit.
 */
int shlo_solve_ex(int r, const double *rho, double E, double nu, double Evoid, long pin_node, double tol, int maxit,
                  double *u, int *iters, double *relres) {
    if (r < 1 || !(tol > 0.0) || maxit < 0) return 1;
    const long N = (long)r * r * r;
    const long L = 3 * N;
    if (pin_node < 0 || pin_node >= N) return 1;
    shlo_bsr A;
    int st = shlo_assemble(r, rho, E, nu, Evoid, &A);
    if (st) return st;
    double *f = (double *)malloc(sizeof(double) * 6 * L);
    shlo_rhs(r, rho, E, nu, Evoid, f);

    /* removed nodes: the pin and every node with a zero diagonal block */
    char *gone = (char *)calloc((size_t)N, 1);
    gone[pin_node] = 1;
    for (long n = 0; n < N; ++n)
        for (long b = A.rowptr[n]; b < A.rowptr[n + 1]; ++b)
            if (A.col[b] == n) {
                int zero = 1;
                for (int i = 0; i < 9; ++i) zero &= (A.val[9 * b + i] == 0.0);
                if (zero) gone[n] = 1;
            }
    /* pinned copy of the operator */
    shlo_bsr P = A;
    P.val = (double *)malloc(sizeof(double) * 9 * A.rowptr[N]);
    memcpy(P.val, A.val, sizeof(double) * 9 * A.rowptr[N]);
    for (long n = 0; n < N; ++n)
        for (long b = P.rowptr[n]; b < P.rowptr[n + 1]; ++b) {
            if (gone[n] || gone[P.col[b]]) {
                for (int i = 0; i < 9; ++i) P.val[9 * b + i] = 0.0;
                if (P.col[b] == n) P.val[9 * b] = P.val[9 * b + 4] = P.val[9 * b + 8] = 1.0;
            }
        }
    double *fp = (double *)malloc(sizeof(double) * 6 * L);
    memcpy(fp, f, sizeof(double) * 6 * L);
    for (int k = 0; k < 6; ++k)
        for (long n = 0; n < N; ++n)
            if (gone[n])
                for (int i = 0; i < 3; ++i) fp[k * L + 3 * n + i] = 0.0;
    free(gone);

    /* Jacobi preconditioner: inverse diagonal of the pinned operator */
    double *dinv = (double *)malloc(sizeof(double) * L);
    for (long n = 0; n < N; ++n)
        for (long b = P.rowptr[n]; b < P.rowptr[n + 1]; ++b)
            if (P.col[b] == n)
                for (int i = 0; i < 3; ++i) dinv[3 * n + i] = 1.0 / P.val[9 * b + 4 * i];

    double *res = (double *)malloc(sizeof(double) * 6 * L);
    double *z = (double *)malloc(sizeof(double) * 6 * L);
    double *p = (double *)malloc(sizeof(double) * 6 * L);
    double *q = (double *)malloc(sizeof(double) * 6 * L);
    double rz[6], fn[6];
    int done[6];
    memset(u, 0, sizeof(double) * 6 * L);
    memcpy(res, fp, sizeof(double) * 6 * L);
    for (int k = 0; k < 6; ++k) {
        for (long i = 0; i < L; ++i) z[k * L + i] = dinv[i] * res[k * L + i];
        memcpy(p + k * L, z + k * L, sizeof(double) * L);
        rz[k] = shlo_dot(L, res + k * L, z + k * L);
        fn[k] = sqrt(shlo_dot(L, fp + k * L, fp + k * L));
        done[k] = (fn[k] == 0.0);
        iters[k] = 0;
    }
    int it = 0;
    for (; it < maxit; ++it) {
        int all = 1;
        for (int k = 0; k < 6; ++k) all &= done[k];
        if (all) break;
        shlo_spmv(&P, 6, p, q);
        for (int k = 0; k < 6; ++k) {
            if (done[k]) continue;
            double *uk = u + k * L, *rk = res + k * L, *pk = p + k * L, *qk = q + k * L, *zk = z + k * L;
            const double alpha = rz[k] / shlo_dot(L, pk, qk);
            for (long i = 0; i < L; ++i) {
                uk[i] += alpha * pk[i];
                rk[i] -= alpha * qk[i];
            }
            iters[k] = it + 1;
            if (sqrt(shlo_dot(L, rk, rk)) <= tol * fn[k]) {
                done[k] = 1;
                continue;
            }
            for (long i = 0; i < L; ++i) zk[i] = dinv[i] * rk[i];
            const double rz_new = shlo_dot(L, rk, zk);
            const double beta = rz_new / rz[k];
            rz[k] = rz_new;
            for (long i = 0; i < L; ++i) pk[i] = zk[i] + beta * pk[i];
        }
    }
    int all = 1;
    for (int k = 0; k < 6; ++k) all &= done[k];

    /* true residual of the pinned system (the system CG solves) */
    shlo_spmv(&P, 6, u, q);
    for (int k = 0; k < 6; ++k) {
        for (long i = 0; i < L; ++i) q[k * L + i] = fp[k * L + i] - q[k * L + i];
        const double fnk = sqrt(shlo_dot(L, fp + k * L, fp + k * L));
        const double rn = sqrt(shlo_dot(L, q + k * L, q + k * L));
        relres[k] = fnk > 0.0 ? rn / fnk : rn;
    }
    free(res); free(z); free(p); free(q); free(dinv); free(fp); free(f);
    free(P.val);
    shlo_free(&A);
    return all ? 0 : 3;
}

/* The ersatz-void problem: node 0 pinned. */
int shlo_solve(int r, const double *rho, double E, double nu, double Evoid, double tol, int maxit, double *u,
               int *iters, double *relres) {
    return shlo_solve_ex(r, rho, E, nu, Evoid, 0, tol, maxit, u, iters, relres);
}

/*
 * C^H_ij = (1/|Y|) sum_e (chi^i + u^i_e)^T K_e (chi^j + u^j_e), |Y| = 1
 * (Eq. inv-design).  C (36, row-major) is that energy form; Calt (36, may be
 * NULL) is sum_e chi^i^T K_e (chi^j + u^j_e), equal to C when K u = f.
 * Per-element terms are summed in element order.
 */
int shlo_chom(int r, const double *rho, double E, double nu, double Evoid, const double *u, double *C, double *Calt) {
    if (r < 1) return 1;
    const long N = (long)r * r * r;
    const double h = 1.0 / r;
    double Ke[576], chi[6][24];
    shlo_element_stiffness(1.0, nu, h, Ke);
    for (int k = 0; k < 6; ++k) shlo_chi(k, h, chi[k]);
    const long CH = 1024;
    const long nch = (N + CH - 1) / CH;
    double *part = (double *)calloc((size_t)nch * 72, sizeof(double));
#pragma omp parallel for schedule(static)
    for (long c = 0; c < nch; ++c) {
        double *pc = part + 72 * c;
        const long hi = (c + 1) * CH < N ? (c + 1) * CH : N;
        for (long e = c * CH; e < hi; ++e) {
            const long ix = e % r, iy = (e / r) % r, iz = e / ((long)r * r);
            const double Ee = shlo_modulus(rho[e], E, Evoid);
            double w[6][24], Kw[6][24];
            for (int k = 0; k < 6; ++k)
                for (int a = 0; a < 8; ++a) {
                    const long n = shlo_node(r, ix + shlo_corner[a][0], iy + shlo_corner[a][1], iz + shlo_corner[a][2]);
                    for (int i = 0; i < 3; ++i) w[k][3 * a + i] = chi[k][3 * a + i] + u[((long)k * N + n) * 3 + i];
                }
            for (int k = 0; k < 6; ++k)
                for (int m = 0; m < 24; ++m) {
                    double s = 0.0;
                    for (int n2 = 0; n2 < 24; ++n2) s += Ke[m * 24 + n2] * w[k][n2];
                    Kw[k][m] = s;
                }
            for (int i = 0; i < 6; ++i)
                for (int j = 0; j < 6; ++j) {
                    double s = 0.0, s2 = 0.0;
                    for (int m = 0; m < 24; ++m) {
                        s += w[i][m] * Kw[j][m];
                        s2 += chi[i][m] * Kw[j][m];
                    }
                    pc[6 * i + j] += Ee * s;
                    pc[36 + 6 * i + j] += Ee * s2;
                }
        }
    }
    for (int i = 0; i < 36; ++i) {
        double s = 0.0, s2 = 0.0;
        for (long c = 0; c < nch; ++c) {
            s += part[72 * c + i];
            s2 += part[72 * c + 36 + i];
        }
        C[i] = s;
        if (Calt) Calt[i] = s2;
    }
    free(part);
    return 0;
}

/*
 * Element sensitivity of the energy form (Eq. chain, the "standard"
 * topology-optimisation term): for each element e,
 *   g_e = sum_ij G_ij (E - E_void) (chi^i + u^i_e)^T Khat (chi^j + u^j_e),
 * i.e. dE/drho_e for an objective with dE/dC^H = G (36, row-major), using
 * that each cell problem is self-adjoint and u^(k) is in equilibrium.
 */
int shlo_element_sensitivity(int r, double E, double nu, double Evoid, const double *u, const double *G, double *g) {
    if (r < 1) return 1;
    const long N = (long)r * r * r;
    const double h = 1.0 / r;
    double Ke[576], chi[6][24];
    shlo_element_stiffness(1.0, nu, h, Ke);
    for (int k = 0; k < 6; ++k) shlo_chi(k, h, chi[k]);
#pragma omp parallel for schedule(static)
    for (long e = 0; e < N; ++e) {
        const long ix = e % r, iy = (e / r) % r, iz = e / ((long)r * r);
        double w[6][24], Kw[6][24];
        for (int k = 0; k < 6; ++k)
            for (int a = 0; a < 8; ++a) {
                const long n = shlo_node(r, ix + shlo_corner[a][0], iy + shlo_corner[a][1], iz + shlo_corner[a][2]);
                for (int i = 0; i < 3; ++i) w[k][3 * a + i] = chi[k][3 * a + i] + u[((long)k * N + n) * 3 + i];
            }
        for (int k = 0; k < 6; ++k)
            for (int m = 0; m < 24; ++m) {
                double s = 0.0;
                for (int n2 = 0; n2 < 24; ++n2) s += Ke[m * 24 + n2] * w[k][n2];
                Kw[k][m] = s;
            }
        double s = 0.0;
        for (int i = 0; i < 6; ++i)
            for (int j = 0; j < 6; ++j) {
                double wk = 0.0;
                for (int m = 0; m < 24; ++m) wk += w[i][m] * Kw[j][m];
                s += G[6 * i + j] * wk;
            }
        g[e] = (E - Evoid) * s;
    }
    return 0;
}

int shlo_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/*
 * Vector-Jacobian product of the field (chain rule of Eq. chain through F and
 * grad F): given per-point seeds Fbar = dE/dF(p) and gFbar = dE/d(grad F)(p),
 *   g_q[j]   += sum_p Fbar dF/dq_j + gFbar . d(grad F)/dq_j
 *   g_pos[j] += sum_p Fbar dF/dx_j + gFbar . d(grad F)/dx_j
 * where, for B_j(p) = sum_hkl alpha w / |n|^2 cos cos cos (charge j's basis
 * sum), F = sum_j q_j B_j, dF/dq_j = B_j, d(grad F)/dq_j = grad B_j,
 * dF/dx_j = -q_j grad B_j and d(grad F)_a/dx_jm = -q_j d_a d_m B_j (every
 * factor depends on p - p_j).
 * With g_alpha (K+1)^3 given (NULL: not computed), also the mode weights of
 * Sec. 4.3: F is linear in alpha_hkl with
 *   dF/dalpha_hkl       = w_hkl/(h^2+k^2+l^2) sum_j q_j cos cos cos
 *   d(grad F)/dalpha_hkl = w_hkl/(h^2+k^2+l^2) sum_j q_j grad(cos cos cos)
 * so g_alpha[hkl] = sum_p Fbar dF/dalpha_hkl + gFbar . d(grad F)/dalpha_hkl
 * (g_alpha[000] = 0: the constant mode is not in the truncated series).
 * Points are split across threads; per-thread partial sums are added in
 * thread order.
 */
int shlo_field_vjp(int nc, const double *pos, const double *q, const double *alpha, int K, long npts,
                   const double *pts, const double *Fbar, const double *gFbar, double *g_pos, double *g_q,
                   double *g_alpha) {
    if (nc < 0 || K < 1 || K > 15 || npts < 0) return 1;
    const int K1 = K + 1;
    int nthr = 1;
#ifdef _OPENMP
    nthr = omp_get_max_threads();
#endif
    const int nmode = K1 * K1 * K1;
    const size_t per_thr = (size_t)nc * 4 + (size_t)nmode;
    double *acc = (double *)calloc((size_t)nthr * per_thr, sizeof(double));
    if (!acc) return 2;
#pragma omp parallel
    {
        int tid = 0;
#ifdef _OPENMP
        tid = omp_get_thread_num();
#endif
        double *my = acc + (size_t)tid * per_thr;
        double *my_alpha = my + (size_t)nc * 4;
        double cs[3][16], sn[3][16];
#pragma omp for schedule(static)
        for (long p = 0; p < npts; ++p) {
            for (int j = 0; j < nc; ++j) {
                for (int d = 0; d < 3; ++d)
                    for (int n = 0; n <= K; ++n) {
                        const double a = 2.0 * SHLO_PI * n * (pts[3 * p + d] - pos[3 * j + d]);
                        cs[d][n] = cos(a);
                        sn[d][n] = sin(a);
                    }
                double B = 0.0, g[3] = {0, 0, 0}, H[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
                for (int h = 0; h <= K; ++h)
                    for (int k = 0; k <= K; ++k)
                        for (int l = 0; l <= K; ++l) {
                            if (h == 0 && k == 0 && l == 0) continue;
                            const double a = alpha ? alpha[(h * K1 + k) * K1 + l] : 1.0;
                            const double coef0 = shlo_weight(h, k, l) / (double)(h * h + k * k + l * l);
                            const double coef = a * coef0;
                            const double w[3] = {2.0 * SHLO_PI * h, 2.0 * SHLO_PI * k, 2.0 * SHLO_PI * l};
                            const int nn[3] = {h, k, l};
                            double c[3], s[3];
                            for (int d = 0; d < 3; ++d) {
                                c[d] = cs[d][nn[d]];
                                s[d] = sn[d][nn[d]];
                            }
                            const double bj = c[0] * c[1] * c[2];
                            double gj[3];
                            B += coef * bj;
                            for (int d = 0; d < 3; ++d) {
                                double t = -w[d] * s[d];
                                for (int e = 0; e < 3; ++e)
                                    if (e != d) t *= c[e];
                                gj[d] = t;
                                g[d] += coef * t;
                            }
                            if (g_alpha) {
                                /* this charge's share of dE/dalpha_hkl at point p */
                                const double *gbp = gFbar + 3 * p;
                                my_alpha[(h * K1 + k) * K1 + l] +=
                                    q[j] * coef0 * (Fbar[p] * bj + gbp[0] * gj[0] + gbp[1] * gj[1] + gbp[2] * gj[2]);
                            }
                            for (int d = 0; d < 3; ++d)
                                for (int m = 0; m < 3; ++m) {
                                    double t;
                                    if (d == m) {
                                        t = -w[d] * w[d] * c[0] * c[1] * c[2];
                                    } else {
                                        const int o = 3 - d - m;
                                        t = w[d] * s[d] * w[m] * s[m] * c[o];
                                    }
                                    H[d][m] += coef * t;
                                }
                        }
                const double fb = Fbar[p];
                const double *gb = gFbar + 3 * p;
                my[4 * j + 0] += fb * B + gb[0] * g[0] + gb[1] * g[1] + gb[2] * g[2];
                for (int m = 0; m < 3; ++m) {
                    double t = fb * g[m];
                    for (int a2 = 0; a2 < 3; ++a2) t += gb[a2] * H[a2][m];
                    my[4 * j + 1 + m] += -q[j] * t;
                }
            }
        }
    }
    for (int j = 0; j < nc; ++j) {
        g_q[j] = 0.0;
        g_pos[3 * j] = g_pos[3 * j + 1] = g_pos[3 * j + 2] = 0.0;
        for (int t = 0; t < nthr; ++t) {
            const double *my = acc + (size_t)t * per_thr;
            g_q[j] += my[4 * j];
            for (int m = 0; m < 3; ++m) g_pos[3 * j + m] += my[4 * j + 1 + m];
        }
    }
    if (g_alpha) {
        for (int m = 0; m < nmode; ++m) {
            g_alpha[m] = 0.0;
            for (int t = 0; t < nthr; ++t) g_alpha[m] += acc[(size_t)t * per_thr + (size_t)nc * 4 + m];
        }
    }
    free(acc);
    return 0;
}
