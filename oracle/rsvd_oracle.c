/*
 * FP64 CPU oracle for the randomized SVD of Erichson, Voronin, Brunton and
 * Kutz, "Randomized Matrix Decompositions Using R" (arXiv:1608.02148).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the plain, slow, obviously correct
 * statement of what the GPU library computes.  It is compiled into its own
 * shared object and is called only by the tests, by the smoke check and by
 * the CPU-baseline leg of the benchmark.  It shares no code, header, table or
 * constant generator with the CUDA library, and the CUDA library never calls
 * it.
 *
 * Everything is computed in IEEE double precision.  Inputs stored as FP32 or
 * BF16 are promoted exactly.  The only library primitives used are the C math
 * functions (sqrt, log, sin, cos).  Matrix products are naive loops; QR is
 * Householder; the SVD of the small factor is one-sided (Hestenes) Jacobi.
 *
 * Layout convention: every matrix is row-major with an explicit leading
 * dimension unless a comment says otherwise.
 *
 * Parity status: every exported function is pinned by the CPU tests (exact
 * rank, brute force against LAPACK on tiny inputs, Eckart-Young, the expected
 * error bound of Eq. (rsvd_expected_error), the power identity of Sec. 2.2.2,
 * the Pythagorean error identities, invariances, and distributional checks of
 * the Philox/Box-Muller test matrix).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ------------------------------------------------------------------------ */
/* Test matrix Omega (Sec. 2.3; Algorithm rqb step 2).                      */
/*                                                                          */
/* The paper draws Omega with R's rnorm and fixes no generator.  Reading    */
/* taken here: Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11), a         */
/* counter-based generator, so that any implementation can reproduce the    */
/* same integer stream element by element.                                  */
/*   key     = (seed & 0xffffffff, seed >> 32)                              */
/*   counter = (r & 0xffffffff, r >> 32, j, 0)   with r = i / 4              */
/* gives four 32-bit words x0..x3 that feed rows 4r..4r+3 of column j.      */
/* ------------------------------------------------------------------------ */

/* One Philox round: two 32x32->64 multiplications by the published
 * multipliers, a word permutation and the key injection. */
static void philox_round(uint32_t c[4], const uint32_t k[2])
{
    const uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)c[0];
    const uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)c[2];
    const uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    const uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    uint32_t n0 = hi1 ^ c[1] ^ k[0];
    uint32_t n1 = lo1;
    uint32_t n2 = hi0 ^ c[3] ^ k[1];
    uint32_t n3 = lo0;
    c[0] = n0; c[1] = n1; c[2] = n2; c[3] = n3;
}

/* Ten rounds; the key is bumped by the Weyl constants between rounds. */
void oracle_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t c[4] = {ctr[0], ctr[1], ctr[2], ctr[3]};
    uint32_t k[2] = {key[0], key[1]};
    for (int round = 0; round < 10; ++round) {
        if (round > 0) {
            k[0] += 0x9E3779B9u;
            k[1] += 0xBB67AE85u;
        }
        philox_round(c, k);
    }
    out[0] = c[0]; out[1] = c[1]; out[2] = c[2]; out[3] = c[3];
}

enum { SDIST_NORMAL = 0, SDIST_UNIF = 1, SDIST_RADEMACHER = 2 };

/* Uniform on (0,1) from a 32-bit word: (x + 1/2) / 2^32. */
static double word_to_open_unit(uint32_t x) { return ((double)x + 0.5) * (1.0 / 4294967296.0); }

/*
 * Fill Omega (rows x l, row-major, leading dimension ld) with the test matrix
 * of Sec. 2.3:
 *   normal     : Box-Muller on the word pairs (x0,x1) -> rows 4r, 4r+1 and
 *                (x2,x3) -> rows 4r+2, 4r+3:  rad = sqrt(-2 ln u_a),
 *                theta = 2 pi u_b, values rad*cos(theta), rad*sin(theta);
 *   unif       : 2u - 1 on (-1, 1), row 4r+t uses x_t;
 *   rademacher : +1 if bit 31 of x_t is clear, else -1.
 * Each value is computed in double and rounded to the nearest float; those
 * float values ARE Omega.  Column j only depends on j, so the columns of a
 * wider Omega extend a narrower one (nested in l).
 */
void oracle_omega(int64_t rows, int64_t l, uint64_t seed, int sdist, float* out, int64_t ld)
{
    const uint32_t key[2] = {(uint32_t)(seed & 0xffffffffu), (uint32_t)(seed >> 32)};
    const double two_pi = 6.283185307179586;
    const int64_t nblk = (rows + 3) / 4;
#pragma omp parallel for schedule(static)
    for (int64_t r = 0; r < nblk; ++r) {
        for (int64_t j = 0; j < l; ++j) {
            const uint32_t ctr[4] = {(uint32_t)((uint64_t)r & 0xffffffffu), (uint32_t)((uint64_t)r >> 32),
                                     (uint32_t)j, 0u};
            uint32_t x[4];
            oracle_philox4x32_10(ctr, key, x);
            double v[4];
            if (sdist == SDIST_NORMAL) {
                for (int h = 0; h < 2; ++h) {
                    const double ua = word_to_open_unit(x[2 * h]);
                    const double ub = word_to_open_unit(x[2 * h + 1]);
                    const double rad = sqrt(-2.0 * log(ua));
                    const double theta = two_pi * ub;
                    v[2 * h] = rad * cos(theta);
                    v[2 * h + 1] = rad * sin(theta);
                }
            } else if (sdist == SDIST_UNIF) {
                for (int t = 0; t < 4; ++t) v[t] = 2.0 * word_to_open_unit(x[t]) - 1.0;
            } else {
                for (int t = 0; t < 4; ++t) v[t] = (x[t] & 0x80000000u) ? -1.0 : 1.0;
            }
            for (int t = 0; t < 4; ++t) {
                const int64_t i = 4 * r + t;
                if (i < rows) out[i * ld + j] = (float)v[t];
            }
        }
    }
}

/* ------------------------------------------------------------------------ */
/* Read access to the input matrix A (Sec. 3.6: the m x n data matrix).     */
/* The stored values (FP32, BF16 or FP64) are promoted exactly to double.   */
/* When trans is set, the logical matrix is the transpose of the stored one */
/* (used when m < n: the method is applied to A^T and U, V are swapped).    */
/* ------------------------------------------------------------------------ */
enum { DT_F32 = 0, DT_BF16 = 1, DT_F64 = 2 };

typedef struct {
    const void* data;
    int dtype;
    int64_t rows, cols; /* logical shape */
    int64_t ld;         /* leading dimension of the STORED row-major matrix */
    int trans;          /* logical(i,j) = stored(j,i) when set */
} amat;

static inline double stored_elem(const amat* A, int64_t r, int64_t c)
{
    const int64_t off = r * A->ld + c;
    if (A->dtype == DT_F32) return (double)((const float*)A->data)[off];
    if (A->dtype == DT_F64) return ((const double*)A->data)[off];
    /* BF16: the 16 stored bits are the high half of an IEEE float. */
    const uint32_t bits = (uint32_t)((const uint16_t*)A->data)[off] << 16;
    float f;
    memcpy(&f, &bits, sizeof f);
    return (double)f;
}

static inline double aget(const amat* A, int64_t i, int64_t j)
{
    return A->trans ? stored_elem(A, j, i) : stored_elem(A, i, j);
}

/* Y (rows x l) = A X with X (cols x l); both row-major, leading dim l.
 * Naive triple loop (Algorithm rqb step 3, Algorithm sub_iterations step 4). */
static void gemm_AX(const amat* A, const double* X, int64_t l, double* Y)
{
    const int64_t m = A->rows, n = A->cols;
#pragma omp parallel
    {
        double* arow = (double*)malloc((size_t)n * sizeof(double));
#pragma omp for schedule(static)
        for (int64_t i = 0; i < m; ++i) {
            for (int64_t t = 0; t < n; ++t) arow[t] = aget(A, i, t);
            double* y = Y + i * l;
            for (int64_t j = 0; j < l; ++j) y[j] = 0.0;
            for (int64_t t = 0; t < n; ++t) {
                const double a = arow[t];
                const double* x = X + t * l;
                for (int64_t j = 0; j < l; ++j) y[j] += a * x[j];
            }
        }
        free(arow);
    }
}

/* Z (cols x l) = A^T X with X (rows x l).  Z(t,j) = sum_i A(i,t) X(i,j),
 * summed over i in increasing order (Algorithm sub_iterations step 3 and
 * Algorithm rqb step 10, since B = Q^T A = (A^T Q)^T).  Threads own disjoint
 * ranges of t. */
static void gemm_AtX(const amat* A, const double* X, int64_t l, double* Z)
{
    const int64_t m = A->rows, n = A->cols;
    for (int64_t e = 0; e < n * l; ++e) Z[e] = 0.0;
#pragma omp parallel
    {
        int nth = 1, tid = 0;
#ifdef _OPENMP
        nth = omp_get_num_threads();
        tid = omp_get_thread_num();
#endif
        const int64_t t0 = n * tid / nth, t1 = n * (tid + 1) / nth;
        for (int64_t i = 0; i < m; ++i) {
            const double* x = X + i * l;
            for (int64_t t = t0; t < t1; ++t) {
                const double a = aget(A, i, t);
                double* z = Z + t * l;
                for (int64_t j = 0; j < l; ++j) z[j] += a * x[j];
            }
        }
    }
}

/* ------------------------------------------------------------------------ */
/* Economic Householder QR (the "qr" of Algorithm sub_iterations steps 2-3  */
/* and Algorithm rqb step 9).  Y is m x l row-major (m >= l).  Returns Q    */
/* (m x l, orthonormal columns) and optionally R (l x l upper triangular).  */
/* Reflector j maps column j of the current trailing block onto            */
/* -sign(x_0) ||x|| e_1.                                                    */
/* ------------------------------------------------------------------------ */
int oracle_householder_qr(int64_t m, int64_t l, const double* Y, double* Q, double* R)
{
    if (m < l || l < 1) return 1;
    /* Column-major working copy W (column c starts at W + c*m). */
    double* W = (double*)malloc((size_t)(m * l) * sizeof(double));
    double* V = (double*)calloc((size_t)(m * l), sizeof(double)); /* reflector j in column j */
    double* rdiag = (double*)malloc((size_t)l * sizeof(double));
    if (!W || !V || !rdiag) { free(W); free(V); free(rdiag); return 2; }
    for (int64_t i = 0; i < m; ++i)
        for (int64_t c = 0; c < l; ++c) W[c * m + i] = Y[i * l + c];

    for (int64_t j = 0; j < l; ++j) {
        double* x = W + j * m;
        double nrm2 = 0.0;
        for (int64_t i = j; i < m; ++i) nrm2 += x[i] * x[i];
        const double nrm = sqrt(nrm2);
        double* v = V + j * m;
        if (nrm == 0.0) { /* zero column: identity reflector, R(j,j) = 0 */
            rdiag[j] = 0.0;
            continue;
        }
        const double alpha = (x[j] >= 0.0) ? -nrm : nrm;
        for (int64_t i = j; i < m; ++i) v[i] = x[i];
        v[j] -= alpha;
        double vn2 = 0.0;
        for (int64_t i = j; i < m; ++i) vn2 += v[i] * v[i];
        const double vn = sqrt(vn2);
        for (int64_t i = j; i < m; ++i) v[i] /= vn;
        rdiag[j] = alpha;
        x[j] = alpha;
        for (int64_t i = j + 1; i < m; ++i) x[i] = 0.0;
        /* Apply H = I - 2 v v^T to the trailing columns. */
#pragma omp parallel for schedule(static)
        for (int64_t c = j + 1; c < l; ++c) {
            double* w = W + c * m;
            double dot = 0.0;
            for (int64_t i = j; i < m; ++i) dot += v[i] * w[i];
            for (int64_t i = j; i < m; ++i) w[i] -= 2.0 * dot * v[i];
        }
    }
    if (R) {
        for (int64_t r = 0; r < l; ++r)
            for (int64_t c = 0; c < l; ++c) R[r * l + c] = (c >= r) ? W[c * m + r] : 0.0;
        for (int64_t r = 0; r < l; ++r) R[r * l + r] = rdiag[r];
    }
    /* Q = H_0 H_1 ... H_{l-1} [I_l; 0]: apply the reflectors in reverse
     * order to the first l columns of the identity. */
    double* Qc = W; /* reuse storage, column-major */
    for (int64_t c = 0; c < l; ++c)
        for (int64_t i = 0; i < m; ++i) Qc[c * m + i] = (i == c) ? 1.0 : 0.0;
    for (int64_t j = l - 1; j >= 0; --j) {
        const double* v = V + j * m;
        if (rdiag[j] == 0.0) continue;
#pragma omp parallel for schedule(static)
        for (int64_t c = 0; c < l; ++c) {
            double* w = Qc + c * m;
            double dot = 0.0;
            for (int64_t i = j; i < m; ++i) dot += v[i] * w[i];
            for (int64_t i = j; i < m; ++i) w[i] -= 2.0 * dot * v[i];
        }
    }
    for (int64_t i = 0; i < m; ++i)
        for (int64_t c = 0; c < l; ++c) Q[i * l + c] = Qc[c * m + i];
    free(W); free(V); free(rdiag);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* One-sided (Hestenes) Jacobi SVD, the "deterministic algorithm" used for  */
/* the small matrix in Algorithm rSVD step 2.  M is rows x cols row-major   */
/* with rows >= cols.  Plane rotations J are applied on the right until all */
/* column pairs are orthogonal to |a_i.a_j| <= 1e-15 ||a_i|| ||a_j||; then  */
/* M J = W has orthogonal columns, s_i = ||w_i||, Ucols = W / s, and        */
/* M = Ucols diag(s) J^T.  Outputs are sorted by descending s:              */
/*   s (cols), Ucols (rows x cols, row-major), J (cols x cols, row-major).  */
/* Returns the number of sweeps used, or -1 if 100 sweeps did not suffice.  */
/* ------------------------------------------------------------------------ */
int oracle_jacobi_svd(int64_t rows, int64_t cols, const double* M, double* s, double* Ucols, double* J)
{
    if (rows < cols || cols < 1) return -2;
    double* W = (double*)malloc((size_t)(rows * cols) * sizeof(double)); /* column-major */
    double* V = (double*)malloc((size_t)(cols * cols) * sizeof(double)); /* column-major */
    double* sv = (double*)malloc((size_t)cols * sizeof(double));
    int64_t* order = (int64_t*)malloc((size_t)cols * sizeof(int64_t));
    for (int64_t i = 0; i < rows; ++i)
        for (int64_t c = 0; c < cols; ++c) W[c * rows + i] = M[i * cols + c];
    for (int64_t i = 0; i < cols; ++i)
        for (int64_t c = 0; c < cols; ++c) V[c * cols + i] = (i == c) ? 1.0 : 0.0;

    const double tol = 1e-15;
    int sweeps = 0, converged = 0;
    while (!converged && sweeps < 100) {
        converged = 1;
        ++sweeps;
        for (int64_t a = 0; a < cols - 1; ++a) {
            for (int64_t b = a + 1; b < cols; ++b) {
                double* wa = W + a * rows;
                double* wb = W + b * rows;
                double alpha = 0.0, beta = 0.0, gamma = 0.0;
                for (int64_t i = 0; i < rows; ++i) {
                    alpha += wa[i] * wa[i];
                    beta += wb[i] * wb[i];
                    gamma += wa[i] * wb[i];
                }
                if (gamma == 0.0 || fabs(gamma) <= tol * sqrt(alpha * beta)) continue;
                converged = 0;
                /* Rotation that zeroes the off-diagonal entry of the 2x2 Gram
                 * [[alpha, gamma], [gamma, beta]]: t is the smaller root of
                 * t^2 + 2 zeta t - 1 = 0 with zeta = (beta - alpha) / (2 gamma). */
                const double zeta = (beta - alpha) / (2.0 * gamma);
                const double t = ((zeta >= 0.0) ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
                const double c = 1.0 / sqrt(1.0 + t * t);
                const double sn = c * t;
                for (int64_t i = 0; i < rows; ++i) {
                    const double x = wa[i], y = wb[i];
                    wa[i] = c * x - sn * y;
                    wb[i] = sn * x + c * y;
                }
                double* va = V + a * cols;
                double* vb = V + b * cols;
                for (int64_t i = 0; i < cols; ++i) {
                    const double x = va[i], y = vb[i];
                    va[i] = c * x - sn * y;
                    vb[i] = sn * x + c * y;
                }
            }
        }
    }
    for (int64_t c = 0; c < cols; ++c) {
        double nrm2 = 0.0;
        for (int64_t i = 0; i < rows; ++i) nrm2 += W[c * rows + i] * W[c * rows + i];
        sv[c] = sqrt(nrm2);
        order[c] = c;
    }
    /* Insertion sort of the column order by descending singular value
     * (stable: equal values keep their index order). */
    for (int64_t c = 1; c < cols; ++c) {
        const int64_t key = order[c];
        int64_t d = c - 1;
        while (d >= 0 && sv[order[d]] < sv[key]) {
            order[d + 1] = order[d];
            --d;
        }
        order[d + 1] = key;
    }
    for (int64_t c = 0; c < cols; ++c) {
        const int64_t src = order[c];
        s[c] = sv[src];
        for (int64_t i = 0; i < rows; ++i)
            Ucols[i * cols + c] = (sv[src] > 0.0) ? W[src * rows + i] / sv[src] : 0.0;
        for (int64_t i = 0; i < cols; ++i) J[i * cols + c] = V[src * cols + i];
    }
    free(W); free(V); free(sv); free(order);
    return converged ? sweeps : -1;
}

/*
 * Pivoted LU of a tall m x l matrix (m >= l), [L, U] = lu(Y) in the sense of
 * Algorithm norm_iterations (Sec. 2.2.2): Gaussian elimination with partial
 * (row) pivoting, the pivot of column j being the first row, in the current
 * order, of largest magnitude at or below j.  Y = L U with L (m x l) a row
 * permutation of a unit lower trapezoidal matrix, returned in Y's own row
 * order, and U (l x l) upper triangular.  perm[j] (optional) is the row of Y
 * chosen as pivot j.  A zero pivot (a column already in the span of the
 * earlier ones) leaves that column of L zero below its pivot row and U's
 * diagonal entry zero.  U and perm may be NULL.  Returns 0 (2: no memory).
 */
int oracle_lu_pivot(int64_t m, int64_t l, const double* Y, double* L, double* U, int64_t* perm)
{
    if (m < l || l < 1) return 1;
    double* W = (double*)malloc((size_t)(m * l) * sizeof(double));
    int64_t* row = (int64_t*)malloc((size_t)m * sizeof(int64_t));
    if (!W || !row) { free(W); free(row); return 2; }
    memcpy(W, Y, (size_t)(m * l) * sizeof(double));
    for (int64_t i = 0; i < m; ++i) row[i] = i;
    for (int64_t j = 0; j < l; ++j) {
        int64_t p = j;
        double best = fabs(W[j * l + j]);
        for (int64_t i = j + 1; i < m; ++i)
            if (fabs(W[i * l + j]) > best) { best = fabs(W[i * l + j]); p = i; }
        if (p != j) {
            for (int64_t c = 0; c < l; ++c) {
                const double t = W[j * l + c];
                W[j * l + c] = W[p * l + c];
                W[p * l + c] = t;
            }
            const int64_t t = row[j];
            row[j] = row[p];
            row[p] = t;
        }
        const double piv = W[j * l + j];
        if (piv == 0.0) continue;
        for (int64_t i = j + 1; i < m; ++i) {
            const double f = W[i * l + j] / piv;
            W[i * l + j] = f;
            for (int64_t c = j + 1; c < l; ++c) W[i * l + c] -= f * W[j * l + c];
        }
    }
    /* L in Y's row order: row row[i] of L is row i of the unit lower trapezoid */
    for (int64_t i = 0; i < m; ++i)
        for (int64_t c = 0; c < l; ++c) {
            double v;
            if (i < l)
                v = (c == i) ? 1.0 : (c < i ? W[i * l + c] : 0.0);
            else
                v = W[i * l + c];
            L[row[i] * l + c] = v;
        }
    if (U)
        for (int64_t r = 0; r < l; ++r)
            for (int64_t c = 0; c < l; ++c) U[r * l + c] = (c >= r) ? W[r * l + c] : 0.0;
    if (perm)
        for (int64_t j = 0; j < l; ++j) perm[j] = row[j];
    free(W);
    free(row);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Randomized QB decomposition, Algorithm rqb with Algorithm sub_iterations */
/* (scheme 0) or Algorithm norm_iterations (scheme 1) (Secs. 2.1-2.2, 3.3). */
/* The logical A is rows x cols with rows >= cols; l <= cols.  Outputs Q    */
/* (rows x l) and B (l x cols), both row-major.                             */
/* ------------------------------------------------------------------------ */
static int rqb_logical(const amat* A, int64_t l, int q, int sdist, uint64_t seed, double* Q, double* B,
                       int scheme)
{
    const int64_t m = A->rows, n = A->cols;
    int rc = 0;
    float* omega_f = (float*)malloc((size_t)(n * l) * sizeof(float));
    double* X = (double*)malloc((size_t)(n * l) * sizeof(double)); /* n x l */
    double* Y = (double*)malloc((size_t)(m * l) * sizeof(double)); /* m x l */
    double* Z = (double*)malloc((size_t)(n * l) * sizeof(double)); /* n x l */
    if (!omega_f || !X || !Y || !Z) { rc = 2; goto done; }

    /* step 2: Omega = rnorm(n, l) (Sec. 2.3) */
    oracle_omega(n, l, seed, sdist, omega_f, l);
    for (int64_t e = 0; e < n * l; ++e) X[e] = (double)omega_f[e];
    /* step 3: Y = A Omega (Eq. YAQ) */
    gemm_AX(A, X, l, Y);
    /* step 4: Y = norm_iterations(A, Y, q) (scheme 1): pivoted LU in place of
     * the QR steps; the L factors span the same subspaces */
    for (int j = 0; j < q && scheme == 1; ++j) {
        if ((rc = oracle_lu_pivot(m, l, Y, Q, NULL, NULL))) goto done; /* [L, ~] = lu(Y)     */
        gemm_AtX(A, Q, l, Z);                                          /* A^T L              */
        if ((rc = oracle_lu_pivot(n, l, Z, X, NULL, NULL))) goto done; /* [L, ~] = lu(A^T L) */
        gemm_AX(A, X, l, Y);                                           /* Y = A L            */
    }
    /* step 4: Y = sub_iterations(A, Y, q) (scheme 0) */
    for (int j = 0; j < q && scheme == 0; ++j) {
        if ((rc = oracle_householder_qr(m, l, Y, Q, NULL))) goto done; /* Q = qr(Y)     */
        gemm_AtX(A, Q, l, Z);                                          /* A^T Q         */
        if ((rc = oracle_householder_qr(n, l, Z, X, NULL))) goto done; /* Q = qr(A^T Q) */
        gemm_AX(A, X, l, Y);                                           /* Y = A Q       */
    }
    /* step 9: Q = qr(Y) */
    if ((rc = oracle_householder_qr(m, l, Y, Q, NULL))) goto done;
    /* step 10: B = Q^T A  (Eq. BQA), formed as (A^T Q)^T */
    gemm_AtX(A, Q, l, Z);
    for (int64_t r = 0; r < l; ++r)
        for (int64_t c = 0; c < n; ++c) B[r * n + c] = Z[c * l + r];
done:
    free(omega_f); free(X); free(Y); free(Z);
    return rc;
}

static int setup_logical(amat* A, const void* data, int dtype, int64_t m, int64_t n, int64_t lda, int* transposed)
{
    if (dtype != DT_F32 && dtype != DT_BF16 && dtype != DT_F64) return 1;
    if (m < 1 || n < 1 || lda < n) return 1;
    A->data = data;
    A->dtype = dtype;
    A->ld = lda;
    /* Without loss of generality m >= n (Sec. 3.3): a wide A is handled
     * through its transpose. */
    *transposed = (m < n);
    A->trans = *transposed;
    A->rows = *transposed ? n : m;
    A->cols = *transposed ? m : n;
    return 0;
}

/* Oversampled width l = min(k + p, min(m, n)) (Sec. 2.2.1). */
int64_t oracle_sketch_width(int64_t m, int64_t n, int k, int p)
{
    const int64_t mn = m < n ? m : n;
    const int64_t l = (int64_t)k + (int64_t)p;
    return l < mn ? l : mn;
}

/*
 * Algorithm rqb on the user's A (m x n, row-major, leading dimension lda,
 * dtype 0 = FP32, 1 = BF16, 2 = FP64).  For m >= n it writes Q (m x l) and
 * B (l x n).  For m < n it factors A^T and writes Q (n x l) and B (l x m)
 * of that transposed problem (so A^T ~ Q B).  Returns 0 on success.
 */
int oracle_rqb_ex(const void* Adata, int dtype, int64_t m, int64_t n, int64_t lda, int k, int p, int q, int sdist,
                  uint64_t seed, int scheme, double* Q, double* B)
{
    amat A;
    int tr = 0;
    if (setup_logical(&A, Adata, dtype, m, n, lda, &tr)) return 1;
    if (k < 1 || k >= (m < n ? m : n) || p < 0 || q < 0 || scheme < 0 || scheme > 1) return 1;
    const int64_t l = oracle_sketch_width(m, n, k, p);
    return rqb_logical(&A, l, q, sdist, seed, Q, B, scheme);
}

int oracle_rqb(const void* Adata, int dtype, int64_t m, int64_t n, int64_t lda, int k, int p, int q, int sdist,
               uint64_t seed, double* Q, double* B)
{
    return oracle_rqb_ex(Adata, dtype, m, n, lda, k, p, q, sdist, seed, 0, Q, B);
}

/*
 * Algorithm rSVD (Sec. 3.3): [Q, B] = rqb(A, k, p, q); [Ut, S, V] = svd(B);
 * U = Q Ut (Eq. UQU); return U(:,1:k), S(1:k), V(:,1:k).
 * The SVD of B is one-sided Jacobi on B^T (cols x l): B^T J = W gives
 * V = W / s and Ut = J, because B = J diag(s) V^T.
 * Outputs: d (k), U (m x k), V (n x k), row-major.  For m < n the method runs
 * on A^T and the roles of U and V are swapped back at the end.
 * If Qout / Bout are non-NULL they receive Q and B of the (possibly
 * transposed) problem.  Returns 0 on success, < 0 if Jacobi did not converge.
 */
int oracle_rsvd_ex(const void* Adata, int dtype, int64_t m, int64_t n, int64_t lda, int k, int p, int q, int sdist,
                   uint64_t seed, int scheme, double* d, double* U, double* V, double* Qout, double* Bout)
{
    amat A;
    int tr = 0;
    if (setup_logical(&A, Adata, dtype, m, n, lda, &tr)) return 1;
    if (k < 1 || k >= (m < n ? m : n) || p < 0 || q < 0 || scheme < 0 || scheme > 1) return 1;
    const int64_t rows = A.rows, cols = A.cols;
    const int64_t l = oracle_sketch_width(m, n, k, p);
    int rc = 0;
    double* Q = (double*)malloc((size_t)(rows * l) * sizeof(double));
    double* B = (double*)malloc((size_t)(l * cols) * sizeof(double));
    double* Bt = (double*)malloc((size_t)(cols * l) * sizeof(double));
    double* s = (double*)malloc((size_t)l * sizeof(double));
    double* Vl = (double*)malloc((size_t)(cols * l) * sizeof(double));
    double* Ut = (double*)malloc((size_t)(l * l) * sizeof(double));
    if (!Q || !B || !Bt || !s || !Vl || !Ut) { rc = 2; goto done; }

    if ((rc = rqb_logical(&A, l, q, sdist, seed, Q, B, scheme))) goto done;
    for (int64_t r = 0; r < l; ++r)
        for (int64_t c = 0; c < cols; ++c) Bt[c * l + r] = B[r * cols + c];
    if (oracle_jacobi_svd(cols, l, Bt, s, Vl, Ut) < 0) rc = -1;

    /* U = Q Ut, truncated to k columns; V and d truncated likewise. */
    double* Uk = tr ? V : U; /* left vectors of the logical problem */
    double* Vk = tr ? U : V; /* right vectors of the logical problem */
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < rows; ++i)
        for (int64_t c = 0; c < k; ++c) {
            double acc = 0.0;
            for (int64_t t = 0; t < l; ++t) acc += Q[i * l + t] * Ut[t * l + c];
            Uk[i * k + c] = acc;
        }
    for (int64_t i = 0; i < cols; ++i)
        for (int64_t c = 0; c < k; ++c) Vk[i * k + c] = Vl[i * l + c];
    for (int64_t c = 0; c < k; ++c) d[c] = s[c];
    if (Qout) memcpy(Qout, Q, (size_t)(rows * l) * sizeof(double));
    if (Bout) memcpy(Bout, B, (size_t)(l * cols) * sizeof(double));
done:
    free(Q); free(B); free(Bt); free(s); free(Vl); free(Ut);
    return rc;
}

int oracle_rsvd(const void* Adata, int dtype, int64_t m, int64_t n, int64_t lda, int k, int p, int q, int sdist,
                uint64_t seed, double* d, double* U, double* V, double* Qout, double* Bout)
{
    return oracle_rsvd_ex(Adata, dtype, m, n, lda, k, p, q, sdist, seed, 0, d, U, V, Qout, Bout);
}

/*
 * Direct power scheme, Algorithm poweriter_direct (Sec. 2.2.2):
 * Y = (A A^T)^q A Omega with no re-orthonormalisation.  The paper does not
 * recommend it in floating point; here it only serves as an exact-arithmetic
 * statement of the subspace that subspace iteration must span.  Y is m x l,
 * m >= n required.
 */
int oracle_power_direct(const void* Adata, int dtype, int64_t m, int64_t n, int64_t lda, int64_t l, int q, int sdist,
                        uint64_t seed, double* Y)
{
    amat A;
    int tr = 0;
    if (setup_logical(&A, Adata, dtype, m, n, lda, &tr) || tr) return 1;
    float* omega_f = (float*)malloc((size_t)(n * l) * sizeof(float));
    double* X = (double*)malloc((size_t)(n * l) * sizeof(double));
    oracle_omega(n, l, seed, sdist, omega_f, l);
    for (int64_t e = 0; e < n * l; ++e) X[e] = (double)omega_f[e];
    gemm_AX(&A, X, l, Y);
    for (int j = 0; j < q; ++j) {
        gemm_AtX(&A, Y, l, X); /* Y = A^T Y */
        gemm_AX(&A, X, l, Y);  /* Y = A Y   */
    }
    free(omega_f); free(X);
    return 0;
}

/* Plain products on the user's matrix, exported for the kernel-level tests:
 * Y = A X (X is n x l) and Z = A^T X (X is m x l), no transposition trick. */
int oracle_gemm_ax(const void* Adata, int dtype, int64_t m, int64_t n, int64_t lda, const double* X, int64_t l,
                   double* Y)
{
    amat A = {Adata, dtype, m, n, lda, 0};
    gemm_AX(&A, X, l, Y);
    return 0;
}

int oracle_gemm_atx(const void* Adata, int dtype, int64_t m, int64_t n, int64_t lda, const double* X, int64_t l,
                    double* Z)
{
    amat A = {Adata, dtype, m, n, lda, 0};
    gemm_AtX(&A, X, l, Z);
    return 0;
}

/* ||A - U diag(d) V^T||_F^2 in double, streamed row by row; U is m x k,
 * V is n x k (row-major), the error measure of Sec. 3.8. */
double oracle_residual_fro2(const void* Adata, int dtype, int64_t m, int64_t n, int64_t lda, const double* U,
                            const double* d, const double* V, int64_t k)
{
    amat A = {Adata, dtype, m, n, lda, 0};
    double total = 0.0;
#pragma omp parallel for schedule(static) reduction(+ : total)
    for (int64_t i = 0; i < m; ++i) {
        double acc = 0.0;
        for (int64_t j = 0; j < n; ++j) {
            double lr = 0.0;
            for (int64_t c = 0; c < k; ++c) lr += U[i * k + c] * d[c] * V[j * k + c];
            const double e = aget(&A, i, j) - lr;
            acc += e * e;
        }
        total += acc;
    }
    return total;
}

/* ||A||_F^2 in double (Sec. 1.5 notation). */
double oracle_fro2(const void* Adata, int dtype, int64_t m, int64_t n, int64_t lda)
{
    amat A = {Adata, dtype, m, n, lda, 0};
    double total = 0.0;
#pragma omp parallel for schedule(static) reduction(+ : total)
    for (int64_t i = 0; i < m; ++i)
        for (int64_t j = 0; j < n; ++j) {
            const double a = aget(&A, i, j);
            total += a * a;
        }
    return total;
}

/* ------------------------------------------------------------------------ */
/* QR with column pivoting, stopped after k steps (the "pivoted QR" of      */
/* Algorithm id step 1 and Algorithm rcur step 2).  X is rows x cols,       */
/* row-major with leading dimension ldx.  Householder reflections; at step  */
/* t the pivot is the column of the trailing block (rows t..) with the      */
/* largest 2-norm, recomputed exactly (ties: lowest original index).        */
/* Outputs: piv[t] (original column index of the t-th pivot), R (k x cols,  */
/* row-major, ld cols): row t of the triangular factor in the ORIGINAL      */
/* column order, so that R(:, piv) is upper triangular.  With force_piv     */
/* non-NULL the pivots are prescribed instead of chosen; resid_chosen[t]    */
/* and resid_max[t] (if non-NULL) receive the 2-norm of the chosen column's */
/* trailing part and the largest such norm at step t.  Returns 0, or 1 for  */
/* bad arguments / an invalid prescribed pivot.                             */
/* ------------------------------------------------------------------------ */
int oracle_pqr(int64_t rows, int64_t cols, const double* X, int64_t ldx, int k, const int64_t* force_piv,
               int64_t* piv, double* R, double* resid_chosen, double* resid_max)
{
    if (rows < 1 || cols < 1 || k < 1 || k > rows || k > cols || ldx < cols) return 1;
    double* W = (double*)malloc((size_t)(rows * cols) * sizeof(double)); /* column-major */
    char* used = (char*)calloc((size_t)cols, 1);
    double* v = (double*)malloc((size_t)rows * sizeof(double));
    if (!W || !used || !v) { free(W); free(used); free(v); return 2; }
    for (int64_t i = 0; i < rows; ++i)
        for (int64_t j = 0; j < cols; ++j) W[j * rows + i] = X[i * ldx + j];
    int rc = 0;
    for (int t = 0; t < k; ++t) {
        /* trailing norms of the unused columns */
        int64_t best = -1;
        double bestn = -1.0;
        for (int64_t j = 0; j < cols; ++j) {
            if (used[j]) continue;
            double s = 0.0;
            for (int64_t i = t; i < rows; ++i) s += W[j * rows + i] * W[j * rows + i];
            if (s > bestn) { bestn = s; best = j; }
        }
        int64_t p = best;
        if (force_piv) {
            p = force_piv[t];
            if (p < 0 || p >= cols || used[p]) { rc = 1; break; }
        }
        double pn = 0.0;
        for (int64_t i = t; i < rows; ++i) pn += W[p * rows + i] * W[p * rows + i];
        if (resid_chosen) resid_chosen[t] = sqrt(pn);
        if (resid_max) resid_max[t] = sqrt(bestn);
        piv[t] = p;
        used[p] = 1;
        /* reflector H = I - 2 u u^T mapping W(t:, p) to -sign(x_t) ||x|| e_1 */
        const double nrm = sqrt(pn);
        double* x = W + p * rows;
        if (nrm > 0.0) {
            const double alpha = (x[t] >= 0.0) ? -nrm : nrm;
            for (int64_t i = t; i < rows; ++i) v[i] = x[i];
            v[t] -= alpha;
            double vn2 = 0.0;
            for (int64_t i = t; i < rows; ++i) vn2 += v[i] * v[i];
            const double vn = sqrt(vn2);
            for (int64_t i = t; i < rows; ++i) v[i] /= vn;
#pragma omp parallel for schedule(static)
            for (int64_t j = 0; j < cols; ++j) {
                double* w = W + j * rows;
                double dot = 0.0;
                for (int64_t i = t; i < rows; ++i) dot += v[i] * w[i];
                for (int64_t i = t; i < rows; ++i) w[i] -= 2.0 * dot * v[i];
            }
        }
        for (int64_t j = 0; j < cols; ++j) R[(int64_t)t * cols + j] = W[j * rows + t];
    }
    free(W); free(used); free(v);
    return rc;
}

/* ------------------------------------------------------------------------ */
/* Interpolative decomposition, Algorithm id: [~, S, P] = qr(X) pivoted     */
/* (k steps); T = S(1:k,1:k)^{-1} S(1:k, k+1:cols) by back substitution;    */
/* Z(:, P) = [I_k, T]; J = P(1:k).  X rows x cols row-major (ld ldx); Z is  */
/* k x cols row-major.  force_piv as in oracle_pqr.  Returns 0, 1 for bad   */
/* arguments, 3 if S(1:k,1:k) has a zero diagonal entry.                    */
/* ------------------------------------------------------------------------ */
int oracle_id(int64_t rows, int64_t cols, const double* X, int64_t ldx, int k, const int64_t* force_piv,
              int64_t* J, double* Z)
{
    double* R = (double*)malloc((size_t)k * (size_t)cols * sizeof(double));
    char* used = (char*)calloc((size_t)cols, 1);
    if (!R || !used) { free(R); free(used); return 2; }
    int rc = oracle_pqr(rows, cols, X, ldx, k, force_piv, J, R, NULL, NULL);
    if (!rc) {
        for (int t = 0; t < k; ++t)
            if (R[(int64_t)t * cols + J[t]] == 0.0) rc = 3;
    }
    if (!rc) {
        for (int t = 0; t < k; ++t) used[J[t]] = 1;
        for (int64_t j = 0; j < cols; ++j) {
            if (used[j]) {
                for (int a = 0; a < k; ++a) Z[(int64_t)a * cols + j] = 0.0;
                continue;
            }
            /* S11 t = S(:, j), S11(a, b) = R(a, J[b]) upper triangular */
            for (int a = k - 1; a >= 0; --a) {
                double s = R[(int64_t)a * cols + j];
                for (int b = a + 1; b < k; ++b) s -= R[(int64_t)a * cols + J[b]] * Z[(int64_t)b * cols + j];
                Z[(int64_t)a * cols + j] = s / R[(int64_t)a * cols + J[a]];
            }
        }
        for (int t = 0; t < k; ++t)
            for (int a = 0; a < k; ++a) Z[(int64_t)a * cols + J[t]] = (a == t) ? 1.0 : 0.0;
    }
    free(R); free(used);
    return rc;
}

int oracle_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void oracle_set_num_threads(int n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

/* ------------------------------------------------------------------------ */
/* Learned (q, p) controller: the network and its loss, for the gradient    */
/* check of the GPU training kernels.                                       */
/*                                                                          */
/* The paper leaves q and p to the user (Sec. 3.4); this network is not     */
/* from the paper.  Its definition is the library's parameter format:       */
/* x_hat = (x - mu) / sd, h1 = relu(W1 x_hat + b1), h2 = relu(W2 h1 + b2),  */
/* o = W3 h2 + b3 with 16 inputs, 64 + 64 hidden units and 2 outputs;       */
/* parameters mu[16], sd[16], W1[64][16], b1[64], W2[64][64], b2[64],       */
/* W3[2][64], b3[2] (row-major).  relu'(0) = 0.  Loss of a sample: the      */
/* pinball loss summed over the outputs, rho_tau(u) = u (tau - [u < 0]),    */
/* u = y - o; the loss of a set is the mean over its samples.  The gradient */
/* is plain reverse-mode differentiation of that expression, in FP64.       */
/* Pinned by central finite differences and by the closed form of a network */
/* whose output is its bias.                                                */
/* ------------------------------------------------------------------------ */
enum { MLP_I = 16, MLP_H = 64, MLP_O = 2 };
enum {
    MLP_MU = 0,
    MLP_SD = MLP_I,
    MLP_W1 = 2 * MLP_I,
    MLP_B1 = MLP_W1 + MLP_H * MLP_I,
    MLP_W2 = MLP_B1 + MLP_H,
    MLP_B2 = MLP_W2 + MLP_H * MLP_H,
    MLP_W3 = MLP_B2 + MLP_H,
    MLP_B3 = MLP_W3 + MLP_O * MLP_H,
    MLP_NP = MLP_B3 + MLP_O
};

int oracle_mlp_params(void) { return MLP_NP; }

static void mlp_layers(const double* P, const double* x, double* xh, double* h1, double* h2, double* o)
{
    for (int t = 0; t < MLP_I; ++t) xh[t] = (x[t] - P[MLP_MU + t]) / P[MLP_SD + t];
    for (int j = 0; j < MLP_H; ++j) {
        double a = P[MLP_B1 + j];
        for (int t = 0; t < MLP_I; ++t) a += P[MLP_W1 + j * MLP_I + t] * xh[t];
        h1[j] = a > 0.0 ? a : 0.0;
    }
    for (int j = 0; j < MLP_H; ++j) {
        double a = P[MLP_B2 + j];
        for (int t = 0; t < MLP_H; ++t) a += P[MLP_W2 + j * MLP_H + t] * h1[t];
        h2[j] = a > 0.0 ? a : 0.0;
    }
    for (int c = 0; c < MLP_O; ++c) {
        double a = P[MLP_B3 + c];
        for (int t = 0; t < MLP_H; ++t) a += P[MLP_W3 + c * MLP_H + t] * h2[t];
        o[c] = a;
    }
}

/* out[i][c] = network output for sample i (X: n x 16, row-major). */
void oracle_mlp_forward(const double* P, const double* X, int64_t n, double* out)
{
    double xh[MLP_I], h1[MLP_H], h2[MLP_H];
    for (int64_t i = 0; i < n; ++i) mlp_layers(P, X + i * MLP_I, xh, h1, h2, out + i * MLP_O);
}

/* Mean pinball loss over n samples; grad (MLP_NP - 32 values, W1 first:
 * the trainable parameters) receives its gradient when non-null. */
double oracle_mlp_loss_grad(const double* P, const double* X, const double* Y, int64_t n, double tau, double* grad)
{
    const int ntrain = MLP_NP - MLP_W1;
    if (grad)
        for (int e = 0; e < ntrain; ++e) grad[e] = 0.0;
    double loss = 0.0;
    double xh[MLP_I], h1[MLP_H], h2[MLP_H], o[MLP_O], d2[MLP_H], d1[MLP_H];
    for (int64_t i = 0; i < n; ++i) {
        mlp_layers(P, X + i * MLP_I, xh, h1, h2, o);
        double dout[MLP_O];
        for (int c = 0; c < MLP_O; ++c) {
            const double u = Y[i * MLP_O + c] - o[c];
            const double w = (u < 0.0) ? tau - 1.0 : tau;
            loss += u * w;
            dout[c] = -w / (double)n;
        }
        if (!grad) continue;
        /* output layer */
        for (int c = 0; c < MLP_O; ++c) {
            grad[MLP_B3 - MLP_W1 + c] += dout[c];
            for (int t = 0; t < MLP_H; ++t) grad[MLP_W3 - MLP_W1 + c * MLP_H + t] += dout[c] * h2[t];
        }
        /* second hidden layer */
        for (int j = 0; j < MLP_H; ++j) {
            double a = 0.0;
            for (int c = 0; c < MLP_O; ++c) a += dout[c] * P[MLP_W3 + c * MLP_H + j];
            d2[j] = h2[j] > 0.0 ? a : 0.0;
        }
        for (int j = 0; j < MLP_H; ++j) {
            grad[MLP_B2 - MLP_W1 + j] += d2[j];
            for (int t = 0; t < MLP_H; ++t) grad[MLP_W2 - MLP_W1 + j * MLP_H + t] += d2[j] * h1[t];
        }
        /* first hidden layer */
        for (int t = 0; t < MLP_H; ++t) {
            double a = 0.0;
            for (int j = 0; j < MLP_H; ++j) a += d2[j] * P[MLP_W2 + j * MLP_H + t];
            d1[t] = h1[t] > 0.0 ? a : 0.0;
        }
        for (int j = 0; j < MLP_H; ++j) {
            grad[MLP_B1 - MLP_W1 + j] += d1[j];
            for (int t = 0; t < MLP_I; ++t) grad[j * MLP_I + t] += d1[j] * xh[t];
        }
    }
    return loss / (double)n;
}
