/*
 * rsvdgb -- randomized SVD for NVIDIA GB300 (sm_103a).
 *
 * C ABI of the library librsvdgb.so.  The method is the randomized SVD of
 * Erichson, Voronin, Brunton and Kutz, "Randomized Matrix Decompositions Using
 * R" (arXiv:1608.02148): the randomized QB decomposition (Algorithm rqb) with
 * subspace iterations (Algorithm sub_iterations) followed by the SVD of the
 * small factor and the back-projection U = Q Ut (Algorithm rSVD, Eq. UQU).
 *
 * General conventions (apply to every call unless its comment says otherwise)
 *  - Pointers named "device" must point to memory of the handle's device.  The
 *    caller owns every input and output buffer; the library never frees them
 *    and never writes to an input.  The handle owns its workspace.
 *  - Matrices are row-major with an explicit leading dimension (elements
 *    between consecutive rows).  FP32 data must be 4-byte aligned, BF16 data
 *    2-byte aligned.
 *  - Calls are asynchronous on the handle's stream: they return after the
 *    launches are queued, and outputs (including rsvdgb_info) are valid once
 *    that stream has been synchronised.  Exceptions: rsvdgb_create,
 *    rsvdgb_destroy and the *_host entry points, which synchronise.
 *  - Argument errors are detected on the host before any launch and returned
 *    as RSVDGB_ERR_INVALID_ARG with nothing queued.  Errors found on the device
 *    (Cholesky breakdown, non-finite input, an expired bounded wait) are
 *    written to rsvdgb_info.status; kernels never trap.
 */
#ifndef RSVDGB_H
#define RSVDGB_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct rsvdgb_handle rsvdgb_handle;

/* Status codes returned by every int-returning call and stored in
 * rsvdgb_info.status. */
enum {
    RSVDGB_OK = 0,
    RSVDGB_ERR_INVALID_ARG = 1, /* bad size, pointer, alignment or option      */
    RSVDGB_ERR_NOMEM = 2,       /* workspace allocation failed                 */
    RSVDGB_ERR_CUDA = 3,        /* a CUDA runtime call failed                  */
    RSVDGB_ERR_BREAKDOWN = 4,   /* Cholesky of a Gram matrix lost definiteness */
    RSVDGB_ERR_NONFINITE = 5,   /* ||A||_F^2 is not finite                     */
    RSVDGB_ERR_TIMEOUT = 6,     /* a bounded device-side wait expired          */
    RSVDGB_ERR_UNSUPPORTED = 7  /* valid request this build does not serve     */
};

/* Element type of the input matrix A. */
enum { RSVDGB_F32 = 0, RSVDGB_BF16 = 1 };

/* Distribution of the test matrix Omega, Sec. 2.3 ("normal", "unif",
 * "rademacher" of the rsvd() argument sdist, Sec. 3.6). */
enum { RSVDGB_SDIST_NORMAL = 0, RSVDGB_SDIST_UNIF = 1, RSVDGB_SDIST_RADEMACHER = 2 };

/* Arithmetic of the passes over A.
 *  FP32        : every pass FP32-accurate (scaled FP16x3 or 3xTF32 products on
 *                the tensor cores, or FP32 FMA), FP32 accumulation.
 *  BF16_SKETCH : sketch and power passes with A and the panel rounded to BF16,
 *                FP32 accumulation; the final projection B = Q^T A stays
 *                FP32-accurate.
 *  FP8_SKETCH  : one pass first writes an E4M3 copy of A (and its transpose)
 *                with a power-of-two scale per row; the sketch and power
 *                passes read those copies (panels quantised per column),
 *                FP32 accumulation; the projection stays FP32-accurate on A.
 *                Tensor-core engine only; the workspace holds 2 m n bytes more. */
enum { RSVDGB_PREC_FP32 = 0, RSVDGB_PREC_BF16_SKETCH = 1, RSVDGB_PREC_FP8_SKETCH = 2 };

/* Storage order of A as passed by the caller. COL_MAJOR is served as the
 * row-major transpose (U and V swap roles internally). */
enum { RSVDGB_ROW_MAJOR = 0, RSVDGB_COL_MAJOR = 1 };

/* Kernel family for the passes over A. AUTO picks the tensor-core kernels
 * where they apply; SIMT forces the FP32 FMA kernels.  TC computes the
 * FP32-accurate products of every pass after the first as scaled FP16x3
 * (A and each panel column multiplied by a power of two, split into FP16
 * hi + lo, three FP16 products: the same accuracy as 3xTF32 at half the
 * tensor-core time); the first pass, which measures max|A| for that scale,
 * is 3xTF32.  TC_TF32 keeps 3xTF32 for every pass. */
enum { RSVDGB_ENGINE_AUTO = 0, RSVDGB_ENGINE_SIMT = 1, RSVDGB_ENGINE_TC = 2, RSVDGB_ENGINE_TC_TF32 = 3 };

/* How q and p are chosen.  FIXED: opts.q and opts.p.  LEARNED: the handle's
 * controller (rsvdgb_controller_load / rsvdgb_controller_set) predicts them
 * from the first sketch, which is taken with the widest oversampling p_max
 * (Omega is nested in l, so its first k + p columns are the sketch for the
 * chosen p); with no controller loaded the call falls back to FIXED.  The
 * learned mode synchronises the handle's stream once, after the first pass,
 * to read the decision. */
enum { RSVDGB_Q_FIXED = 0, RSVDGB_Q_LEARNED = 1 };

/* Renormalisation between the passes of the power iterations (Sec. 2.2.2).
 * SUBSPACE: Algorithm sub_iterations, an orthonormal basis (CholeskyQR here)
 * of each sketch.  LU: Algorithm norm_iterations, the L factor of a pivoted
 * LU (here a tall-skinny LU with tournament pivoting: l pivot rows chosen by
 * a reduction tree of small partial-pivoting LUs, then L = Y U^{-1} with U
 * from the LU of those rows).  Both keep the span, so they give the same
 * result in exact arithmetic; the final basis of the QB step is always
 * orthonormal.  LU runs on the tensor-core engine with l <= 112. */
enum { RSVDGB_POWER_SUBSPACE = 0, RSVDGB_POWER_LU = 1 };

typedef struct rsvdgb_opts {
    int32_t p;       /* oversampling, l = k + p (Sec. 2.2.1); default 10         */
    int32_t q;       /* subspace iterations (Sec. 2.2.2); default 2              */
    int32_t sdist;   /* RSVDGB_SDIST_*; default NORMAL                            */
    int32_t prec;    /* RSVDGB_PREC_*; default FP32                               */
    uint64_t seed;   /* Philox key of Omega; default 0                           */
    int32_t layout;  /* RSVDGB_ROW_MAJOR / COL_MAJOR; default ROW_MAJOR          */
    int32_t engine;  /* RSVDGB_ENGINE_*; default AUTO                             */
    int32_t q_mode;  /* RSVDGB_Q_FIXED / RSVDGB_Q_LEARNED; default FIXED          */
    int32_t p_max;   /* learned mode: largest oversampling (>= 2); default 10     */
    int32_t q_max;   /* learned mode: largest q; default 6                        */
    int32_t batched_eager; /* 1: rsvdgb_rsvd_batched runs its stages eagerly
                              instead of replaying its CUDA graph; default 0  */
    int32_t power;   /* RSVDGB_POWER_*: how the power iterations renormalise;
                        default SUBSPACE                                       */
    int32_t check_orth; /* 1: measure max |(Q^T Q - I)_ij| of the final basis
                           into info.orth_max (one extra Gram of Q); default 0 */
} rsvdgb_opts;

/* Diagnostics written by the device at the end of a call (device memory). */
typedef struct rsvdgb_info {
    int32_t status;      /* RSVDGB_OK or a device-detected error code          */
    int32_t q_used;      /* subspace iterations performed                      */
    int32_t p_used;      /* oversampling used (l - k after clamping)           */
    int32_t l;           /* sketch width l = min(k + p, min(m, n))             */
    double fro2_A;       /* ||A||_F^2, accumulated in FP64 during the sketch   */
    double fro2_B;       /* ||B||_F^2 = sum of all l squared singular values   */
    double err2_QB;      /* ||A - Q B||_F^2 = fro2_A - fro2_B                  */
    double err2_k;       /* ||A - U_k S_k V_k^T||_F^2 = fro2_A - sum_k s_i^2   */
    int32_t breakdowns;  /* Cholesky breakdowns met (each retried with a shift) */
    int32_t engine;      /* kernel family that ran the passes: RSVDGB_ENGINE_SIMT, _TC or _TC_TF32 */
    int32_t jacobi_sweeps; /* sweeps of the one-sided Jacobi SVD of the l x l factor */
    float orth_max;      /* max_ij |(Q^T Q - I)_ij| of the final basis Q (FP32
                            Gram) when opts.check_orth, else -1               */
    int32_t reserved[4];
} rsvdgb_info;

/* Create a handle bound to CUDA device `device` and stream `cuda_stream`
 * (a cudaStream_t; NULL = the legacy default stream).  The handle's workspace
 * grows on demand and is freed by rsvdgb_destroy.  Returns RSVDGB_OK,
 * RSVDGB_ERR_INVALID_ARG (h NULL, bad device) or RSVDGB_ERR_CUDA. */
int rsvdgb_create(rsvdgb_handle** h, int device, void* cuda_stream);

/* Synchronise the handle's stream and free the handle and its workspace. */
int rsvdgb_destroy(rsvdgb_handle* h);

/* Rebind the handle to another stream of the same device. */
int rsvdgb_set_stream(rsvdgb_handle* h, void* cuda_stream);

/* Defaults of the paper's rsvd() (Sec. 3.6, remark in Sec. 3.3): p = 10,
 * q = 2, sdist = normal; prec FP32, seed 0, row-major, engine AUTO. */
void rsvdgb_default_opts(rsvdgb_opts* o);

/* Human-readable name of a status code (static storage). */
const char* rsvdgb_status_string(int status);

/* Sketch width l = min(k + p, min(m, n)) that a call with these sizes uses
 * (Sec. 2.2.1 with the clamp to min(m, n)). */
int rsvdgb_sketch_width(int64_t m, int64_t n, int k, int p);

/*
 * rsvd(A, k, nu, nv, p, q, sdist) of Sec. 3.6 -- Algorithm rSVD.
 *   A      device, m x n (row-major, leading dimension lda >= n; with
 *          opts->layout = COL_MAJOR it is n x m column-major, i.e. lda >= m),
 *          element type dtype (RSVDGB_F32 or RSVDGB_BF16).  Read only.
 *   k      target rank, 1 <= k < min(m, n) (Algorithm rqb input condition).
 *   nu, nv number of left / right singular vectors to return, 0..k; -1 = k.
 *   d      device float[k]: singular values, descending.
 *   U      device float, m x nu row-major with ldu >= nu (may be NULL if nu = 0).
 *   V      device float, n x nv row-major with ldv >= nv (NOT transposed, as in
 *          the paper's return value v; may be NULL if nv = 0).
 *   info   device rsvdgb_info or NULL.
 * A is factored as A ~ U diag(d) V^T.  Singular vectors are defined up to the
 * sign of each pair (u_i, v_i).  Returns RSVDGB_OK once queued,
 * RSVDGB_ERR_INVALID_ARG, RSVDGB_ERR_NOMEM or RSVDGB_ERR_CUDA.
 */
int rsvdgb_rsvd(rsvdgb_handle* h, const void* A, int64_t m, int64_t n, int64_t lda, int dtype, int k, int nu, int nv,
                const rsvdgb_opts* opts, float* d, float* U, int64_t ldu, float* V, int64_t ldv, rsvdgb_info* info);

/*
 * rsvd() of Sec. 3.6 (Algorithm rSVD) as rsvdgb_rsvd, but A, d, U, V and
 * info are HOST pointers (pinned memory gives full copy bandwidth; pageable
 * memory works).  The call copies A to a device buffer owned by the handle,
 * runs the factorisation, copies the results back and synchronises.  Returns the device status (info->status) if
 * the launches succeeded.
 */
int rsvdgb_rsvd_host(rsvdgb_handle* h, const void* A, int64_t m, int64_t n, int64_t lda, int dtype, int k, int nu,
                     int nv, const rsvdgb_opts* opts, float* d, float* U, int64_t ldu, float* V, int64_t ldv,
                     rsvdgb_info* info);

/*
 * rpca(A, k, center, scale, retx, p, q) of Sec. 4.4 -- Algorithm rpca
 * (Sec. 4.2): the k dominant principal components of the data matrix A
 * (m observations in rows x n variables in columns).
 *   A, m, n, lda, dtype, opts   as in rsvdgb_rsvd (device, read only; opts
 *          NULL = defaults; opts->layout = COL_MAJOR: A stored n x m).
 *   k      1 <= k < min(m, n).
 *   center nonzero: subtract the column means mu_j.
 *   scale  nonzero: divide column j by s_j = sqrt(sum_i (a_ij - mu_j)^2 / (m - 1))
 *          (the standard deviation with `center`; without it the root mean
 *          square with the same m - 1 denominator).  A constant column
 *          (s_j = 0) is analysed as the zero column.
 *   rotation  device float, n x k row-major (ldr >= k): the eigenvectors W
 *          (NULL: not returned).
 *   eigvals   device float[k], required: Lambda = sigma^2 / (m - 1), descending.
 *   sdev      device float[k] or NULL: sqrt(Lambda).
 *   x      device float, m x k row-major (ldx >= k): the principal
 *          components Z = U Sigma = X W (NULL: not returned, retx = FALSE).
 *   center_out, scale_out  device float[n] or NULL: mu (0 without `center`)
 *          and s (1 without `scale`).
 *   info   device rsvdgb_info or NULL; fro2_A is ||X||_F^2 of the centred,
 *          scaled matrix X.
 * The centring and scaling are applied implicitly: A is never copied or
 * modified; each product with X is a product with A plus a rank-one
 * correction, and the statistics cost one extra pass over A.  Eigenvectors
 * are defined up to sign.  Returns as rsvdgb_rsvd (RSVDGB_ERR_INVALID_ARG
 * also for eigvals NULL or a leading dimension < k).
 */
int rsvdgb_rpca(rsvdgb_handle* h, const void* A, int64_t m, int64_t n, int64_t lda, int dtype, int k, int center,
                int scale, const rsvdgb_opts* opts, float* rotation, int64_t ldr, float* eigvals, float* sdev,
                float* x, int64_t ldx, float* center_out, float* scale_out, rsvdgb_info* info);

/*
 * rpca() of Sec. 4.4 (Algorithm rpca) as rsvdgb_rpca, with HOST pointers
 * for A and every output (staged through a device buffer owned by the
 * handle; the call synchronises).
 * Returns the device status (info->status) if the launches succeeded.
 */
int rsvdgb_rpca_host(rsvdgb_handle* h, const void* A, int64_t m, int64_t n, int64_t lda, int dtype, int k,
                     int center, int scale, const rsvdgb_opts* opts, float* rotation, int64_t ldr, float* eigvals,
                     float* sdev, float* x, int64_t ldx, float* center_out, float* scale_out, rsvdgb_info* info);

/*
 * rid(A, k, p, q) of Sec. 7.2 -- Algorithm rid: the randomized column
 * interpolative decomposition A ~ C Z with C = A(:, J).
 *   A, m, n, lda, dtype, opts  as in rsvdgb_rsvd; m >= n is required (the
 *          row ID is the column ID of A^T: call with A^T),
 *          otherwise RSVDGB_ERR_UNSUPPORTED.
 *   k      1 <= k < n, k <= 256.
 *   C      device float, m x k row-major (ldc >= k): the k columns of A, or NULL.
 *   Z      device float, k x n row-major (ldz >= n): the interpolation matrix
 *          (Z(:, J) = I), or NULL.
 *   J      device int64[k], required: the column indices, in pivot order.
 *          After a breakdown (below) the entries from the failed step on
 *          are -1, and C's matching columns and all of Z are zero.
 * Steps: [~, B] = rqb(A, k, p, q) with opts' p and q; QR with column pivoting
 * of the l x n factor B stopped after k steps (Algorithm id); Z(:, P) =
 * [I, S11^{-1} S12]; C = A(:, J).  A pivot step that finds no remaining
 * direction (rank of B below k) sets info->status = RSVDGB_ERR_BREAKDOWN.
 */
int rsvdgb_rid(rsvdgb_handle* h, const void* A, int64_t m, int64_t n, int64_t lda, int dtype, int k,
               const rsvdgb_opts* opts, float* C, int64_t ldc, float* Z, int64_t ldz, int64_t* J, rsvdgb_info* info);

/*
 * rcur(A, k, p, q) of Sec. 7.1 -- Algorithm rcur: A ~ C U R with C = A(:, J)
 * and R = A(I, :).  Arguments as rsvdgb_rid, plus
 *   U      device float, k x k row-major (ldu >= k), or NULL.
 *   R      device float, k x n row-major (ldr >= n), or NULL.
 *   I      device int64[k], required: the row indices, in pivot order.
 * Steps: [C, Z, J] = rid(A, k, p, q); QR with column pivoting of C^T (k
 * steps) gives I; R = A(I, :); U = Z pinv(R), with pinv(R) = Q_R S^{-T} from
 * the CholeskyQR2 factorisation R^T = Q_R S (R of full row rank).
 */
int rsvdgb_rcur(rsvdgb_handle* h, const void* A, int64_t m, int64_t n, int64_t lda, int dtype, int k,
                const rsvdgb_opts* opts, float* C, int64_t ldc, float* U, int64_t ldu, float* R, int64_t ldr,
                int64_t* J, int64_t* I, rsvdgb_info* info);

/* Options of rsvdgb_rrpca (Algorithm rrpca, Sec. 5.2). */
typedef struct rsvdgb_rrpca_opts {
    float lambda;     /* weight of ||S||_1; <= 0: 1 / sqrt(max(m, n)) (Sec. 5)       */
    float tol;        /* stop when ||A - L - S||_F <= tol ||A||_F; default 1e-5     */
    float rho;        /* mu <- min(rho mu, 1e7 mu_0) per iteration; default 1.5     */
    int32_t maxiter;  /* default 50                                                 */
    int32_t k0;       /* initial target rank; default 2 (Algorithm rrpca step 1)    */
    int32_t reserved[3];
} rsvdgb_rrpca_opts;

/* Host-side report of rsvdgb_rrpca. */
typedef struct rsvdgb_rrpca_result {
    int32_t iters;    /* iterations run                                   */
    int32_t rank;     /* singular values kept in L at the last iteration  */
    int32_t k_next;   /* predicted target rank after the last iteration   */
    int32_t status;   /* RSVDGB_OK or the device status of an rSVD        */
    double err;       /* ||A - L - S||_F / ||A||_F at the last iteration  */
    double mu;        /* penalty parameter after the last iteration       */
    double reserved[2];
} rsvdgb_rrpca_result;

/* Defaults of the rrpca() signature of Sec. 5.4: lambda <= 0 (that is,
 * max(m, n)^(-1/2), Sec. 5), maxiter 50, tol 1e-5; k0 = 2 (Algorithm rrpca
 * step 1); rho = 1.5 (a reading of the cited IALM method). */
void rsvdgb_default_rrpca_opts(rsvdgb_rrpca_opts* o);

/*
 * rrpca(A, lambda, maxiter, tol, p, q) of Sec. 5.4 -- Algorithm rrpca: robust
 * PCA A = L + S (low-rank plus sparse) by the inexact augmented Lagrange
 * multiplier method with one randomized SVD (rsvdgb_rsvd, opts' p and q,
 * Omega seed opts->seed + iteration) per iteration.
 *   A      device float, m x n row-major (lda >= n; opts->layout must be
 *          row-major, dtype FP32).  Read only.
 *   L, S   device float, m x n row-major (ldl, lds >= n): the low-rank and the
 *          sparse part.  S is required (it holds the iterate); L may be NULL.
 *   res    host rsvdgb_rrpca_result or NULL.
 * Readings of the steps the paper leaves to the cited method: mu_0 = 1.25 /
 * ||A||_2 (||A||_2 from a rank-1 rSVD of A), Z_0 = A / max(||A||_2,
 * max|a_ij| / lambda), target rank predicted from the number of singular
 * values above 1/mu (next = that + 1 when it is below the target, else
 * that + 5 % of min(m, n)), capped so that k + p <= 224.  The loop runs on
 * the host and synchronises the handle's stream twice per iteration.
 * Returns RSVDGB_OK, an argument / CUDA error (RSVDGB_ERR_INVALID_ARG also
 * for A = 0, checked before any rSVD runs), RSVDGB_ERR_NONFINITE for an A
 * with a NaN or infinity, or the status of an rSVD.
 */
int rsvdgb_rrpca(rsvdgb_handle* h, const float* A, int64_t m, int64_t n, int64_t lda, const rsvdgb_rrpca_opts* ro,
                 const rsvdgb_opts* opts, float* L, int64_t ldl, float* S, int64_t lds, rsvdgb_rrpca_result* res);

/* One matrix of a batch: device pointer to A (m x n row-major, lda >= n). */
typedef struct rsvdgb_matrix_desc {
    const void* A;
    int64_t m;
    int64_t n;
    int64_t lda;
    int32_t dtype;     /* RSVDGB_F32 (the batched path reads FP32 only) */
    int32_t reserved;
} rsvdgb_matrix_desc;

/* Outputs of one matrix of a batch (device pointers; U or V may be NULL). */
typedef struct rsvdgb_result_desc {
    float* d;          /* k singular values, descending            */
    float* U;          /* m x k row-major, leading dimension ldu    */
    int64_t ldu;
    float* V;          /* n x k row-major, leading dimension ldv    */
    int64_t ldv;
} rsvdgb_result_desc;

/*
 * Algorithm rSVD (Sec. 3.3) on a batch of `batch` matrices of uneven shapes
 * with one target rank k and one set of options (p, q, sdist, seed; each
 * matrix uses l = min(k + p, min(m, n)), which must be <= 32).
 *   descs, outs  HOST arrays of `batch` descriptors holding device pointers.
 *   infos        device array of `batch` rsvdgb_info, or NULL.
 * Every step of the method runs as one grouped kernel over the whole batch
 * (work items: matrix x row block / column block); the steps are captured in
 * a CUDA graph per batch layout and replayed with one graph launch.  The
 * first call with a new layout (descriptor contents, k, options) builds a plan
 * (device descriptor and work-item tables, scratch pools), tunes the grid of
 * the grouped kernels with a few timed runs and captures the graph; it
 * synchronises the handle's stream once.  Later calls with the same layout
 * are asynchronous.  FP32 arithmetic (FMA); Omega as in rsvdgb_omega per
 * matrix.  Returns RSVDGB_OK, RSVDGB_ERR_INVALID_ARG, RSVDGB_ERR_UNSUPPORTED
 * (l > 32 or non-FP32 data), RSVDGB_ERR_NOMEM or RSVDGB_ERR_CUDA.
 */
int rsvdgb_rsvd_batched(rsvdgb_handle* h, int batch, const rsvdgb_matrix_desc* descs, int k, const rsvdgb_opts* opts,
                        const rsvdgb_result_desc* outs, rsvdgb_info* infos);

/*
 * Algorithm rqb (Sec. 3.3): A ~ Q B with Q (m x l) orthonormal and
 * B = Q^T A (l x n), Eq. BQA.  Q is written row-major m x l (ldq >= l), B
 * row-major l x n (ldb >= n); both device float.  Requires m >= n with a
 * row-major A (the transposition trick of rsvdgb_rsvd is not applied here).
 */
int rsvdgb_rqb(rsvdgb_handle* h, const void* A, int64_t m, int64_t n, int64_t lda, int dtype, int k,
               const rsvdgb_opts* opts, float* Q, int64_t ldq, float* B, int64_t ldb, rsvdgb_info* info);

/*
 * The test matrix Omega of Sec. 2.3 (Algorithm rqb step 2), rows x l,
 * written row-major to the device buffer out (ld >= l).  Element (i, j) comes
 * from Philox4x32-10 with key (seed mod 2^32, seed >> 32) and counter
 * (i/4 mod 2^32, i/4 >> 32, j, 0); normal entries are Box-Muller on word pairs
 * (x0,x1) -> rows 4r, 4r+1 and (x2,x3) -> rows 4r+2, 4r+3, computed in double
 * and rounded to float; unif = 2u - 1; rademacher = sign from bit 31.
 */
int rsvdgb_omega(rsvdgb_handle* h, int64_t rows, int l, uint64_t seed, int sdist, float* out, int64_t ld);

/*
 * Kernel-level access to the two passes over A (the products A Omega of
 * Algorithm rqb step 3 and A^T Q, A Q of Algorithm sub_iterations), for tests
 * and tuning:
 *   rsvdgb_pass_ax  : Y (m x l) = A X,    X device float n x l row-major (ldx)
 *   rsvdgb_pass_atx : Z (n x l) = A^T X,  X device float m x l row-major (ldx)
 * Outputs row-major with leading dimension ldy / ldz.  `engine` and `prec`
 * select the kernel family and arithmetic as in rsvdgb_opts.
 */
int rsvdgb_pass_ax(rsvdgb_handle* h, const void* A, int64_t m, int64_t n, int64_t lda, int dtype, const float* X,
                   int64_t ldx, int l, float* Y, int64_t ldy, int engine, int prec);
int rsvdgb_pass_atx(rsvdgb_handle* h, const void* A, int64_t m, int64_t n, int64_t lda, int dtype, const float* X,
                    int64_t ldx, int l, float* Z, int64_t ldz, int engine, int prec);

/* Size of the static device scratch used by rsvdgb_pass_atx_noalloc (16 MiB
 * per device that loads the library, held until the process exits). */
#define RSVDGB_NOALLOC_SCRATCH_BYTES (16u << 20)

/*
 * Allocation-free A^T X.  The paper has no counterpart: this entry point
 * serves callers that cannot allocate device memory while they run -- code
 * whose device memory is owned by a pool or arena, code that must not risk
 * the device synchronisation a cudaMalloc / cudaFree can cause, or real-time
 * code with a fixed memory budget.
 *   Computes Z (n x l) = A^T X like rsvdgb_pass_atx with the FP32 FMA kernels:
 *   A device m x n row-major (lda >= n, F32 or BF16), X device float m x l
 *   row-major (ldx >= l), Z device float n x l row-major (ldz >= l); the work
 *   is queued on cuda_stream of the CURRENT device.  No handle is needed.
 *   Scratch: the K-split partial sums go to a static device array of
 *   RSVDGB_NOALLOC_SCRATCH_BYTES; the call allocates and frees nothing.  A
 *   problem with n * ldz * 4 bytes above that size is rejected with
 *   RSVDGB_ERR_INVALID_ARG before anything is queued.
 *   The first call on a device looks up the array's device address (once per
 *   device and CUDA context: again after a cudaDeviceReset); make that first
 *   call before any stream capture.  All calls on a device share the array
 *   and it keeps the last call's contents, so calls that overlap on the GPU
 *   (other streams, other host threads) race.
 * Returns RSVDGB_OK once queued, RSVDGB_ERR_INVALID_ARG, or RSVDGB_ERR_CUDA
 * (also, without queueing anything, when an earlier CUDA error is still
 * pending on the calling thread: it is left for its owner to read).
 */
int rsvdgb_pass_atx_noalloc(void* cuda_stream, const void* A, int64_t m, int64_t n, int64_t lda, int dtype,
                            const float* X, int64_t ldx, int l, float* Z, int64_t ldz);

/* ------------------------------------------------------------------------
 * Learned (q, p) controller.  The paper leaves q and p to the user
 * (Sec. 3.4 recommends p = 10, q = 1 or 2, more iterations for slowly
 * decaying spectra; no counterpart exists for choosing them per matrix).
 * A small MLP (16 -> 64 -> 64 -> 2, ReLU, FP32) maps 16 statistics of the
 * first sketch (the diagonal of the CholeskyQR factor R of Y = A Omega
 * relative to R_11 at indices around k -- R_jj^2 estimates the rank-(j-1)
 * range-finder error -- the sketch energy against ||A||_F^2, shape) to
 * (q, log2 p).
 * Parameters: RSVDGB_MLP_PARAMS floats, laid out as mu[16], sd[16] (input
 * standardisation), W1[64][16], b1[64], W2[64][64], b2[64], W3[2][64], b3[2].
 * File format (little-endian): 8 bytes "RSVDMLP1", int32 RSVDGB_MLP_PARAMS,
 * then the parameters as float32.
 * ---------------------------------------------------------------------- */
#define RSVDGB_MLP_PARAMS 5410
#define RSVDGB_MLP_FEATURES 16

typedef struct rsvdgb_train_opts {
    int32_t epochs;  /* passes over the data set; default 300                  */
    int32_t batch;   /* minibatch size; default 256                            */
    float lr;        /* Adam step size; default 2e-3                           */
    float tau;       /* pinball-loss quantile in (0, 1); default 0.99          */
    uint64_t seed;   /* initialisation and shuffling; default 0                */
    int32_t reserved[4];
} rsvdgb_train_opts;

/* Defaults of rsvdgb_train_opts (no counterpart in the paper). */
void rsvdgb_default_train_opts(rsvdgb_train_opts* o);

/* No counterpart in the paper (q and p are the user's, Sec. 3.4).  Load a
 * parameter file (format above) into the handle; the learned mode of
 * rsvdgb_rsvd then uses it.  RSVDGB_ERR_INVALID_ARG for a missing or
 * malformed file.  Synchronises the handle's stream. */
int rsvdgb_controller_load(rsvdgb_handle* h, const char* path);

/* As rsvdgb_controller_load, from host memory (RSVDGB_MLP_PARAMS floats);
 * no counterpart in the paper. */
int rsvdgb_controller_set(rsvdgb_handle* h, const float* params_host);

/* No counterpart in the paper.  Train on a data set file and write the
 * parameter file.  The data set is 8 bytes "RSVDDS01", int32 n, int32
 * RSVDGB_MLP_FEATURES, then n x 16 float32 features (as
 * rsvdgb_controller_features writes them) and n x 2 float32 targets
 * (q, log2 p).  Training runs on the handle's GPU (minibatch pinball
 * loss, hand-written forward/backward kernels, Adam); the trained parameters
 * are also loaded into the handle.  final_loss (host, may be NULL) receives
 * the mean loss over the data set.  Synchronises. */
int rsvdgb_controller_train(rsvdgb_handle* h, const char* dataset_path, const rsvdgb_train_opts* opts,
                            const char* out_path, float* final_loss);

/* No counterpart in the paper.  The 16 controller features of A (device
 * output feats[16]): pass 1 (Algorithm rqb step 3) with the sketch width
 * k + opts->p_max (clamped to min(m, n)), the CholeskyQR factor of the
 * sketch and ||A||_F^2, as the learned mode computes them.  Arguments
 * as rsvdgb_rsvd; asynchronous. */
int rsvdgb_controller_features(rsvdgb_handle* h, const void* A, int64_t m, int64_t n, int64_t lda, int dtype, int k,
                               const rsvdgb_opts* opts, float* feats);

/* No counterpart in the paper.  Network evaluation and gradient on device
 * arrays (P: RSVDGB_MLP_PARAMS floats; X: n x 16; Y: n x 2; out: n x 2).  rsvdgb_mlp_grad writes the
 * gradient of the mean pinball loss (quantile tau) with respect to the
 * trainable parameters (RSVDGB_MLP_PARAMS - 32 floats, W1 first) and the mean
 * loss (device float).  Asynchronous. */
int rsvdgb_mlp_forward(rsvdgb_handle* h, const float* P, const float* X, int n, float* out);
int rsvdgb_mlp_grad(rsvdgb_handle* h, const float* P, const float* X, const float* Y, int n, float tau, float* grad,
                    float* loss);

/*
 * Test hook for failure detection (the paper has no counterpart).  Arms the
 * handle so that the next rsvdgb_rid / rsvdgb_rcur call runs its pivoted-QR
 * kernel with one CTA leaving out its arrival at the first grid barrier and
 * every barrier wait bounded by spin_ticks clock64 ticks (spin_ticks >= 1).
 * All waits then run out: the kernel records RSVDGB_ERR_TIMEOUT in that
 * call's info.status and returns, and the CUDA context stays usable -- no
 * device fault is raised.  The setting is consumed by that launch.
 * Returns RSVDGB_OK or RSVDGB_ERR_INVALID_ARG.
 */
int rsvdgb_test_pqr_barrier(rsvdgb_handle* h, int64_t spin_ticks);

/*
 * Instrumentation (not part of the paper's method).
 *  rsvdgb_profile_passes : when enable != 0, the handle records a CUDA event
 *      pair on its stream around every launch of a pass kernel over A (the
 *      sketch, power and projection passes) and accumulates the algorithmic
 *      bytes of A each launch must read.  enable = 0 stops recording; either
 *      call clears what was recorded.
 *  rsvdgb_profile_read : synchronises the handle's stream and returns the
 *      summed event time in milliseconds, the number of recorded launches and
 *      the summed algorithmic bytes.  Any output pointer may be NULL.
 *  rsvdgb_kernel_launches : process-wide count of kernels this library has
 *      launched (all handles, all devices).
 */
int rsvdgb_profile_passes(rsvdgb_handle* h, int enable);
int rsvdgb_profile_read(rsvdgb_handle* h, double* pass_ms, int64_t* pass_launches, double* pass_bytes);
int64_t rsvdgb_kernel_launches(void);

#ifdef __cplusplus
}
#endif

#endif /* RSVDGB_H */
