// Internal declarations shared by the CUDA translation units of librsvdgb.
//
// Storage convention inside the library: every tall-skinny matrix (the test
// matrix Omega, the sketch Y, the bases Q and Q_n, A^T Y, B^T) is stored
// COLUMN-MAJOR: column j of an r x l matrix starts at base + j * ld, with ld
// a multiple of 32 elements.  Columns l..l_pad-1 and rows r..ld-1 are kept at
// zero.  This makes every such matrix a K-major operand for the tensor cores
// and gives coalesced column accesses for the FP32 kernels.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/rsvdgb.h"

namespace rsvdgb {

#define RSVDGB_CUDA_TRY(expr)                                   \
    do {                                                        \
        cudaError_t err_ = (expr);                              \
        if (err_ != cudaSuccess) return RSVDGB_ERR_CUDA;        \
    } while (0)

// ---------------------------------------------------------------------------
// Learned (q, p) controller (controller.cu)
// ---------------------------------------------------------------------------
constexpr int kMlpIn = 16, kMlpHidden = 64, kMlpOut = 2;
// mu[16], sd[16], W1[64][16], b1[64], W2[64][64], b2[64], W3[2][64], b3[2]
constexpr int kMlpParams = 2 * kMlpIn + kMlpHidden * kMlpIn + kMlpHidden + kMlpHidden * kMlpHidden + kMlpHidden +
                           kMlpOut * kMlpHidden + kMlpOut;
// 16 features of the first sketch from its CholeskyQR factor R (lmax x lmax,
// row-major) and ||A||_F^2.
void launch_controller_features(cudaStream_t s, const float* R, int lmax, const double* fro2, int64_t m, int64_t n,
                                int k, int p_max, float* feats);
// out[i][0..1] = MLP(X[i]) for n samples (device pointers, P = kMlpParams floats).
void launch_mlp_forward(cudaStream_t s, const float* P, const float* X, int n, float* out);
// (q, p) from the network output: q in [0, q_max], p in [p_min, p_max], k + p <= mn.
void launch_controller_decide(cudaStream_t s, const float* out2, int q_max, int p_min, int p_max, int k, int64_t mn,
                              int* qp);
// Gradient of the mean pinball loss over nb samples (rows idx[0..nb) of X, Y,
// or the first nb rows when idx is null) with respect to the trainable
// parameters (kMlpParams - 32 floats, W1 first); loss (may be null) gets the
// mean loss.  scratch holds mlp_grad_scratch_floats(nb) floats.
size_t mlp_grad_scratch_floats(int nb);
int launch_mlp_grad(cudaStream_t s, const float* P, const float* X, const float* Y, const int* idx, int nb, float tau,
                    float* scratch, float* grad, float* loss);
// Train from host data (n samples); writes kMlpParams floats to P_host_out.
int mlp_train(cudaStream_t s, const float* X_host, const float* Y_host, int n, int epochs, int batch, float lr,
              float tau, uint64_t seed, float* P_host_out, float* final_loss);

// Process-wide count of kernel launches issued by the library.
void count_launches(int n = 1);
int64_t launches_so_far();

inline int64_t round_up(int64_t x, int64_t m) { return (x + m - 1) / m * m; }
inline int64_t ceil_div(int64_t x, int64_t m) { return (x + m - 1) / m; }

// ---------------------------------------------------------------------------
// Test matrix (Sec. 2.3)
// ---------------------------------------------------------------------------
// Writes Omega (rows x l) column-major into out (column j at out + j*ld),
// zero-filling rows rows..rows_pad-1 and columns l..l_pad-1.
void launch_omega(cudaStream_t s, int64_t rows, int64_t rows_pad, int l, int l_pad, uint64_t seed, int sdist,
                  float* out, int64_t ld);
// Row-major variant used by the public rsvdgb_omega entry point.
void launch_omega_rowmajor(cudaStream_t s, int64_t rows, int l, uint64_t seed, int sdist, float* out, int64_t ld);

// ---------------------------------------------------------------------------
// FP32 FMA (SIMT) general product  C = op(A) op(B)
//   op(A)(i,k) = AT ? A[k*lda + i] : A[i*lda + k]          (M x K)
//   op(B)(k,j) = BT ? B[j*ldb + k] : B[k*ldb + j]          (K x N)
//   C(i,j) stored at CT ? C[j*ldc + i] : C[i*ldc + j]       (M x N)
// With splits > 1 the K range is cut into `splits` chunks and chunk z writes
// its partial product at C + z * split_stride (reduce afterwards).
// If fro2 != nullptr, the squares of op(A) are summed (FP64 atomics) from the
// first N-tile of every block row: that is ||A||_F^2 when A is read once.
// ---------------------------------------------------------------------------
struct GemmArgs {
    const void* A;
    int64_t lda;
    int a_bf16;  // op(A) elements stored as BF16 (only for A, not B)
    const float* B;
    int64_t ldb;
    float* C;
    int64_t ldc;
    int64_t M, N, K;
    int splits;
    int64_t split_stride;
    double* fro2;
};
void launch_simt_gemm(cudaStream_t s, bool AT, bool BT, bool CT, const GemmArgs& g);

// Sum `splits` partial matrices (each rows x cols with leading dimension ld,
// consecutive partials split_stride apart) in FP32, in a fixed order, and
// Tensor-core Gram G = X^T X (Z == nullptr or Z == X) or cross product
// G = X^T Z (l x l, row-major, ld l) of column-major rows x l matrices with
// leading dimension ld (columns l..l_pad-1 zero), FP32-accurate (3xTF32).
// part receives up to tc_gram_max_ctas(sm_count) partials of l_pad x l_pad.
// Returns RSVDGB_ERR_UNSUPPORTED when tc_gram_supported() is false.
bool tc_gram_supported(const float* X, const float* Z, int64_t ld, int l_pad);
int64_t tc_gram_max_ctas(int sm_count);
int launch_tc_gram(cudaStream_t s, int sm_count, const float* X, const float* Z, int64_t rows, int64_t ld, int l,
                   int l_pad, float* part, float* G, int* status);

// write out with leading dimension ld_out.
void launch_reduce_splits(cudaStream_t s, const float* part, int splits, int64_t split_stride, int64_t rows,
                          int64_t cols, int64_t ld, float* out, int64_t ld_out);

// ---------------------------------------------------------------------------
// Tensor-core passes over A (tcgen05 + TMA, 3xTF32, FP32 A only)
//   trans = false: out (m x l_pad, column-major ld_out) = A P, P = n x l_pad
//                  given column-major as TF32 hi/lo parts (Phi, Plo, ldp);
//                  optional out_hi/out_lo receive the TF32 split of out.
//   trans = true : partial sums of A^T P (n x l_pad per split, column-major
//                  ld_out, consecutive splits l_pad*ld_out apart) with P = m x
//                  l_pad; *splits_out receives the split count to reduce.
// fro2 (optional) accumulates ||A||_F^2.  Device errors go to *status.
// ---------------------------------------------------------------------------
bool tc_pass_supported(int64_t m, int64_t n, int64_t lda, int l_pad, const void* A, int a_bf16);
// General form: A is the stored row-major m x n FP32 matrix (lda); with
// trans = false the kernel forms A P (lanes = rows of A, K = n), with
// trans = true A^T P (lanes = columns of A, K = m).  The panel P (K x l_pad)
// is given column-major as TF32 hi/lo parts.  K is split into want_splits
// ranges (<= 0: automatic).  With one split and out != null the result goes
// straight to out (column-major, ld_out) and to out_hi/out_lo if given, and
// *splits_out is 0; otherwise the splits write partials (l_pad x ld_out each,
// consecutive partials l_pad*ld_out apart) to `partial`, and *splits_out is
// the count to reduce.  fro2 (optional) accumulates ||A||_F^2.  With
// out_rowmajor (direct output only) out is written row-major:
// out[idx * ld_out + j] for j < out_cols.  With bf16_panel the products run in
// BF16 (A rounded to nearest BF16, P given as one BF16 panel in Phi with
// leading dimension ldp elements; Plo unused), one MMA per K step.  With
// a_bf16, A (passed through the float pointer) holds BF16 values: exact in
// TF32, so the FP32-accurate product needs two MMAs (a p_hi + a p_lo).
// aff_h / aff_r (direct, unchunked, column-major outputs only) apply
// out_ij = aff_r[i] (acc_ij - aff_u[i] aff_h[j]) in the epilogue (aff_h null:
// no shift; aff_u, aff_r null: 1), before the TF32 split.
// chunk_stages > 0 bounds each tensor-memory accumulation chain to that many
// 32-wide K stages; the chunks are summed in the output in FP32 (the tensor
// core's accumulation truncates, which biases long sums toward zero).
// Options of the scaled FP16x3 form and of FP16 output splits:
//   h16: the products run as scaled FP16x3; Phi / Plo are then the FP16 hi /
//        lo parts (uint16, leading dimension ldp elements) of the panel with
//        column j scaled by 1 / pinv[j] (a power of two); A is scaled by the
//        power of two that brings the max|A| held in *amax_in (float bits)
//        into [2^13, 2^14);
//   amax_out: the pass also accumulates max|a| into *amax_out (float bits;
//        zero it beforehand); a pass taking statistics is never FP16x3;
//   out_h16 / out_l16: a direct column-major output also gets its FP16 hi /
//        lo split (same layout as out), column j scaled by split_sc[j] (or by
//        split_sc_const when split_sc is null).
struct TcExtra {
    int h16 = 0;
    const unsigned int* amax_in = nullptr;
    const float* pinv = nullptr;
    unsigned int* amax_out = nullptr;
    uint16_t* out_h16 = nullptr;
    uint16_t* out_l16 = nullptr;
    const float* split_sc = nullptr;
    float split_sc_const = 0.f;
};
int launch_tc_gemm(cudaStream_t s, int sm_count, bool trans, const float* A, int64_t m, int64_t n, int64_t lda,
                   const float* Phi, const float* Plo, int64_t ldp, int l_pad, float* out, float* out_hi,
                   float* out_lo, int64_t ld_out, float* partial, int64_t want_splits, int64_t* splits_out,
                   int* status, double* fro2, int out_rowmajor = 0, int out_cols = 0, int bf16_panel = 0,
                   int a_bf16 = 0, int chunk_stages = 0, const float* aff_h = nullptr,
                   const float* aff_u = nullptr, const float* aff_r = nullptr, const TcExtra* x = nullptr);
// Z = X T (xt.cu) for a column-major rows x l matrix X (ld) and an l x l
// row-major upper triangular T (entries below the diagonal must be zero),
// in FP32 FMA; Z column-major (ld) over l_pad columns, rows beyond `rows` up
// to ld and columns beyond l written as zero.  split 1: Zh / Zl get Z's TF32
// hi / lo (floats); split 2: the FP16 hi / lo (uint16) of sc Z.  l_pad a
// multiple of 16 up to 112, ld a multiple of 4, X 16-byte aligned.
bool xt_supported(int l_pad);
int launch_xt(cudaStream_t s, int sm_count, const float* X, int64_t ld, int64_t rows, int l, int l_pad, const float* T,
              float* Z, int split, void* Zh, void* Zl, float sc);
// Pivoted LU of a tall column-major rows x l matrix X (ld) for the normalized
// power iterations (tslu.cu): tournament pivoting picks l pivot rows; U (l x
// l row-major, upper triangular) is the LU factor of those rows and T = U^{-1}
// (l x l row-major), so that L = X T.  scratch: tslu_scratch_ints(rows, l)
// ints.  A zero pivot in U sets *status = RSVDGB_ERR_BREAKDOWN.  l <= 112,
// rows >= l.
bool tslu_supported(int l);
int64_t tslu_scratch_ints(int64_t rows, int l);
int launch_tslu(cudaStream_t s, const float* X, int64_t ld, int64_t rows, int l, int* scratch, float* U, float* T,
                int* status);
// FP8 (E4M3) power passes (fp8.cu, fp8_pass.cu).  launch_fp8_prep: A (m x n
// row-major, lda; FP32 or BF16) -> A8 (row-major bytes, ld8 >= n, multiple of
// 16), At8 (its transpose, column-major: At8[c * ldt + i], ldt >= m, multiple
// of 16) and the row powers of two rs (m floats); adds ||A||_F^2 to *fro2 and
// max|A| (bits) to *amax when non-null.  launch_fp8_panel: column-major K x l
// panel P (ld a multiple of 4, 16-byte aligned), optionally row-scaled by r,
// -> P8 (column-major bytes, ld8 >= K, multiple of 16, l_pad columns) and
// column powers of two ts; cm is l_pad + 1 uints of scratch that must be zero
// on entry and is left zero.
// launch_f8_pass: out (lanes x l_pad column-major, ld_out) = A8_lanes P8 with
// the lane-major copy A8 (A8 for the A side, At8 for the A^T side: lanes x
// k_total, ld_a8 bytes), rows scaled by row_scale (optional) and columns by
// col_scale; with K splits the partials go to `partial` and *splits_out is
// their count (0: written to out).
void launch_fp8_prep(cudaStream_t s, const void* A, int64_t lda, int a_bf16, int64_t m, int64_t n, uint8_t* A8,
                     int64_t ld8, uint8_t* At8, int64_t ldt, float* rs, double* fro2, unsigned int* amax);
void launch_fp8_panel(cudaStream_t s, const float* P, int64_t ld, int64_t K, int l, int l_pad, const float* r,
                      uint8_t* P8, int64_t ld8, float* ts, unsigned int* cm);
int launch_f8_pass(cudaStream_t s, int sm_count, bool trans, const uint8_t* A8, int64_t lanes, int64_t k_total,
                   int64_t ld_a8, const uint8_t* P8, int64_t ld_p8, int l_pad, const float* row_scale,
                   const float* col_scale, float* out, int64_t ld_out, float* partial, int64_t* splits_out,
                   int* status);
int64_t f8_pass_max_splits(int64_t lanes, int64_t k_total, int l_pad, int sm_count);
// Scaled FP16 hi / lo split of a column-major rows x l panel (ld even) over
// l_pad columns for the FP16x3 passes: column j is multiplied by the power of
// two bringing its max magnitude into [2^13, 2^14), pinv[j] receives the
// inverse of that factor (1 for columns >= l); rows >= rows and columns >= l
// are written as zero.
void launch_panel_f16(cudaStream_t s, const float* in, int64_t ld, int64_t rows, int l, int l_pad, uint16_t* hi,
                      uint16_t* lo, float* pinv);
// max|a| of a row-major rows x cols matrix (FP32, or BF16 bits when a_bf16),
// atomicMax'ed as float bits into *amax (zero it beforehand).
void launch_absmax(cudaStream_t s, int sm_count, const void* A, int64_t lda, int a_bf16, int64_t rows, int64_t cols,
                   unsigned int* amax);
int64_t tc_pass_max_splits(int64_t m, int64_t n, int l_pad, int sm_count);
int64_t tc_split_count(int64_t k_total, int64_t units, int sm_count);
// l x l row-major T -> column-major L x L TF32 hi/lo panel (zero padded),
// i.e. out[j * L + c] = T[c * l + j].
void launch_small_panel(cudaStream_t s, const float* T, int l, int L, float* hi, float* lo);
// BF16 (round to nearest) copy of a column-major rows x l matrix over l_pad
// columns, zero outside rows x l.
void launch_to_bf16(cudaStream_t s, const float* in, int64_t ld, int64_t rows, int l, int l_pad, void* out);
// TF32 split of a column-major rows x l matrix (ld) into hi + lo parts over
// l_pad columns; rows >= rows and columns >= l are written as zero.
void launch_split_tf32(cudaStream_t s, const float* in, int64_t ld, int64_t rows, int l, int l_pad, float* hi,
                       float* lo);

// ---------------------------------------------------------------------------
// Small l x l kernels (one CTA)
// ---------------------------------------------------------------------------
// Cholesky G + shift*I = R^T R of a symmetric l x l Gram matrix (FP32,
// row-major, ld = l, 16-byte aligned) by Gaussian elimination that also
// produces R^{-T}; writes R (if non-null) and T = R^{-1} as FP32 row-major
// l x l (upper triangular, zero below).  A pivot that is not positive and
// finite restarts the factorization with a larger diagonal shift (three
// retries, each counted in *breakdowns); if the last attempt fails too,
// *status = RSVDGB_ERR_BREAKDOWN.
void launch_chol_inv(cudaStream_t s, const float* G, int l, float shift_rel, float* R, float* T, int* status,
                     int* breakdowns);
// C = A B for l x l FP32 row-major matrices (used for T1 T2 and R2 R1).
void launch_small_matmul(cudaStream_t s, const float* A, const float* B, float* C, int l);
// One-sided Jacobi SVD of the l x l FP32 matrix M (row-major): M J = W with
// orthogonal columns.  Outputs (sorted by descending sigma):
//   sigma[l] (FP32), Ut (l x l row-major, Ut[:,c] = W[:,c] / sigma_c),
//   Jt (l x l row-major, right vectors; only the first kv columns written).
void launch_jacobi_svd(cudaStream_t s, const float* M, int l, float* sigma, float* Ut, float* Jt, float* work,
                       int* sweeps, int kv);
// Transpose an l x l row-major matrix: out = in^T.
void launch_small_transpose(cudaStream_t s, const float* in, float* out, int l);
// d[0..k) = sigma[0..k); info fields from fro2_A and sigma.
void launch_finalize_info(cudaStream_t s, const float* sigma, int l, int k, float* d, const double* fro2A,
                          const int* status, const int* breakdowns, int q, int p_used, int engine,
                          const int* sweeps, rsvdgb_info* info, const float* orth = nullptr);
// max_ij |G_ij - delta_ij| of an l x l row-major Gram into *out (device).
void launch_orth_err(cudaStream_t s, const float* G, int l, float* out);
// Raise the dynamic shared-memory limit of the one-CTA kernels on the
// current device (called once per handle).
int init_small_kernels();
// Zero the status / breakdown counters, ||A||_F^2 and max|A| (each may be
// null), set fillv[0..nfill) to fillval (fillv may be null) and zero
// zerov[0..nzero) (zerov may be null).
void launch_clear_scalars(cudaStream_t s, int* status, int* breakdowns, double* fro2, unsigned int* amax = nullptr,
                          float* fillv = nullptr, int nfill = 0, float fillval = 0.f, unsigned int* zerov = nullptr,
                          int nzero = 0);

// Convert a column-major r x l (ld) matrix to row-major (ldo) with cols
// columns (cols <= l), i.e. out[i*ldo + j] = in[j*ld + i].
void launch_colmajor_to_rowmajor(cudaStream_t s, const float* in, int64_t ld, int64_t rows, int cols, float* out,
                                 int64_t ldo);
void launch_rowmajor_to_colmajor(cudaStream_t s, const float* in, int64_t ldi, int64_t rows, int cols, int cols_pad,
                                 float* out, int64_t ld);

// Randomized PCA (pca.cu): implicit centring / scaling of the data matrix.
// Per-variable statistics in one pass over the stored matrix S (rows_s x
// cols_s, lda): the variables are the columns of S (vars_are_cols) or its
// rows.  Writes mu (centre or 0), cmul (1 / scale, 0 for a constant
// variable, or 1), the optional user copies, and ||X||_F^2 of the analysed
// matrix to *fro2.  part holds stats_chunks(...) x nvar double2.
int64_t stats_chunks(bool vars_are_cols, int64_t rows_s, int64_t cols_s, int sm_count);
void launch_var_stats(cudaStream_t s, int sm_count, const void* S, int64_t lda, int64_t rows_s, int64_t cols_s,
                      int a_bf16, bool vars_are_cols, int center, int scale, double2* part, float* mu, float* cmul,
                      float* center_out, float* scale_out, double* fro2_part, double* fro2);
// part[c * l + j] (c < *chunks_out <= kAffineMaxChunks): partial sums of
// sum_i X_ij w_i over row chunks (w null: 1); X column-major rows x l (ld).
constexpr int kAffineMaxChunks = 64;
void launch_affine_dot(cudaStream_t s, int sm_count, const float* X, int64_t ld, int64_t rows, int l, const float* w,
                       double* part, int* chunks_out);
// h[j] = sum of the chunk partials of column j (j < l).
void launch_affine_h(cudaStream_t s, const double* part, int chunks, int l, float* h);
// out_ij = r_i (out_ij - u_i h_j), h_j = sum of the chunk partials of
// column j (part null: no shift; u, r null: 1); optional TF32 split.
void launch_affine_post(cudaStream_t s, float* out, int64_t ld, int64_t rows, int l, const float* r, const float* u,
                        const double* part, int chunks, float* hi, float* lo);
// out_ij = r_i in_ij (column-major; in == out allowed), optional TF32 split;
// zero over the padding (rows up to ld, columns up to l_pad).
void launch_scale_rows(cudaStream_t s, const float* in, int64_t ld, int64_t rows, int l, int l_pad, const float* r,
                       float* out, float* hi, float* lo);
// T[i * l + c] *= sigma[c] for c < ncols (l x l row-major).
void launch_scale_cols_small(cudaStream_t s, float* T, int l, int ncols, const float* sigma);
// eig = sigma^2 / (m_obs - 1), sdev = sigma / sqrt(m_obs - 1) (first k).
void launch_pca_values(cudaStream_t s, const float* sigma, int k, int64_t m_obs, float* eig, float* sdev);

// Interpolative / CUR decompositions (rid.cu).
// Column-pivoted QR (k steps) of the r x N matrix X (column j at X + j*ldx,
// r <= 256, k <= r, r*k floats of shared memory per CTA): pivots (int, k),
// R rows (k x N row-major, optional), one cooperative launch with a bounded
// grid barrier.  Workspace: nrm (N doubles), max_slots (double, int64)
// slots, one counter.
// spin_limit bounds each barrier wait (clock64 ticks; <= 0: the default of
// about 2 s); absent_cta >= 0 (a test hook) makes that CTA skip its arrival at
// the first barrier, so that every wait runs out and RSVDGB_ERR_TIMEOUT is
// recorded.
int launch_pqr(cudaStream_t s, int sm_count, const float* X, int64_t ldx, int r, int64_t N, int k, int* piv,
               float* R, double* nrm, double* slot_val, int64_t* slot_idx, int max_slots, unsigned int* bar,
               int* status, long long spin_limit = 0, int absent_cta = -1);
// Z (k x N, ld ldz) of the ID from R and the pivots (Algorithm id steps 2-5).
void launch_id_solve(cudaStream_t s, const float* R, int64_t N, int k, const int* piv, float* Z, int64_t ldz,
                     int* status);
// C (rows x k, ld ldc) = columns idx of the logical matrix of the stored S.
void launch_gather_cols(cudaStream_t s, const void* S, int64_t lda, int a_bf16, bool trans, int64_t rows,
                        const int* idx, int k, float* C, int64_t ldc);
// R (k x cols, ld ldr) = rows idx of the logical matrix; Rt its transpose
// (column-major, ld ldt); either may be null.
void launch_gather_rows(cudaStream_t s, const void* S, int64_t lda, int a_bf16, bool trans, int64_t cols,
                        const int* idx, int k, float* R, int64_t ldr, float* Rt, int64_t ldt);
// X (r x N column-major, ld ldx) = transpose of the column-major N x r Bt.
void launch_transpose_cm(cudaStream_t s, const float* Bt, int64_t ldb, int64_t N, int r, float* X, int64_t ldx);
// W (k x k row-major) = Z Q, Z k x N row-major, Q N x k column-major.
void launch_zq(cudaStream_t s, const float* Z, int64_t ldz, const float* Q, int64_t ldq, int64_t N, int k, float* W);
void launch_piv_to_i64(cudaStream_t s, const int* piv, int k, int64_t* out);

// Robust PCA (rrpca.cu).
int64_t ialm_blocks(int64_t m, int64_t n);
// *amax (bits of max|a|, start from 0) and *sumsq = ||A||_F^2 (part: nblocks doubles).
void launch_absmax_sumsq(cudaStream_t s, const float* A, int64_t lda, int64_t m, int64_t n, unsigned int* amax,
                         double* part, int nblocks, double* sumsq);
// Z = A / dual, S = 0, X = A + Z / mu0 (Z, X: m x n with ld n).
void launch_ialm_init(cudaStream_t s, const float* A, int64_t lda, int64_t m, int64_t n, float inv_dual,
                      float inv_mu0, float* S, int64_t lds, float* Z, float* X);
// One fused IALM update (mode 0; *err2 = ||A - L - S||_F^2, part: ialm_blocks
// doubles) or the reconstruction of L = U diag(sig) V^T into Lout (mode 1).
void launch_ialm_step(cudaStream_t s, const float* A, int64_t lda, int64_t m, int64_t n, const float* U, int64_t ldu,
                      const float* V, int64_t ldv, const float* sig, int kl, float mu, float inv_mu,
                      float inv_mu_next, float thr, float* S, int64_t lds, float* Z, float* X, double* part,
                      double* err2, int mode, float* Lout, int64_t ldl);

// Batched rSVD (batched.cu): plan cache owned by the handle.
struct BatchedPlan;
void destroy_plan(BatchedPlan* pl);
int batched_rsvd(BatchedPlan** cache, int device, int sm_count, cudaStream_t stream, int B,
                 const rsvdgb_matrix_desc* descs, int k, const rsvdgb_opts& o, const rsvdgb_result_desc* outs,
                 rsvdgb_info* infos);

}  // namespace rsvdgb
