// Host orchestration and the C ABI of librsvdgb.
//
// rsvdgb_rsvd runs Algorithm rSVD of Sec. 3.3 on the device:
//   1  l = min(k + p, min(m, n))                          (Sec. 2.2.1)
//   2  Omega (n x l) from Philox                          (Sec. 2.3)
//   3  Y = A Omega                                        (Eq. YAQ)
//   4  q times: Q = qr(Y); Q = qr(A^T Q); Y = A Q         (Algorithm sub_iterations)
//   9  Q = qr(Y)                                          (Algorithm rqb step 9)
//  10  B = Q^T A                                          (Eq. BQA)
//      [Ut, S, V] = svd(B); U = Q Ut                      (Algorithm rSVD, Eq. UQU)
// Every step is a kernel on the handle's stream; nothing synchronises with
// the host.  "qr" is CholeskyQR: Gram matrix, Cholesky, basis change.  The
// m-side factorisations inside the iteration only need the span of Y, so they
// use one Cholesky step; the final Q, the n-side bases and the factorisation
// of B^T use two (CholeskyQR2).  The SVD of B is taken as B^T = Q_B R_B
// (CholeskyQR2) followed by the one-sided Jacobi SVD of the l x l R_B^T:
// R_B^T J = W Sigma gives B = W Sigma (Q_B J)^T, i.e. Ut = W and V = Q_B J.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>
#include <vector>

#include "internal.cuh"

static_assert(RSVDGB_MLP_PARAMS == rsvdgb::kMlpParams, "controller parameter count");
static_assert(RSVDGB_MLP_FEATURES == rsvdgb::kMlpIn, "controller feature count");

using namespace rsvdgb;

namespace rsvdgb {
namespace {
std::atomic<int64_t> g_launches{0};
}
void count_launches(int n) { g_launches.fetch_add(n, std::memory_order_relaxed); }
int64_t launches_so_far() { return g_launches.load(std::memory_order_relaxed); }
}  // namespace rsvdgb

// Event pairs bracketing the pass kernels over A (instrumentation).
struct PassProfile {
    bool on = false;
    std::vector<cudaEvent_t> ev;  // 2 per recorded launch
    size_t used = 0;              // recorded launches
    double bytes = 0.0;           // algorithmic bytes of A over the recorded launches
};

struct rsvdgb_handle {
    int device = 0;
    cudaStream_t stream = nullptr;
    int sm_count = 148;
    void* ws = nullptr;
    size_t ws_bytes = 0;
    void* host_stage = nullptr;  // device buffers for the *_host entry points
    size_t host_stage_bytes = 0;
    void* aux = nullptr;  // iterates of rsvdgb_rrpca (kept apart from ws, which its rSVDs resize)
    size_t aux_bytes = 0;
    PassProfile prof;
    // test hook (rsvdgb_test_pqr_barrier): the next pivoted-QR launch of a
    // rid / rcur call leaves CTA 0's first grid-barrier arrival out and bounds
    // the waits by test_spin ticks; consumed by that launch
    int test_pqr_absent = 0;
    long long test_spin = 0;
    BatchedPlan* batched = nullptr;  // plan of the last batch layout
    float* ctl_params = nullptr;     // learned (q, p) controller (device, kMlpParams floats)
    float* ctl_scratch = nullptr;    // features, network output, decision (device)
    int* ctl_host = nullptr;         // pinned host copy of the decision (q, p)
};

namespace {

constexpr int kMaxL = 224;  // widest sketch the one-CTA l x l kernels hold in shared memory
// Tensor-core accumulation chains of the products whose scale matters (the
// projection B = Q^T A, Grams on the pass kernel, the C-ABI products) are cut
// every kExactChunk K stages of 32 (the accumulator truncates; see tc_pass.cu).
constexpr int kExactChunk = 16;

// Bump allocator over the handle's workspace (256-byte aligned pieces).
struct Carve {
    char* base;
    size_t off = 0;
    explicit Carve(void* b) : base((char*)b) {}
    template <class T>
    T* take(size_t count)
    {
        off = (size_t)round_up((int64_t)off, 256);
        T* p = base ? (T*)(base + off) : nullptr;
        off += count * sizeof(T);
        return p;
    }
};

// Implicit centring / scaling of the logical matrix (randomized PCA): the
// analysed matrix is X = (A - 1 mu^T) diag(c) when the variables are the
// logical columns, X = diag(c) (A - mu 1^T) when they are the logical rows
// (the data matrix had fewer observations than variables).  mu null: no
// centring; c null: no scaling.  part: partial sums of the correction vector.
struct Affine {
    bool rows;
    const float* mu;
    const float* c;
    double* part;
};

// Problem geometry after the m >= n normalisation.  The logical matrix is
// either the stored row-major matrix S or its transpose.
struct Geom {
    const void* A;
    int64_t lda;
    int a_bf16;
    int64_t m, n;  // logical rows >= logical cols
    bool trans;    // logical = S^T
    bool swap_uv;  // user's U <- logical V
    int l;
    int L;         // l rounded up to 16 (tensor-core N granularity)
    bool use_tc;   // passes over A on the tensor cores
    bool h16 = false;  // FP32-accurate passes after the first as scaled FP16x3 (tensor cores)
    bool lu = false;   // power iterations renormalised by pivoted LU (Algorithm norm_iterations)
    bool fp8 = false;  // sketch and power passes on E4M3 copies of A (mixed precision)
    bool bf16;     // sketch and power passes in BF16 (mixed precision)
    int64_t ldm, ldn;
    const Affine* aff = nullptr;  // randomized PCA: products with X instead of A
    int64_t pca_nvar = 0;         // randomized PCA: number of variables (0: plain rSVD)
    int rid_k = 0;                // interpolative / CUR decomposition of rank rid_k (0: none)
    bool rid_cur = false;         // ... with the CUR step
    // stored matrix dimensions (rows x cols of the row-major S)
    int64_t sm() const { return trans ? n : m; }
    int64_t sn() const { return trans ? m : n; }
};

struct Work {
    float *Pt, *Yt, *Qt, *Wt, *Zt, *part;
    float *Pth, *Ptl, *Yth, *Ytl;  // TF32 hi/lo parts of the panels (tensor-core engine)
    float *Qth, *Qtl, *Th, *Tl;    // hi/lo of the first CholeskyQR2 basis and of a small factor
    void *Ptb, *Ytb;               // BF16 panels (mixed precision)
    float* G;  // l x l Gram (sum of per-CTA FP32 partials)
    float *T1, *T2, *T, *R1, *R2, *RB, *M, *sigma, *Ut, *Jt, *jwork;
    int *status, *breakdowns, *sweeps;
    double* fro2;
    float* orth;  // max |Q^T Q - I| of the final basis (opts.check_orth)
    // randomized PCA: centre and multiplier per variable, statistics and
    // correction partial sums
    float *mu, *cmul;
    double2* spart;
    double *hpart, *fpart;
    float* hvec;  // correction vector h of the current pass
    // interpolative / CUR decompositions
    float *Xb, *Rk, *Zw, *Cw;
    double *pnrm, *slot_v;
    int64_t* slot_i;
    int* piv;
    unsigned int* bar;
    // scaled FP16x3 passes: max|A| (float bits, from the first pass) and the
    // inverse column scales of the n-side panel (Pth / Ptl then hold its FP16
    // hi / lo) and of the m-side panels (constant: their columns are unit
    // vectors up to rounding)
    unsigned int* amax;
    float *Ppinv, *Qpinv;
    int* luscr;  // pivot-row proposals of the tall-skinny LU (normalized power iterations)
    // FP8 passes: E4M3 copies of the stored matrix (row-major A8, transposed
    // At8), its row powers of two, the quantised panel and its column scales
    uint8_t *A8, *At8, *P8;
    int64_t ld8, ldt8, ldp8;
    float *rs8, *ts8;
    unsigned int* cm8;  // the panel quantisation's column maxima and CTA count (zero between panels)
};

constexpr int kPqrSlots = 1024;  // per-CTA maxima of the pivoted QR (its grid is at most this wide)

int splits_for(int64_t tiles, int64_t K, int sm_count)
{
    int64_t want = ceil_div(4 * (int64_t)sm_count, std::max<int64_t>(tiles, 1));
    int64_t cap = std::max<int64_t>(1, K / 256);
    want = std::min<int64_t>(std::min<int64_t>(want, cap), 256);
    return (int)std::max<int64_t>(want, 1);
}

size_t partial_floats(const Geom& g, int sm_count)
{
    const int64_t L = g.L;
    // largest K-split product: A^T-side pass (M = n, K = m), Grams (M = N = l)
    int64_t tiles_at = ceil_div(g.n, 64) * ceil_div(L, 64);
    int64_t s_at = splits_for(tiles_at, g.m, sm_count);
    int64_t tiles_g = ceil_div(L, 64) * ceil_div(L, 64);
    int64_t s_gm = splits_for(tiles_g, g.m, sm_count);
    int64_t need = std::max<int64_t>(s_at * L * g.ldn, s_gm * L * L);
    // the transposed A-side pass splits over K = n with M = m
    int64_t tiles_a = ceil_div(g.m, 64) * ceil_div(L, 64);
    int64_t s_a = splits_for(tiles_a, g.n, sm_count);
    need = std::max<int64_t>(need, s_a * L * g.ldm);
    if (g.use_tc) {
        // tensor-core A^T-side kernel on the stored matrix: lanes = stored columns
        const int64_t s_tc = tc_pass_max_splits(g.sm(), g.sn(), g.L, sm_count);
        need = std::max<int64_t>(need, s_tc * L * std::max(g.ldm, g.ldn));
        // tensor-core Gram: at most one split per SM, L x L each
        need = std::max<int64_t>(need, (int64_t)sm_count * L * L);
        // FP8 passes: splits over the stored rows (lanes = stored columns) or columns
        const int64_t s8 = std::max(f8_pass_max_splits(g.sn(), g.sm(), g.L, sm_count),
                                    f8_pass_max_splits(g.sm(), g.sn(), g.L, sm_count));
        need = std::max<int64_t>(need, s8 * L * std::max(g.ldm, g.ldn));
    }
    return (size_t)need;
}

void carve_work(Carve& c, const Geom& g, int sm_count, Work& w, int L_lo = 0)
{
    const int64_t L = g.L;
    w.Pt = c.take<float>(L * g.ldn);
    w.Yt = c.take<float>(L * g.ldm);
    w.Qt = c.take<float>(L * g.ldm);
    w.Pth = w.Ptl = w.Yth = w.Ytl = w.Qth = w.Qtl = w.Th = w.Tl = nullptr;
    if (g.use_tc) {
        w.Pth = c.take<float>(L * g.ldn);
        w.Ptl = c.take<float>(L * g.ldn);
        w.Yth = c.take<float>(L * g.ldm);
        w.Ytl = c.take<float>(L * g.ldm);
        w.Qth = c.take<float>(L * g.ldm);
        w.Qtl = c.take<float>(L * g.ldm);
        w.Th = c.take<float>(L * L);
        w.Tl = c.take<float>(L * L);
    }
    w.Ptb = w.Ytb = nullptr;
    if (g.bf16) {
        w.Ptb = c.take<uint16_t>(L * g.ldn);
        w.Ytb = c.take<uint16_t>(L * g.ldm);
    }
    w.Wt = c.take<float>(L * g.ldn);
    w.Zt = c.take<float>(L * g.ldn);
    // split-K partials: the learned mode runs the sketch at g.L and the rest at
    // any narrower width down to L_lo, so take the largest need over them
    size_t part = partial_floats(g, sm_count);
    for (int Lx = std::max(16, L_lo); L_lo > 0 && Lx < g.L; Lx += 16) {
        Geom gx = g;
        gx.L = Lx;
        gx.l = std::min(gx.l, Lx);
        part = std::max(part, partial_floats(gx, sm_count));
    }
    w.part = c.take<float>(part);
    w.G = c.take<float>(L * L);
    w.T1 = c.take<float>(L * L);
    w.T2 = c.take<float>(L * L);
    w.T = c.take<float>(L * L);
    w.R1 = c.take<float>(L * L);
    w.R2 = c.take<float>(L * L);
    w.RB = c.take<float>(L * L);
    w.M = c.take<float>(L * L);
    w.sigma = c.take<float>(256);
    w.Ut = c.take<float>(L * L);
    w.Jt = c.take<float>(L * L);
    // Jacobi columns when they do not fit in shared memory: 2 x l x Lp with the
    // padded column stride Lp <= l rounded up to 32
    w.jwork = c.take<float>(2 * (L + 32) * (L + 32));
    w.luscr = g.lu ? c.take<int>(tslu_scratch_ints(std::max(g.ldm, g.ldn), g.L)) : nullptr;
    w.A8 = w.At8 = w.P8 = nullptr;
    w.rs8 = w.ts8 = nullptr;
    w.cm8 = nullptr;
    w.ld8 = round_up(g.sn(), 16);
    w.ldt8 = round_up(g.sm(), 16);
    w.ldp8 = round_up(std::max(g.m, g.n), 16);
    if (g.fp8) {
        w.A8 = c.take<uint8_t>((size_t)g.sm() * w.ld8);
        w.At8 = c.take<uint8_t>((size_t)g.sn() * w.ldt8);
        w.P8 = c.take<uint8_t>((size_t)g.L * w.ldp8);
        w.rs8 = c.take<float>(g.sm());
        w.ts8 = c.take<float>(g.L);
        w.cm8 = c.take<unsigned int>(g.L + 1);
    }
    w.amax = c.take<unsigned int>(1);
    w.Ppinv = c.take<float>(L);
    w.Qpinv = c.take<float>(L);
    w.status = c.take<int>(1);
    w.breakdowns = c.take<int>(1);
    w.sweeps = c.take<int>(1);
    w.fro2 = c.take<double>(1);
    w.orth = c.take<float>(1);
    w.mu = w.cmul = nullptr;
    w.spart = nullptr;
    w.hpart = w.fpart = nullptr;
    w.hvec = nullptr;
    w.Xb = w.Rk = w.Zw = w.Cw = nullptr;
    w.pnrm = w.slot_v = nullptr;
    w.slot_i = nullptr;
    w.piv = nullptr;
    w.bar = nullptr;
    if (g.rid_k > 0) {
        const int kk = g.rid_k;
        w.Xb = c.take<float>(L * g.n);
        w.Rk = c.take<float>((size_t)kk * g.n);
        w.Zw = c.take<float>((size_t)kk * g.n);
        w.pnrm = c.take<double>(std::max(g.m, g.n));
        w.slot_v = c.take<double>(kPqrSlots);
        w.slot_i = c.take<int64_t>(kPqrSlots);
        w.piv = c.take<int>(2 * kk);
        w.bar = c.take<unsigned int>(1);
        if (g.rid_cur) w.Cw = c.take<float>((size_t)g.m * kk);
    }
    if (g.pca_nvar > 0) {
        const bool vars_are_cols = (g.swap_uv == g.trans);
        const int64_t chunks = stats_chunks(vars_are_cols, g.sm(), g.sn(), sm_count);
        w.mu = c.take<float>(g.pca_nvar);
        w.cmul = c.take<float>(g.pca_nvar);
        w.spart = c.take<double2>(chunks * g.pca_nvar);
        w.hpart = c.take<double>((size_t)kAffineMaxChunks * L);
        w.fpart = c.take<double>(ceil_div(g.pca_nvar, 32));
        w.hvec = c.take<float>(L);
    }
}

int ensure_workspace(rsvdgb_handle* h, size_t bytes)
{
    if (bytes <= h->ws_bytes) return RSVDGB_OK;
    if (h->ws) {
        cudaStreamSynchronize(h->stream);
        cudaFree(h->ws);
        h->ws = nullptr;
        h->ws_bytes = 0;
    }
    if (cudaMalloc(&h->ws, bytes) != cudaSuccess) {
        cudaGetLastError();
        return RSVDGB_ERR_NOMEM;
    }
    h->ws_bytes = bytes;
    RSVDGB_CUDA_TRY(cudaMemsetAsync(h->ws, 0, bytes, h->stream));
    return RSVDGB_OK;
}

// ----- tall-skinny products on the logical matrix ---------------------------

// Generic tall product with optional K split: C = op(A) op(B), written to
// C (layout CT) with the partial buffer used when splitting.
void prof_mark(rsvdgb_handle* h, bool start, double bytes)
{
    if (!h || !h->prof.on) return;
    PassProfile& p = h->prof;
    const size_t idx = 2 * p.used + (start ? 0 : 1);
    while (p.ev.size() <= idx) {
        cudaEvent_t e;
        if (cudaEventCreate(&e) != cudaSuccess) {
            p.on = false;
            return;
        }
        p.ev.push_back(e);
    }
    cudaEventRecord(p.ev[idx], h->stream);
    if (!start) {
        p.used += 1;
        p.bytes += bytes;
    }
}

// When `prof` is non-null the main product kernel is bracketed by an event
// pair and counted as one pass over A of `pass_bytes` algorithmic bytes.
void tall_gemm(cudaStream_t s, int sm, bool AT, bool BT, bool CT, const void* A, int64_t lda, int a_bf16,
               const float* B, int64_t ldb, float* C, int64_t ldc, int64_t M, int64_t N, int64_t K, float* part,
               double* fro2, rsvdgb_handle* prof = nullptr, double pass_bytes = 0.0)
{
    GemmArgs a{};
    a.A = A;
    a.lda = lda;
    a.a_bf16 = a_bf16;
    a.B = B;
    a.ldb = ldb;
    a.M = M;
    a.N = N;
    a.K = K;
    a.fro2 = fro2;
    const int64_t tiles = ceil_div(M, 64) * ceil_div(N, 64);
    const int splits = splits_for(tiles, K, sm);
    if (splits <= 1) {
        a.C = C;
        a.ldc = ldc;
        a.splits = 1;
        a.split_stride = 0;
        prof_mark(prof, true, 0);
        launch_simt_gemm(s, AT, BT, CT, a);
        prof_mark(prof, false, pass_bytes);
        return;
    }
    // partials in the same layout as C but packed with leading dimension ldc
    const int64_t rows = CT ? N : M, cols = CT ? M : N;
    a.C = part;
    a.ldc = ldc;
    a.splits = splits;
    a.split_stride = rows * ldc;
    prof_mark(prof, true, 0);
    launch_simt_gemm(s, AT, BT, CT, a);
    prof_mark(prof, false, pass_bytes);
    launch_reduce_splits(s, part, splits, rows * ldc, rows, cols, ldc, C, ldc);
}

double a_bytes(const Geom& g) { return (double)g.m * (double)g.n * (g.a_bf16 ? 2.0 : 4.0); }

// One pass over A:  out = A_logical P (A_side) or A_logical^T P (!A_side).
// P is column-major (K x l, ldP) in FP32 (SIMT engine) or as its split parts
// (tensor-core engine: TF32 hi / lo, or FP16 hi / lo with x->h16).  out is
// column-major (rows x l, ldO); when out_h/out_l are given (tensor-core
// engine) they receive its TF32 split.
void pass_over_A(rsvdgb_handle* h, const Geom& g, Work& w, bool A_side, const float* P, const float* Ph,
                 const float* Pl, float* out, float* out_h, float* out_l, double* fro2, const void* Pbf = nullptr,
                 int chunk = 0, const float* aff_h = nullptr, const float* aff_u = nullptr,
                 const float* aff_r = nullptr, const TcExtra* x = nullptr)
{
    const cudaStream_t s = h->stream;
    const int64_t rows = A_side ? g.m : g.n;
    const int64_t K = A_side ? g.n : g.m;
    const int64_t ldP = A_side ? g.ldn : g.ldm;
    const int64_t ldO = A_side ? g.ldm : g.ldn;
    if (!g.use_tc) {
        // logical(i,k) = trans ? S[k*lda + i] : S[i*lda + k]; the transpose flips it
        const bool AT = A_side ? g.trans : !g.trans;
        tall_gemm(s, h->sm_count, AT, true, true, g.A, g.lda, g.a_bf16, P, ldP, out, ldO, rows, g.l, K, w.part,
                  fro2, h, a_bytes(g));
        return;
    }
    // Tensor-core engine.  The kernel's lanes are stored rows (A X kernel) or
    // stored columns (A^T X kernel, K split across CTAs, partials reduced).
    const bool stored_atx = (A_side == g.trans);
    int64_t splits = 0;
    prof_mark(h, true, 0);
    if (Pbf)
        launch_tc_gemm(s, h->sm_count, stored_atx, (const float*)g.A, g.sm(), g.sn(), g.lda, (const float*)Pbf,
                       nullptr, ldP, g.L, out, out_h, out_l, ldO, w.part, stored_atx ? 0 : 1, &splits, w.status, fro2,
                       0, 0, 1, g.a_bf16, chunk, aff_h, aff_u, aff_r, x);
    else
        launch_tc_gemm(s, h->sm_count, stored_atx, (const float*)g.A, g.sm(), g.sn(), g.lda, Ph, Pl, ldP, g.L, out,
                       out_h, out_l, ldO, w.part, stored_atx ? 0 : 1, &splits, w.status, fro2, 0, 0, 0, g.a_bf16,
                       chunk, aff_h, aff_u, aff_r, x);
    prof_mark(h, false, a_bytes(g));
    if (splits > 0) {
        launch_reduce_splits(s, w.part, (int)splits, (int64_t)g.L * ldO, g.l, rows, ldO, out, ldO);
        if (out_h) launch_split_tf32(s, out, ldO, rows, g.l, g.L, out_h, out_l);
    }
}

// Scale of the FP16 hi / lo split of an m-side basis Q (the panel of an
// FP16x3 A^T-side pass): its columns are unit vectors up to rounding, so
// |q_ij| <= 1 (a little more after a Cholesky step on an ill-conditioned
// sketch) and 2^13 keeps them below FP16's range with room to spare.
constexpr float kQSplitScale = 8192.f;

// G (l x l) = X^T X for a column-major rows x l matrix X (leading dimension
// ld) on the tensor cores (3xTF32).  Up to l_pad = 128 the Gram kernel reads
// X once; wider sketches use the pass kernel on X^T with the TF32 hi/lo
// parts of X (Xh, Xl) as its panel.
bool tc_gram_direct(const Geom& g, const float* Xt, int64_t ld) { return tc_gram_supported(Xt, nullptr, ld, g.L); }

void tc_gram(rsvdgb_handle* h, const Geom& g, Work& w, const float* Xt, const float* Xh, const float* Xl, int64_t ld,
             int64_t rows)
{
    if (tc_gram_direct(g, Xt, ld)) {
        launch_tc_gram(h->stream, h->sm_count, Xt, nullptr, rows, ld, g.l, g.L, w.part, w.G, w.status);
        return;
    }
    int64_t splits = 0;
    launch_tc_gemm(h->stream, h->sm_count, false, Xt, g.L, rows, ld, Xh, Xl, ld, g.L, nullptr, nullptr, nullptr, g.L,
                   w.part, 0, &splits, w.status, nullptr, 0, 0, 0, 0, kExactChunk);
    launch_reduce_splits(h->stream, w.part, (int)splits, (int64_t)g.L * g.L, g.l, g.l, g.L, w.G, g.l);
}

// Z = X T (rows x l, column-major) for a column-major rows x l matrix X and
// an l x l row-major upper triangular T.  Zh / Zl (optional) receive
// Z's split: TF32 hi / lo floats, or with f16 the FP16 hi / lo (uint16) of
// kQSplitScale Z (Z is then a basis with unit columns).
void tc_times_small(rsvdgb_handle* h, const Geom& g, Work& w, const float* Xt, int64_t ld, int64_t rows,
                    const float* T, float* Zt, float* Zh, float* Zl, bool f16 = false)
{
    // T is a Cholesky factor's inverse (upper triangular): up to l_pad = 112
    // the FP32 FMA kernel streams X once at the bandwidth bound
    if (xt_supported(g.L) && launch_xt(h->stream, h->sm_count, Xt, ld, rows, g.l, g.L, T, Zt,
                                       Zh ? (f16 ? 2 : 1) : 0, Zh, Zl, kQSplitScale) == RSVDGB_OK)
        return;
    launch_small_panel(h->stream, T, g.l, g.L, w.Th, w.Tl);
    int64_t splits = 0;
    TcExtra x{};
    if (f16 && Zh) {
        x.out_h16 = (uint16_t*)Zh;
        x.out_l16 = (uint16_t*)Zl;
        x.split_sc_const = kQSplitScale;
    }
    launch_tc_gemm(h->stream, h->sm_count, true, Xt, g.L, rows, ld, w.Th, w.Tl, g.L, g.L, Zt, f16 ? nullptr : Zh,
                   f16 ? nullptr : Zl, ld, nullptr, 1, &splits, w.status, nullptr, 0, 0, 0, 0, 0, nullptr, nullptr,
                   nullptr, f16 ? &x : nullptr);
}

// One FP8 pass: out (rows x l, column-major) = A_logical P (A_side) or
// A_logical^T P, P the FP32 panel (K x l, column-major).  The lanes of the
// FP8 kernel are the stored rows (A8, whose row powers of two scale the
// output) or the stored columns (At8; K then runs over the stored rows, whose
// powers of two scale the panel before it is quantised).
void pass_fp8(rsvdgb_handle* h, const Geom& g, Work& w, bool A_side, const float* P, float* out)
{
    const cudaStream_t s = h->stream;
    const bool stored_atx = (A_side == g.trans);
    const int64_t K = A_side ? g.n : g.m;
    const int64_t rows = A_side ? g.m : g.n;
    const int64_t ldP = A_side ? g.ldn : g.ldm;
    const int64_t ldO = A_side ? g.ldm : g.ldn;
    launch_fp8_panel(s, P, ldP, K, g.l, g.L, stored_atx ? w.rs8 : nullptr, w.P8, w.ldp8, w.ts8, w.cm8);
    int64_t splits = 0;
    prof_mark(h, true, 0);
    launch_f8_pass(s, h->sm_count, stored_atx, stored_atx ? w.At8 : w.A8, rows, K, stored_atx ? w.ldt8 : w.ld8,
                   w.P8, w.ldp8, g.L, stored_atx ? nullptr : w.rs8, w.ts8, out, ldO, w.part, &splits, w.status);
    prof_mark(h, false, (double)g.m * (double)g.n);
    if (splits > 0) launch_reduce_splits(s, w.part, (int)splits, (int64_t)g.L * ldO, g.l, rows, ldO, out, ldO);
}

// Y = A_logical X with X = Pt (n x l) -> Yt (m x l).  The first pass
// (first = true) measures ||A||_F^2 (fro2) and, for the FP16x3 form, max|A|;
// later passes use the FP16x3 form where the geometry has it (the panel's
// FP16 split in Pth / Ptl, scales in Ppinv).  Y's TF32 split goes to Yth /
// Ytl only when the Gram of Y runs on the pass kernel (wide sketches).
// In mixed precision the product runs in BF16 on the BF16 copy of the panel.
// With an affine map (randomized PCA) the result is Y = X_pca Pt: the panel
// was already scaled by split_panel when the variables are the columns;
// here the correction Y = r (A P - u h^T) follows the pass, with
// h = P^T mu (columns: u = 1, r = 1) or h = P^T 1 (rows: u = mu, r = c).
void apply_A(rsvdgb_handle* h, const Geom& g, Work& w, double* fro2, bool first)
{
    if (g.fp8) {
        // the statistics of A came from the FP8 copy's pass (launch_fp8_prep)
        pass_fp8(h, g, w, true, w.Pt, w.Yt);
        if (!tc_gram_direct(g, w.Yt, g.ldm)) launch_split_tf32(h->stream, w.Yt, g.ldm, g.m, g.l, g.L, w.Yth, w.Ytl);
        return;
    }
    const Affine* af = g.aff;
    const bool corr = af && (af->mu || (af->rows && af->c));
    int chunks = 0;
    if (af && af->mu)
        launch_affine_dot(h->stream, h->sm_count, w.Pt, g.ldn, g.n, g.l, af->rows ? nullptr : af->mu, af->part,
                          &chunks);
    // the tensor-core A-side pass on row-major A writes Y directly: the
    // correction runs in its epilogue; otherwise in a separate kernel
    const bool fused = corr && g.use_tc && !g.trans;
    const float *fh = nullptr, *fu = nullptr, *fr = nullptr;
    if (fused) {
        if (af->mu) {
            launch_affine_h(h->stream, af->part, chunks, g.l, w.hvec);
            fh = w.hvec;
            fu = af->rows ? af->mu : nullptr;
        }
        fr = af->rows ? af->c : nullptr;
    }
    const bool y_split = g.use_tc && !tc_gram_direct(g, w.Yt, g.ldm);
    TcExtra x{};
    const bool h16 = g.h16 && !first && !g.bf16;
    if (g.h16 && first) x.amax_out = w.amax;
    if (h16) {
        x.h16 = 1;
        x.amax_in = w.amax;
        x.pinv = w.Ppinv;
    }
    pass_over_A(h, g, w, true, w.Pt, w.Pth, w.Ptl, w.Yt, y_split ? w.Yth : nullptr, y_split ? w.Ytl : nullptr,
                af ? nullptr : fro2, g.bf16 ? w.Ptb : nullptr, 0, fh, fu, fr, g.use_tc ? &x : nullptr);
    if (corr && !fused)
        launch_affine_post(h->stream, w.Yt, g.ldm, g.m, g.l, af->rows ? af->c : nullptr,
                           af->rows ? af->mu : nullptr, af->mu ? af->part : nullptr, chunks,
                           y_split ? w.Yth : nullptr, y_split ? w.Ytl : nullptr);
}

// W = A_logical^T X with the m-side basis X (m x l, column-major, ldm; its
// split in Xh / Xl: TF32 hi / lo, or the FP16 hi / lo of kQSplitScale X when
// the geometry runs FP16x3) -> Wt (n x l).  `accurate` keeps the
// FP32-accurate product (the projection B = Q^T A); otherwise mixed precision
// runs it in BF16.  With an affine map: W = X_pca^T X, i.e.
// W = c (A^T X - mu h^T) with h = X^T 1 (variables = columns), or
// W = A^T (c X) - 1 h^T with h = (c X)^T mu (rows; c X staged in the scratch
// buffer S with its TF32 split Sh / Sl).
void apply_At(rsvdgb_handle* h, const Geom& g, Work& w, bool accurate, const float* X, const float* Xh,
              const float* Xl, float* S, float* Sh, float* Sl)
{
    if (g.fp8 && !accurate) {
        pass_fp8(h, g, w, false, X, w.Wt);
        return;
    }
    const Affine* af = g.aff;
    const cudaStream_t s = h->stream;
    const bool mixed = g.bf16 && !accurate;
    const float *Y = X, *Yh = Xh, *Yl = Xl;
    if (af && af->rows && af->c) {
        const bool want_split = g.use_tc && !mixed;
        launch_scale_rows(s, X, g.ldm, g.m, g.l, g.L, af->c, S, want_split ? Sh : nullptr,
                          want_split ? Sl : nullptr);
        Y = S;
        Yh = Sh;
        Yl = Sl;
    }
    int chunks = 0;
    if (af && af->mu)
        launch_affine_dot(s, h->sm_count, Y, g.ldm, g.m, g.l, af->rows ? af->mu : nullptr, af->part, &chunks);
    if (mixed) {
        launch_to_bf16(s, Y, g.ldm, g.m, g.l, g.L, w.Ytb);
        pass_over_A(h, g, w, false, Y, nullptr, nullptr, w.Wt, nullptr, nullptr, nullptr, w.Ytb);
    } else {
        TcExtra x{};
        if (g.h16) {
            x.h16 = 1;
            x.amax_in = w.amax;
            x.pinv = w.Qpinv;
        }
        // the projection B = Q^T A (accurate) keeps its scale: short accumulation chains
        pass_over_A(h, g, w, false, Y, Yh, Yl, w.Wt, nullptr, nullptr, nullptr, nullptr, accurate ? kExactChunk : 0,
                    nullptr, nullptr, nullptr, g.h16 ? &x : nullptr);
    }
    if (af && (af->mu || (!af->rows && af->c)))
        launch_affine_post(s, w.Wt, g.ldn, g.n, g.l, af->rows ? nullptr : af->c, af->rows ? nullptr : af->mu,
                           af->mu ? af->part : nullptr, chunks, nullptr, nullptr);
}

// After the panel Pt changed: its split for the tensor-core engine -- TF32
// hi / lo for the first pass, the scaled FP16 hi / lo (with Ppinv) for the
// later FP16x3 passes -- or its BF16 copy in mixed precision.  With an affine
// map whose variables are the logical columns, the panel is first scaled by
// the multipliers (P <- diag(c) P).
void split_panel(cudaStream_t s, const Geom& g, Work& w, bool first)
{
    if (g.fp8) return;  // quantised by the FP8 pass itself
    if (g.aff && !g.aff->rows && g.aff->c) {
        const bool tf = g.use_tc && !g.bf16;
        launch_scale_rows(s, w.Pt, g.ldn, g.n, g.l, g.L, g.aff->c, w.Pt, tf ? w.Pth : nullptr, tf ? w.Ptl : nullptr);
        if (g.bf16) launch_to_bf16(s, w.Pt, g.ldn, g.n, g.l, g.L, w.Ptb);
        return;
    }
    if (g.bf16)
        launch_to_bf16(s, w.Pt, g.ldn, g.n, g.l, g.L, w.Ptb);
    else if (g.h16 && !first)
        launch_panel_f16(s, w.Pt, g.ldn, g.n, g.l, g.L, (uint16_t*)w.Pth, (uint16_t*)w.Ptl, w.Ppinv);
    else if (g.use_tc)
        launch_split_tf32(s, w.Pt, g.ldn, g.n, g.l, g.L, w.Pth, w.Ptl);
}

// G (l x l) = X^T Z for column-major rows x l matrices X and Z
// (Z = X gives the Gram matrix).
void cross_gram(cudaStream_t s, int sm, const float* Xt, const float* Zt, int64_t ld, int64_t rows, int l,
                float* part, float* G, int l_pad = 0, int* status = nullptr)
{
    if (l_pad > 0 && tc_gram_supported(Xt, Zt, ld, l_pad)) {
        launch_tc_gram(s, sm, Xt, Zt, rows, ld, l, l_pad, part, G, status);
        return;
    }
    GemmArgs a{};
    a.A = Xt;
    a.lda = ld;
    a.B = Zt;
    a.ldb = ld;
    a.M = l;
    a.N = l;
    a.K = rows;
    const int64_t tiles = ceil_div(l, 64) * ceil_div(l, 64);
    const int splits = splits_for(tiles, rows, sm);
    a.C = part;
    a.ldc = l;
    a.splits = splits;
    a.split_stride = (int64_t)l * l;
    launch_simt_gemm(s, false, true, false, a);
    launch_reduce_splits(s, part, splits, (int64_t)l * l, l, l, l, G, l);
}

void gram(cudaStream_t s, int sm, const float* Xt, int64_t ld, int64_t rows, int l, float* part, float* G,
          int l_pad = 0, int* status = nullptr)
{
    cross_gram(s, sm, Xt, Xt, ld, rows, l, part, G, l_pad, status);
}

// Zt (rows x l, column-major) = X T with X column-major (rows x l) and T an
// l x l row-major matrix.
void times_small(cudaStream_t s, int sm, const float* Xt, int64_t ld, int64_t rows, int l, const float* T, float* Zt,
                 float* part)
{
    tall_gemm(s, sm, true, false, true, Xt, ld, 0, T, l, Zt, ld, rows, l, l, part, nullptr);
}

// CholeskyQR2 of a column-major rows x l matrix X (in Xt): Q1 = X R1^{-1},
// Q = Q1 R2^{-1}, the orthonormal basis written to Qt (tmp holds Q1; Xt, tmp
// and Qt are distinct).  l_pad > 0 puts the Grams on the tensor cores where
// the shape allows it.
void cholqr2(cudaStream_t s, int sm, Work& w, const float* Xt, int64_t ld, int64_t rows, int l, float* tmp, float* Qt,
             int l_pad)
{
    gram(s, sm, Xt, ld, rows, l, w.part, w.G, l_pad, w.status);
    launch_chol_inv(s, w.G, l, 0.f, w.R1, w.T1, w.status, w.breakdowns);
    times_small(s, sm, Xt, ld, rows, l, w.T1, tmp, w.part);
    gram(s, sm, tmp, ld, rows, l, w.part, w.G, l_pad, w.status);
    launch_chol_inv(s, w.G, l, 0.f, w.R2, w.T2, w.status, w.breakdowns);
    times_small(s, sm, tmp, ld, rows, l, w.T2, Qt, w.part);
}

struct Outputs {
    float* d;
    float* U;  // logical left vectors, row-major (ldU), nU columns
    int64_t ldU;
    int nU;
    float* V;  // logical right vectors
    int64_t ldV;
    int nV;
    float* Qrow;  // optional row-major Q (m x l) for rqb
    int64_t ldq;
    float* Brow;  // optional row-major B (l x n) for rqb
    int64_t ldb;
    rsvdgb_info* info;
    bool check_orth;  // measure max |Q^T Q - I| of the final basis into info.orth_max
    int sigma_cols;  // 1: columns of the logical U scaled by sigma; 2: of V (PCA scores)
    const struct RidSpec* rid;  // interpolative / CUR decomposition instead of the SVD of B
};

// Outputs of Algorithms rid / rcur (device pointers; C, Z, U, R may be null).
struct RidSpec {
    bool cur;
    float* C;
    int64_t ldc;  // m x k
    float* Z;
    int64_t ldz;  // k x n
    int64_t* J;   // k column indices
    float* U;
    int64_t ldu;  // k x k
    float* R;
    int64_t ldr;  // k x n
    int64_t* I;   // k row indices
};

// Randomized PCA on top of the rSVD (Algorithm rpca): centring / scaling
// flags, the user's optional copies of the centre and scale, the eigenvalue
// and standard-deviation outputs, and the number of observations.
struct PcaSpec {
    int center, scale;
    float *center_out, *scale_out;
    float *eig, *sdev;
    int64_t m_obs;
};

// Algorithm rqb (+ rSVD when d != nullptr) on the logical matrix.
// Learned choice of (q, p): the sketch is taken at the widest width, the
// controller's decision is read back (one stream synchronisation) and the
// run continues with the first k + p columns of that sketch.
struct Learned {
    int k;
    int p_max, q_max;
    float* feats_out;  // features only (rsvdgb_controller_features): stop after them
};

// Steps 2-3 at the geometry g: Omega, Y = A Omega with ||A||_F^2, Gram of Y.
void sketch(rsvdgb_handle* h, const Geom& g, Work& w, int sdist, uint64_t seed)
{
    const cudaStream_t s = h->stream;
    launch_omega(s, g.n, g.ldn, g.l, g.L, seed, sdist, w.Pt, g.ldn);
    split_panel(s, g, w, true);
    if (g.fp8)
        launch_fp8_prep(s, g.A, g.lda, g.a_bf16, g.sm(), g.sn(), w.A8, w.ld8, w.At8, w.ldt8, w.rs8, w.fro2,
                        w.amax);
    apply_A(h, g, w, w.fro2, true);
    if (g.use_tc)
        tc_gram(h, g, w, w.Yt, w.Yth, w.Ytl, g.ldm, g.m);
    else
        gram(s, h->sm_count, w.Yt, g.ldm, g.m, g.l, w.part, w.G);
}

// Controller features of the sketch in w (its Gram in w.G), from the
// CholeskyQR factor R of Y (Y = Q R) and ||A||_F^2.
void sketch_features(rsvdgb_handle* h, const Geom& g, Work& w, int k, int p_max, float* feats)
{
    const cudaStream_t s = h->stream;
    launch_chol_inv(s, w.G, g.l, 0.f, w.R1, w.T, w.status, w.breakdowns);
    launch_controller_features(s, w.R1, g.l, w.fro2, g.m, g.n, k, p_max, feats);
}

// Algorithm id on B (from B^T in Wt) and the rest of Algorithms rid / rcur.
int rid_tail(rsvdgb_handle* h, const Geom& g, Work& w, int k, const RidSpec& r)
{
    const cudaStream_t s = h->stream;
    const int sm = h->sm_count;
    const int l = g.l;
    // B (l x n, column j contiguous) from B^T
    launch_transpose_cm(s, w.Wt, g.ldn, g.n, l, w.Xb, g.L);
    const int absent = h->test_pqr_absent ? 0 : -1;
    const long long spin = h->test_pqr_absent ? h->test_spin : 0;
    h->test_pqr_absent = 0;
    int rc = launch_pqr(s, sm, w.Xb, g.L, l, g.n, k, w.piv, w.Rk, w.pnrm, w.slot_v, w.slot_i, kPqrSlots, w.bar,
                        w.status, spin, absent);
    if (rc) return rc;
    float* Z = r.Z ? r.Z : w.Zw;
    const int64_t ldz = r.Z ? r.ldz : g.n;
    launch_id_solve(s, w.Rk, g.n, k, w.piv, Z, ldz, w.status);
    launch_piv_to_i64(s, w.piv, k, r.J);
    float* C = r.C ? r.C : (r.cur ? w.Cw : nullptr);
    const int64_t ldc = r.C ? r.ldc : k;
    if (C) launch_gather_cols(s, g.A, g.lda, g.a_bf16, g.trans, g.m, w.piv, k, C, ldc);
    if (!r.cur) return RSVDGB_OK;
    // row pivots: the pivoted QR of C^T (k x m; its column i is row i of C)
    rc = launch_pqr(s, sm, C, ldc, k, g.m, k, w.piv + k, nullptr, w.pnrm, w.slot_v, w.slot_i, kPqrSlots, w.bar,
                    w.status);
    if (rc) return rc;
    launch_piv_to_i64(s, w.piv + k, k, r.I);
    // R = A(I, :) and R^T (n x k column-major, zero beyond column k) in Wt
    RSVDGB_CUDA_TRY(cudaMemsetAsync(w.Wt, 0, sizeof(float) * (size_t)g.L * g.ldn, s));
    launch_gather_rows(s, g.A, g.lda, g.a_bf16, g.trans, g.n, w.piv + k, k, r.R, r.ldr, w.Wt, g.ldn);
    // U = Z pinv(R): R^T = Q_R S (CholeskyQR2), pinv(R) = Q_R S^{-T},
    // U = (Z Q_R) (T1 T2)^T with S^{-1} = T1 T2
    cholqr2(s, sm, w, w.Wt, g.ldn, g.n, k, w.Zt, w.Pt, g.use_tc ? (int)round_up(k, 16) : 0);
    launch_zq(s, Z, ldz, w.Pt, g.ldn, g.n, k, w.M);
    launch_small_matmul(s, w.T1, w.T2, w.RB, k);
    launch_small_transpose(s, w.RB, w.Ut, k);
    launch_small_matmul(s, w.M, w.Ut, w.Jt, k);
    if (r.U)
        RSVDGB_CUDA_TRY(cudaMemcpy2DAsync(r.U, r.ldu * sizeof(float), w.Jt, k * sizeof(float), k * sizeof(float), k,
                                          cudaMemcpyDeviceToDevice, s));
    return RSVDGB_OK;
}

int engine_code(const Geom& g)
{
    return !g.use_tc ? RSVDGB_ENGINE_SIMT : (g.h16 ? RSVDGB_ENGINE_TC : RSVDGB_ENGINE_TC_TF32);
}

int run_fp32(rsvdgb_handle* h, Geom g, int k, int q, int sdist, uint64_t seed, const Outputs& o,
             const Learned* lc = nullptr, const PcaSpec* pca = nullptr)
{
    const cudaStream_t s = h->stream;
    const int sm = h->sm_count;
    // the randomized PCA's implicit centring runs on the 3xTF32 or BF16 passes
    if (pca) g.h16 = false;
    if (pca && g.fp8) return RSVDGB_ERR_UNSUPPORTED;
    Carve probe(nullptr);
    Work w{};
    const int L_lo = lc ? (int)round_up(std::min<int64_t>((int64_t)k + 2, g.n), 16) : 0;
    carve_work(probe, g, sm, w, L_lo);
    int rc = ensure_workspace(h, probe.off + 1024);
    if (rc) return rc;
    Carve c(h->ws);
    carve_work(c, g, sm, w, L_lo);

    // the m-side bases carry the fixed FP16 split scale kQSplitScale
    launch_clear_scalars(s, w.status, w.breakdowns, w.fro2, w.amax, w.Qpinv, g.L, 1.f / kQSplitScale, w.cm8,
                         w.cm8 ? g.L + 1 : 0);
    Affine aff{};
    if (pca) {
        // randomized PCA: per-variable centre and scale in one pass over A;
        // every later product with A becomes a product with the centred,
        // scaled X (||X||_F^2 comes from the statistics)
        launch_var_stats(s, sm, g.A, g.lda, g.sm(), g.sn(), g.a_bf16, g.swap_uv == g.trans, pca->center,
                         pca->scale, w.spart, w.mu, w.cmul, pca->center_out, pca->scale_out, w.fpart, w.fro2);
        aff.rows = g.swap_uv;
        aff.mu = pca->center ? w.mu : nullptr;
        aff.c = pca->scale ? w.cmul : nullptr;
        aff.part = w.hpart;
        g.aff = &aff;
    }
    // steps 2-3: Omega (n x l) into the panel, Y = A Omega with ||A||_F^2, Gram
    sketch(h, g, w, sdist, seed);
    if (lc) {
        float* feats = lc->feats_out ? lc->feats_out : h->ctl_scratch;
        sketch_features(h, g, w, k, lc->p_max, feats);
        if (lc->feats_out) {
            RSVDGB_CUDA_TRY(cudaGetLastError());
            return RSVDGB_OK;
        }
        // a shifted retry of the sketch's Cholesky (a sketch wider than the rank
        // of A) is not a breakdown of the factorisation that is reported
        RSVDGB_CUDA_TRY(cudaMemsetAsync(w.status, 0, sizeof(int), s));
        RSVDGB_CUDA_TRY(cudaMemsetAsync(w.breakdowns, 0, sizeof(int), s));
        float* out2 = h->ctl_scratch + 16;
        int* qp = (int*)(h->ctl_scratch + 32);
        launch_mlp_forward(s, h->ctl_params, feats, 1, out2);
        launch_controller_decide(s, out2, lc->q_max, 2, lc->p_max, k, g.n, qp);
        RSVDGB_CUDA_TRY(cudaMemcpyAsync(h->ctl_host, qp, 2 * sizeof(int), cudaMemcpyDeviceToHost, s));
        RSVDGB_CUDA_TRY(cudaStreamSynchronize(s));
        q = h->ctl_host[0];
        // continue with the first k + p columns of the sketch (Omega nested in l)
        const int lw = g.l;
        g.l = (int)std::min<int64_t>((int64_t)k + h->ctl_host[1], g.n);
        g.L = (int)round_up(g.l, 16);
        // the Gram of the first l columns is the leading l x l block of the
        // wide sketch's Gram (each entry is the same sum of products)
        if (g.l < lw) {
            const size_t row = sizeof(float) * (size_t)g.l;
            RSVDGB_CUDA_TRY(cudaMemcpy2DAsync(w.M, row, w.G, sizeof(float) * (size_t)lw, row, (size_t)g.l,
                                              cudaMemcpyDeviceToDevice, s));
            RSVDGB_CUDA_TRY(cudaMemcpyAsync(w.G, w.M, row * (size_t)g.l, cudaMemcpyDeviceToDevice, s));
        }
    }
    const int l = g.l;
    // split of an m-side basis for the A^T-side pass that reads it: none in
    // mixed precision (BF16 copy), FP16 with the FP16x3 passes, else TF32
    const bool q_split = g.use_tc && !g.bf16 && !g.fp8;
    // step 4, Algorithm norm_iterations: each sketch is renormalised by the L
    // factor of a pivoted LU, L = Y U^{-1} (U from the tall-skinny LU's pivot
    // rows); only the final basis (step 9) is orthonormal
    for (int it = 0; it < q && g.lu; ++it) {
        launch_tslu(s, w.Yt, g.ldm, g.m, l, w.luscr, w.R1, w.T, w.status);
        tc_times_small(h, g, w, w.Yt, g.ldm, g.m, w.T, w.Qt, q_split ? w.Qth : nullptr, q_split ? w.Qtl : nullptr,
                       g.h16);
        apply_At(h, g, w, false, w.Qt, w.Qth, w.Qtl, w.Yt, w.Yth, w.Ytl);
        launch_tslu(s, w.Wt, g.ldn, g.n, l, w.luscr, w.R2, w.T1, w.status);
        times_small(s, sm, w.Wt, g.ldn, g.n, l, w.T1, w.Pt, w.part);
        split_panel(s, g, w, false);
        apply_A(h, g, w, nullptr, false);
        if (it == q - 1) tc_gram(h, g, w, w.Yt, w.Yth, w.Ytl, g.ldm, g.m);
    }
    // step 4, Algorithm sub_iterations
    for (int it = 0; it < q && !g.lu; ++it) {
        // Q = qr(Y) by one Cholesky step, Q = Y R^{-1}: only the span is carried
        // forward.  Q is formed before A^T Q so that the directions of small
        // singular values keep their relative accuracy (A^T Y T would carry
        // them at the size sigma^2 / sigma_1^2 within its columns).
        launch_chol_inv(s, w.G, l, 0.f, w.R1, w.T, w.status, w.breakdowns);
        if (g.use_tc)
            tc_times_small(h, g, w, w.Yt, g.ldm, g.m, w.T, w.Qt, q_split ? w.Qth : nullptr,
                           q_split ? w.Qtl : nullptr, g.h16);
        else
            times_small(s, sm, w.Yt, g.ldm, g.m, l, w.T, w.Qt, w.part);
        apply_At(h, g, w, false, w.Qt, w.Qth, w.Qtl, w.Yt, w.Yth, w.Ytl);
        // Q = qr(A^T Q) on the n side: here too only the span is carried
        // forward, so one CholeskyQR step, Q_n = Z R^{-1}, into the panel
        gram(s, sm, w.Wt, g.ldn, g.n, l, w.part, w.G, g.use_tc ? (int)g.L : 0, w.status);
        launch_chol_inv(s, w.G, l, 0.f, w.R1, w.T1, w.status, w.breakdowns);
        times_small(s, sm, w.Wt, g.ldn, g.n, l, w.T1, w.Pt, w.part);
        split_panel(s, g, w, false);
        // Y = A Q
        apply_A(h, g, w, nullptr, false);
        if (g.use_tc)
            tc_gram(h, g, w, w.Yt, w.Yth, w.Ytl, g.ldm, g.m);
        else
            gram(s, sm, w.Yt, g.ldm, g.m, l, w.part, w.G);
    }
    // step 9: Q = qr(Y) with CholeskyQR2 (the first Gram is already in G):
    // Y1 = Y T1, G = Y1^T Y1, Q = Y1 T2.  Q ends up in Yt.
    launch_chol_inv(s, w.G, l, 0.f, w.R1, w.T1, w.status, w.breakdowns);
    if (g.use_tc) {
        // the TF32 split of Q1 is needed only when the Gram runs on the pass kernel
        const bool direct = tc_gram_direct(g, w.Qt, g.ldm);
        tc_times_small(h, g, w, w.Yt, g.ldm, g.m, w.T1, w.Qt, direct ? nullptr : w.Qth, direct ? nullptr : w.Qtl);
        tc_gram(h, g, w, w.Qt, w.Qth, w.Qtl, g.ldm, g.m);
    } else {
        times_small(s, sm, w.Yt, g.ldm, g.m, l, w.T1, w.Qt, w.part);
        gram(s, sm, w.Qt, g.ldm, g.m, l, w.part, w.G);
    }
    launch_chol_inv(s, w.G, l, 0.f, w.R2, w.T2, w.status, w.breakdowns);
    if (g.use_tc)
        tc_times_small(h, g, w, w.Qt, g.ldm, g.m, w.T2, w.Yt, w.Yth, w.Ytl, g.h16);
    else
        times_small(s, sm, w.Qt, g.ldm, g.m, l, w.T2, w.Yt, w.part);
    // optional check of the final basis: max |Q^T Q - I| from one more Gram
    if (o.check_orth) {
        gram(s, sm, w.Yt, g.ldm, g.m, l, w.part, w.G, (g.use_tc && g.L <= 128) ? (int)g.L : 0, w.status);
        launch_orth_err(s, w.G, l, w.orth);
    }
    // step 10: B^T = A^T Q (n x l, column-major: row j of B is contiguous)
    apply_At(h, g, w, true, w.Yt, w.Yth, w.Ytl, w.Qt, w.Qth, w.Qtl);
    if (o.rid) {
        const int rc = rid_tail(h, g, w, k, *o.rid);
        if (rc) return rc;
        launch_finalize_info(s, nullptr, 0, k, nullptr, w.fro2, w.status, w.breakdowns, q, l - k, engine_code(g),
                             nullptr, o.info, o.check_orth ? w.orth : nullptr);
        RSVDGB_CUDA_TRY(cudaGetLastError());
        return RSVDGB_OK;
    }
    if (o.Qrow) launch_colmajor_to_rowmajor(s, w.Yt, g.ldm, g.m, l, o.Qrow, o.ldq);
    if (o.Brow)
        RSVDGB_CUDA_TRY(cudaMemcpy2DAsync(o.Brow, o.ldb * sizeof(float), w.Wt, g.ldn * sizeof(float),
                                          g.n * sizeof(float), l, cudaMemcpyDeviceToDevice, s));
    if (o.d) {
        // [Ut, S, V] = svd(B): B^T = Q_B R_B, then Jacobi on R_B^T.  R_B is
        // formed as Q_B^T B^T from the computed Q_B, so that B^T = Q_B R_B
        // holds to FP32 rounding whatever the error of the triangular
        // factors (R2 R1 would carry the inverse's error l u kappa).
        cholqr2(s, sm, w, w.Wt, g.ldn, g.n, l, w.Zt, w.Pt, g.use_tc ? (int)g.L : 0);
        cross_gram(s, sm, w.Pt, w.Wt, g.ldn, g.n, l, w.part, w.G, g.use_tc ? (int)g.L : 0, w.status);
        launch_small_transpose(s, w.G, w.M, l);
        launch_jacobi_svd(s, w.M, l, w.sigma, w.Ut, w.Jt, w.jwork, w.sweeps, o.nV);
        // principal component scores Z = U Sigma (Algorithm rpca step 3):
        // scale the small factor before the back-projection
        if (o.sigma_cols == 1) launch_scale_cols_small(s, w.Ut, l, o.nU, w.sigma);
        if (o.sigma_cols == 2) launch_scale_cols_small(s, w.Jt, l, o.nV, w.sigma);
        // U = Q Ut (Eq. UQU) and V = Q_B J, truncated
        if (o.nU > 0) {
            if (g.use_tc) {
                launch_small_panel(s, w.Ut, l, g.L, w.Th, w.Tl);
                int64_t splits = 0;
                launch_tc_gemm(s, sm, true, w.Yt, g.L, g.m, g.ldm, w.Th, w.Tl, g.L, g.L, o.U, nullptr, nullptr, o.ldU,
                               nullptr, 1, &splits, w.status, nullptr, 1, o.nU);
            } else {
                tall_gemm(s, sm, true, false, false, w.Yt, g.ldm, 0, w.Ut, l, o.U, o.ldU, g.m, o.nU, l, w.part,
                          nullptr);
            }
        }
        if (o.nV > 0)
            tall_gemm(s, sm, true, false, false, w.Pt, g.ldn, 0, w.Jt, l, o.V, o.ldV, g.n, o.nV, l, w.part,
                      nullptr);
    } else {
        // rqb only: singular values not requested; still report the QB error
        // through a cheap Gram of B (sigma unused).
    }
    launch_finalize_info(s, o.d ? w.sigma : nullptr, o.d ? l : 0, k, o.d, w.fro2, w.status, w.breakdowns, q,
                         l - k, engine_code(g), o.d ? w.sweeps : nullptr, o.info, o.check_orth ? w.orth : nullptr);
    // Lambda = Sigma^2 / (m - 1) over the singular values just copied to d
    if (pca) launch_pca_values(s, w.sigma, k, pca->m_obs, pca->eig, pca->sdev);
    RSVDGB_CUDA_TRY(cudaGetLastError());
    return RSVDGB_OK;
}

}  // namespace

// ===========================================================================
// C ABI
// ===========================================================================
namespace {

bool aligned(const void* p, size_t a) { return ((uintptr_t)p % a) == 0; }

int check_handle(rsvdgb_handle* h)
{
    if (!h) return RSVDGB_ERR_INVALID_ARG;
    if (cudaSetDevice(h->device) != cudaSuccess) return RSVDGB_ERR_CUDA;
    return RSVDGB_OK;
}

// Validate a user matrix and build the m >= n geometry.
int make_geom(const void* A, int64_t m, int64_t n, int64_t lda, int dtype, int layout, int k, int p, int engine,
              int prec, Geom& g)
{
    if (!A || m < 1 || n < 1) return RSVDGB_ERR_INVALID_ARG;
    if (dtype != RSVDGB_F32 && dtype != RSVDGB_BF16) return RSVDGB_ERR_INVALID_ARG;
    if (layout != RSVDGB_ROW_MAJOR && layout != RSVDGB_COL_MAJOR) return RSVDGB_ERR_INVALID_ARG;
    if (!aligned(A, dtype == RSVDGB_F32 ? 4 : 2)) return RSVDGB_ERR_INVALID_ARG;
    const int64_t inner = layout == RSVDGB_ROW_MAJOR ? n : m;
    if (lda < inner) return RSVDGB_ERR_INVALID_ARG;
    const int64_t mn = std::min(m, n);
    if (k < 1 || k >= mn || p < 0) return RSVDGB_ERR_INVALID_ARG;
    g.A = A;
    g.lda = lda;
    g.a_bf16 = dtype == RSVDGB_BF16;
    g.m = std::max(m, n);
    g.n = mn;
    g.swap_uv = m < n;
    // stored S is A (row-major) or A^T (column-major); the logical matrix is
    // A when m >= n and A^T otherwise.
    const bool logical_is_A = m >= n;
    const bool S_is_A = layout == RSVDGB_ROW_MAJOR;
    g.trans = (logical_is_A != S_is_A);
    g.l = (int)std::min<int64_t>((int64_t)k + p, mn);
    g.ldm = round_up(g.m, 32);
    g.ldn = round_up(g.n, 32);
    g.L = (int)round_up(g.l, 16);
    if (g.l > kMaxL) return RSVDGB_ERR_UNSUPPORTED;
    if (engine < RSVDGB_ENGINE_AUTO || engine > RSVDGB_ENGINE_TC_TF32) return RSVDGB_ERR_INVALID_ARG;
    const bool tc_ok = tc_pass_supported(g.sm(), g.sn(), g.lda, g.L, A, g.a_bf16);
    if ((engine == RSVDGB_ENGINE_TC || engine == RSVDGB_ENGINE_TC_TF32) && !tc_ok) return RSVDGB_ERR_UNSUPPORTED;
    g.use_tc = (engine != RSVDGB_ENGINE_SIMT) && tc_ok;
    g.h16 = g.use_tc && engine != RSVDGB_ENGINE_TC_TF32;
    if (prec != RSVDGB_PREC_FP32 && prec != RSVDGB_PREC_BF16_SKETCH && prec != RSVDGB_PREC_FP8_SKETCH)
        return RSVDGB_ERR_INVALID_ARG;
    g.bf16 = (prec == RSVDGB_PREC_BF16_SKETCH);
    g.fp8 = (prec == RSVDGB_PREC_FP8_SKETCH);
    // mixed precision runs on the tensor cores
    if ((g.bf16 || g.fp8) && !g.use_tc) return RSVDGB_ERR_UNSUPPORTED;
    return RSVDGB_OK;
}

// The power-iteration scheme of the options (RSVDGB_POWER_*): the LU form
// runs on the tensor-core engine with l <= 112.
int apply_power(Geom& g, int power)
{
    if (power != RSVDGB_POWER_SUBSPACE && power != RSVDGB_POWER_LU) return RSVDGB_ERR_INVALID_ARG;
    if (power == RSVDGB_POWER_LU) {
        if (!g.use_tc || !tslu_supported(g.l) || !xt_supported(g.L)) return RSVDGB_ERR_UNSUPPORTED;
        g.lu = true;
    }
    return RSVDGB_OK;
}

const char* kStatusNames[] = {"RSVDGB_OK",           "RSVDGB_ERR_INVALID_ARG", "RSVDGB_ERR_NOMEM",
                              "RSVDGB_ERR_CUDA",     "RSVDGB_ERR_BREAKDOWN",   "RSVDGB_ERR_NONFINITE",
                              "RSVDGB_ERR_TIMEOUT",  "RSVDGB_ERR_UNSUPPORTED"};

}  // namespace

extern "C" {

void rsvdgb_default_opts(rsvdgb_opts* o)
{
    if (!o) return;
    std::memset(o, 0, sizeof(*o));
    o->p = 10;
    o->q = 2;
    o->sdist = RSVDGB_SDIST_NORMAL;
    o->prec = RSVDGB_PREC_FP32;
    o->seed = 0;
    o->layout = RSVDGB_ROW_MAJOR;
    o->engine = RSVDGB_ENGINE_AUTO;
    o->q_mode = RSVDGB_Q_FIXED;
    o->p_max = 10;
    o->q_max = 6;
}

void rsvdgb_default_train_opts(rsvdgb_train_opts* o)
{
    if (!o) return;
    std::memset(o, 0, sizeof(*o));
    o->epochs = 300;
    o->batch = 256;
    o->lr = 2e-3f;
    o->tau = 0.99f;
    o->seed = 0;
}

const char* rsvdgb_status_string(int status)
{
    if (status < 0 || status > RSVDGB_ERR_UNSUPPORTED) return "RSVDGB_UNKNOWN_STATUS";
    return kStatusNames[status];
}

int rsvdgb_sketch_width(int64_t m, int64_t n, int k, int p)
{
    const int64_t mn = std::min(m, n);
    return (int)std::min<int64_t>((int64_t)k + p, mn);
}

int rsvdgb_create(rsvdgb_handle** h, int device, void* cuda_stream)
{
    if (!h) return RSVDGB_ERR_INVALID_ARG;
    *h = nullptr;
    int count = 0;
    if (cudaGetDeviceCount(&count) != cudaSuccess) {
        cudaGetLastError();
        return RSVDGB_ERR_CUDA;
    }
    if (device < 0 || device >= count) return RSVDGB_ERR_INVALID_ARG;
    RSVDGB_CUDA_TRY(cudaSetDevice(device));
    rsvdgb_handle* hh = new (std::nothrow) rsvdgb_handle();
    if (!hh) return RSVDGB_ERR_NOMEM;
    hh->device = device;
    hh->stream = (cudaStream_t)cuda_stream;
    cudaDeviceGetAttribute(&hh->sm_count, cudaDevAttrMultiProcessorCount, device);
    if (init_small_kernels() != RSVDGB_OK) {
        delete hh;
        return RSVDGB_ERR_CUDA;
    }
    *h = hh;
    return RSVDGB_OK;
}

int rsvdgb_destroy(rsvdgb_handle* h)
{
    if (!h) return RSVDGB_ERR_INVALID_ARG;
    cudaSetDevice(h->device);
    cudaStreamSynchronize(h->stream);
    if (h->ws) cudaFree(h->ws);
    if (h->host_stage) cudaFree(h->host_stage);
    if (h->aux) cudaFree(h->aux);
    for (cudaEvent_t e : h->prof.ev) cudaEventDestroy(e);
    destroy_plan(h->batched);
    if (h->ctl_params) cudaFree(h->ctl_params);
    if (h->ctl_scratch) cudaFree(h->ctl_scratch);
    if (h->ctl_host) cudaFreeHost(h->ctl_host);
    delete h;
    return RSVDGB_OK;
}

int rsvdgb_set_stream(rsvdgb_handle* h, void* cuda_stream)
{
    if (!h) return RSVDGB_ERR_INVALID_ARG;
    h->stream = (cudaStream_t)cuda_stream;
    return RSVDGB_OK;
}

int rsvdgb_rsvd(rsvdgb_handle* h, const void* A, int64_t m, int64_t n, int64_t lda, int dtype, int k, int nu, int nv,
                const rsvdgb_opts* opts, float* d, float* U, int64_t ldu, float* V, int64_t ldv, rsvdgb_info* info)
{
    int rc = check_handle(h);
    if (rc) return rc;
    rsvdgb_opts o;
    if (opts)
        o = *opts;
    else
        rsvdgb_default_opts(&o);
    if (o.q < 0 || o.sdist < 0 || o.sdist > 2) return RSVDGB_ERR_INVALID_ARG;
    if (o.q_mode != RSVDGB_Q_FIXED && o.q_mode != RSVDGB_Q_LEARNED) return RSVDGB_ERR_INVALID_ARG;
    if (o.q_mode == RSVDGB_Q_LEARNED && (o.p_max < 2 || o.q_max < 0)) return RSVDGB_ERR_INVALID_ARG;
    // learned mode with a loaded controller: sketch at the widest width first
    const bool learned = o.q_mode == RSVDGB_Q_LEARNED && h->ctl_params != nullptr;
    Geom g{};
    rc = make_geom(A, m, n, lda, dtype, o.layout, k, learned ? o.p_max : o.p, o.engine, o.prec, g);
    if (rc) return rc;
    rc = apply_power(g, o.power);
    if (rc) return rc;
    if (nu < 0) nu = k;
    if (nv < 0) nv = k;
    if (nu > k || nv > k || !d) return RSVDGB_ERR_INVALID_ARG;
    if (nu > 0 && (!U || ldu < nu)) return RSVDGB_ERR_INVALID_ARG;
    if (nv > 0 && (!V || ldv < nv)) return RSVDGB_ERR_INVALID_ARG;
    Outputs out{};
    out.d = d;
    out.info = info;
    out.check_orth = o.check_orth != 0;
    if (!g.swap_uv) {
        out.U = U; out.ldU = ldu; out.nU = nu;
        out.V = V; out.ldV = ldv; out.nV = nv;
    } else {
        out.U = V; out.ldU = ldv; out.nU = nv;
        out.V = U; out.ldV = ldu; out.nV = nu;
    }
    if (learned) {
        const Learned lc{k, o.p_max, o.q_max, nullptr};
        return run_fp32(h, g, k, o.q, o.sdist, o.seed, out, &lc);
    }
    return run_fp32(h, g, k, o.q, o.sdist, o.seed, out);
}

int rsvdgb_rqb(rsvdgb_handle* h, const void* A, int64_t m, int64_t n, int64_t lda, int dtype, int k,
               const rsvdgb_opts* opts, float* Q, int64_t ldq, float* B, int64_t ldb, rsvdgb_info* info)
{
    int rc = check_handle(h);
    if (rc) return rc;
    rsvdgb_opts o;
    if (opts)
        o = *opts;
    else
        rsvdgb_default_opts(&o);
    if (o.q < 0 || o.sdist < 0 || o.sdist > 2) return RSVDGB_ERR_INVALID_ARG;
    if (m < n || o.layout != RSVDGB_ROW_MAJOR) return RSVDGB_ERR_INVALID_ARG;
    Geom g{};
    rc = make_geom(A, m, n, lda, dtype, o.layout, k, o.p, o.engine, o.prec, g);
    if (rc) return rc;
    rc = apply_power(g, o.power);
    if (rc) return rc;
    if (!Q || !B || ldq < g.l || ldb < n) return RSVDGB_ERR_INVALID_ARG;
    Outputs out{};
    out.Qrow = Q;
    out.ldq = ldq;
    out.Brow = B;
    out.ldb = ldb;
    out.info = info;
    out.check_orth = o.check_orth != 0;
    return run_fp32(h, g, k, o.q, o.sdist, o.seed, out);
}

}  // extern "C"

namespace {
// A handle-owned device buffer that grows on demand.
int ensure_buffer(rsvdgb_handle* h, void** buf, size_t* have, size_t bytes)
{
    if (bytes <= *have) return RSVDGB_OK;
    if (*buf) {
        cudaStreamSynchronize(h->stream);
        cudaFree(*buf);
        *buf = nullptr;
        *have = 0;
    }
    if (cudaMalloc(buf, bytes) != cudaSuccess) {
        cudaGetLastError();
        return RSVDGB_ERR_NOMEM;
    }
    *have = bytes;
    return RSVDGB_OK;
}

// Device staging buffer of the *_host entry points.
int ensure_host_stage(rsvdgb_handle* h, size_t bytes) { return ensure_buffer(h, &h->host_stage, &h->host_stage_bytes, bytes); }
}  // namespace

extern "C" {

int rsvdgb_rsvd_host(rsvdgb_handle* h, const void* A, int64_t m, int64_t n, int64_t lda, int dtype, int k, int nu,
                     int nv, const rsvdgb_opts* opts, float* d, float* U, int64_t ldu, float* V, int64_t ldv,
                     rsvdgb_info* info)
{
    int rc = check_handle(h);
    if (rc) return rc;
    if (!A || !d || m < 1 || n < 1) return RSVDGB_ERR_INVALID_ARG;
    rsvdgb_opts o;
    if (opts)
        o = *opts;
    else
        rsvdgb_default_opts(&o);
    if (nu < 0) nu = k;
    if (nv < 0) nv = k;
    if (nu > k || nv > k || k < 1) return RSVDGB_ERR_INVALID_ARG;
    const size_t esz = dtype == RSVDGB_BF16 ? 2 : 4;
    const int64_t rows_s = o.layout == RSVDGB_ROW_MAJOR ? m : n;
    const int64_t cols_s = o.layout == RSVDGB_ROW_MAJOR ? n : m;
    if (lda < cols_s) return RSVDGB_ERR_INVALID_ARG;
    // device staging: A (packed), d, U, V, info
    size_t off = 0;
    auto take = [&](size_t bytes) {
        off = (size_t)round_up((int64_t)off, 256);
        size_t at = off;
        off += bytes;
        return at;
    };
    const size_t oA = take((size_t)rows_s * cols_s * esz);
    const size_t od = take((size_t)k * sizeof(float));
    const size_t oU = take((size_t)m * std::max(nu, 1) * sizeof(float));
    const size_t oV = take((size_t)n * std::max(nv, 1) * sizeof(float));
    const size_t oI = take(sizeof(rsvdgb_info));
    rc = ensure_host_stage(h, off);
    if (rc) return rc;
    char* base = (char*)h->host_stage;
    // contiguous rows: one linear copy (the pitched form ran at about two
    // thirds of the linear copy's rate on the host-to-device link)
    if (lda == cols_s)
        RSVDGB_CUDA_TRY(cudaMemcpyAsync(base + oA, A, (size_t)rows_s * cols_s * esz, cudaMemcpyHostToDevice,
                                        h->stream));
    else
        RSVDGB_CUDA_TRY(cudaMemcpy2DAsync(base + oA, cols_s * esz, A, lda * esz, cols_s * esz, rows_s,
                                          cudaMemcpyHostToDevice, h->stream));
    rc = rsvdgb_rsvd(h, base + oA, m, n, cols_s, dtype, k, nu, nv, &o, (float*)(base + od),
                     nu > 0 ? (float*)(base + oU) : nullptr, std::max(nu, 1), nv > 0 ? (float*)(base + oV) : nullptr,
                     std::max(nv, 1), (rsvdgb_info*)(base + oI));
    if (rc) return rc;
    RSVDGB_CUDA_TRY(cudaMemcpyAsync(d, base + od, (size_t)k * sizeof(float), cudaMemcpyDeviceToHost, h->stream));
    if (nu > 0 && U)
        RSVDGB_CUDA_TRY(cudaMemcpy2DAsync(U, ldu * sizeof(float), base + oU, nu * sizeof(float), nu * sizeof(float), m,
                                          cudaMemcpyDeviceToHost, h->stream));
    if (nv > 0 && V)
        RSVDGB_CUDA_TRY(cudaMemcpy2DAsync(V, ldv * sizeof(float), base + oV, nv * sizeof(float), nv * sizeof(float), n,
                                          cudaMemcpyDeviceToHost, h->stream));
    rsvdgb_info hinfo;
    RSVDGB_CUDA_TRY(cudaMemcpyAsync(&hinfo, base + oI, sizeof(hinfo), cudaMemcpyDeviceToHost, h->stream));
    RSVDGB_CUDA_TRY(cudaStreamSynchronize(h->stream));
    if (info) *info = hinfo;
    return hinfo.status;
}

int rsvdgb_rpca(rsvdgb_handle* h, const void* A, int64_t m, int64_t n, int64_t lda, int dtype, int k, int center,
                int scale, const rsvdgb_opts* opts, float* rotation, int64_t ldr, float* eigvals, float* sdev,
                float* x, int64_t ldx, float* center_out, float* scale_out, rsvdgb_info* info)
{
    int rc = check_handle(h);
    if (rc) return rc;
    rsvdgb_opts o;
    if (opts)
        o = *opts;
    else
        rsvdgb_default_opts(&o);
    if (o.q < 0 || o.sdist < 0 || o.sdist > 2) return RSVDGB_ERR_INVALID_ARG;
    if (o.q_mode != RSVDGB_Q_FIXED && o.q_mode != RSVDGB_Q_LEARNED) return RSVDGB_ERR_INVALID_ARG;
    if (o.q_mode == RSVDGB_Q_LEARNED && (o.p_max < 2 || o.q_max < 0)) return RSVDGB_ERR_INVALID_ARG;
    const bool learned = o.q_mode == RSVDGB_Q_LEARNED && h->ctl_params != nullptr;
    Geom g{};
    rc = make_geom(A, m, n, lda, dtype, o.layout, k, learned ? o.p_max : o.p, o.engine, o.prec, g);
    if (rc) return rc;
    if (!eigvals) return RSVDGB_ERR_INVALID_ARG;
    if (rotation && ldr < k) return RSVDGB_ERR_INVALID_ARG;
    if (x && ldx < k) return RSVDGB_ERR_INVALID_ARG;
    g.pca_nvar = n;
    const int nx = x ? k : 0, nr = rotation ? k : 0;
    Outputs out{};
    out.d = eigvals;
    out.info = info;
    if (!g.swap_uv) {
        out.U = x; out.ldU = ldx; out.nU = nx;
        out.V = rotation; out.ldV = ldr; out.nV = nr;
        out.sigma_cols = x ? 1 : 0;
    } else {
        out.U = rotation; out.ldU = ldr; out.nU = nr;
        out.V = x; out.ldV = ldx; out.nV = nx;
        out.sigma_cols = x ? 2 : 0;
    }
    PcaSpec pc{center ? 1 : 0, scale ? 1 : 0, center_out, scale_out, eigvals, sdev, m};
    if (learned) {
        const Learned lc{k, o.p_max, o.q_max, nullptr};
        return run_fp32(h, g, k, o.q, o.sdist, o.seed, out, &lc, &pc);
    }
    return run_fp32(h, g, k, o.q, o.sdist, o.seed, out, nullptr, &pc);
}

int rsvdgb_rpca_host(rsvdgb_handle* h, const void* A, int64_t m, int64_t n, int64_t lda, int dtype, int k,
                     int center, int scale, const rsvdgb_opts* opts, float* rotation, int64_t ldr, float* eigvals,
                     float* sdev, float* x, int64_t ldx, float* center_out, float* scale_out, rsvdgb_info* info)
{
    int rc = check_handle(h);
    if (rc) return rc;
    if (!A || !eigvals || m < 1 || n < 1 || k < 1) return RSVDGB_ERR_INVALID_ARG;
    if ((rotation && ldr < k) || (x && ldx < k)) return RSVDGB_ERR_INVALID_ARG;
    rsvdgb_opts o;
    if (opts)
        o = *opts;
    else
        rsvdgb_default_opts(&o);
    const size_t esz = dtype == RSVDGB_BF16 ? 2 : 4;
    const int64_t rows_s = o.layout == RSVDGB_ROW_MAJOR ? m : n;
    const int64_t cols_s = o.layout == RSVDGB_ROW_MAJOR ? n : m;
    if (lda < cols_s) return RSVDGB_ERR_INVALID_ARG;
    size_t off = 0;
    auto take = [&](size_t bytes) {
        off = (size_t)round_up((int64_t)off, 256);
        size_t at = off;
        off += bytes;
        return at;
    };
    const size_t oA = take((size_t)rows_s * cols_s * esz);
    const size_t oE = take((size_t)k * sizeof(float));
    const size_t oS = take((size_t)k * sizeof(float));
    const size_t oR = take((size_t)n * k * sizeof(float));
    const size_t oX = take((size_t)m * k * sizeof(float));
    const size_t oC = take((size_t)n * sizeof(float));
    const size_t oSc = take((size_t)n * sizeof(float));
    const size_t oI = take(sizeof(rsvdgb_info));
    rc = ensure_host_stage(h, off);
    if (rc) return rc;
    char* base = (char*)h->host_stage;
    auto dev = [&](size_t o_) { return (float*)(base + o_); };
    if (lda == cols_s)
        RSVDGB_CUDA_TRY(cudaMemcpyAsync(base + oA, A, (size_t)rows_s * cols_s * esz, cudaMemcpyHostToDevice,
                                        h->stream));
    else
        RSVDGB_CUDA_TRY(cudaMemcpy2DAsync(base + oA, cols_s * esz, A, lda * esz, cols_s * esz, rows_s,
                                          cudaMemcpyHostToDevice, h->stream));
    rc = rsvdgb_rpca(h, base + oA, m, n, cols_s, dtype, k, center, scale, &o, rotation ? dev(oR) : nullptr, k,
                     dev(oE), sdev ? dev(oS) : nullptr, x ? dev(oX) : nullptr, k,
                     center_out ? dev(oC) : nullptr, scale_out ? dev(oSc) : nullptr, (rsvdgb_info*)(base + oI));
    if (rc) return rc;
    const cudaStream_t s = h->stream;
    RSVDGB_CUDA_TRY(cudaMemcpyAsync(eigvals, dev(oE), (size_t)k * sizeof(float), cudaMemcpyDeviceToHost, s));
    if (sdev) RSVDGB_CUDA_TRY(cudaMemcpyAsync(sdev, dev(oS), (size_t)k * sizeof(float), cudaMemcpyDeviceToHost, s));
    if (rotation)
        RSVDGB_CUDA_TRY(cudaMemcpy2DAsync(rotation, ldr * sizeof(float), dev(oR), k * sizeof(float),
                                          k * sizeof(float), n, cudaMemcpyDeviceToHost, s));
    if (x)
        RSVDGB_CUDA_TRY(cudaMemcpy2DAsync(x, ldx * sizeof(float), dev(oX), k * sizeof(float), k * sizeof(float), m,
                                          cudaMemcpyDeviceToHost, s));
    if (center_out)
        RSVDGB_CUDA_TRY(cudaMemcpyAsync(center_out, dev(oC), (size_t)n * sizeof(float), cudaMemcpyDeviceToHost, s));
    if (scale_out)
        RSVDGB_CUDA_TRY(cudaMemcpyAsync(scale_out, dev(oSc), (size_t)n * sizeof(float), cudaMemcpyDeviceToHost, s));
    rsvdgb_info hinfo;
    RSVDGB_CUDA_TRY(cudaMemcpyAsync(&hinfo, base + oI, sizeof(hinfo), cudaMemcpyDeviceToHost, s));
    RSVDGB_CUDA_TRY(cudaStreamSynchronize(s));
    if (info) *info = hinfo;
    return hinfo.status;
}

static int rid_common(rsvdgb_handle* h, const void* A, int64_t m, int64_t n, int64_t lda, int dtype, int k,
                      const rsvdgb_opts* opts, const RidSpec& r, rsvdgb_info* info)
{
    int rc = check_handle(h);
    if (rc) return rc;
    rsvdgb_opts o;
    if (opts)
        o = *opts;
    else
        rsvdgb_default_opts(&o);
    if (o.q < 0 || o.sdist < 0 || o.sdist > 2) return RSVDGB_ERR_INVALID_ARG;
    if (m < n) return RSVDGB_ERR_UNSUPPORTED;  // the row ID is the column ID of A^T
    Geom g{};
    rc = make_geom(A, m, n, lda, dtype, o.layout, k, o.p, o.engine, o.prec, g);
    if (rc) return rc;
    if (k > 256 || !r.J || (r.cur && !r.I)) return RSVDGB_ERR_INVALID_ARG;
    if ((r.C && r.ldc < k) || (r.Z && r.ldz < n) || (r.U && r.ldu < k) || (r.R && r.ldr < n))
        return RSVDGB_ERR_INVALID_ARG;
    g.rid_k = k;
    g.rid_cur = r.cur;
    Outputs out{};
    out.info = info;
    out.check_orth = o.check_orth != 0;
    out.rid = &r;
    return run_fp32(h, g, k, o.q, o.sdist, o.seed, out);
}

int rsvdgb_rid(rsvdgb_handle* h, const void* A, int64_t m, int64_t n, int64_t lda, int dtype, int k,
               const rsvdgb_opts* opts, float* C, int64_t ldc, float* Z, int64_t ldz, int64_t* J, rsvdgb_info* info)
{
    const RidSpec r{false, C, ldc, Z, ldz, J, nullptr, 0, nullptr, 0, nullptr};
    return rid_common(h, A, m, n, lda, dtype, k, opts, r, info);
}

int rsvdgb_rcur(rsvdgb_handle* h, const void* A, int64_t m, int64_t n, int64_t lda, int dtype, int k,
                const rsvdgb_opts* opts, float* C, int64_t ldc, float* U, int64_t ldu, float* R, int64_t ldr,
                int64_t* J, int64_t* I, rsvdgb_info* info)
{
    const RidSpec r{true, C, ldc, nullptr, 0, J, U, ldu, R, ldr, I};
    return rid_common(h, A, m, n, lda, dtype, k, opts, r, info);
}

void rsvdgb_default_rrpca_opts(rsvdgb_rrpca_opts* o)
{
    if (!o) return;
    *o = rsvdgb_rrpca_opts{};
    o->lambda = 0.f;
    o->tol = 1e-5f;
    o->rho = 1.5f;
    o->maxiter = 50;
    o->k0 = 2;
}

int rsvdgb_rrpca(rsvdgb_handle* h, const float* A, int64_t m, int64_t n, int64_t lda, const rsvdgb_rrpca_opts* ro_in,
                 const rsvdgb_opts* opts, float* L, int64_t ldl, float* S, int64_t lds, rsvdgb_rrpca_result* res)
{
    int rc = check_handle(h);
    if (rc) return rc;
    rsvdgb_opts o;
    if (opts)
        o = *opts;
    else
        rsvdgb_default_opts(&o);
    rsvdgb_rrpca_opts ro;
    if (ro_in)
        ro = *ro_in;
    else
        rsvdgb_default_rrpca_opts(&ro);
    if (!A || !S || m < 2 || n < 2 || lda < n || lds < n || (L && ldl < n)) return RSVDGB_ERR_INVALID_ARG;
    if (ro.maxiter < 1 || !(ro.tol > 0.f) || !(ro.rho >= 1.f) || ro.k0 < 1 || o.p < 0 || o.q < 0)
        return RSVDGB_ERR_INVALID_ARG;
    if (o.layout != RSVDGB_ROW_MAJOR || o.q_mode != RSVDGB_Q_FIXED) return RSVDGB_ERR_UNSUPPORTED;
    if (!aligned(A, 4) || !aligned(S, 4)) return RSVDGB_ERR_INVALID_ARG;
    const int64_t ns = std::min(m, n);
    const int kmax = (int)std::min<int64_t>(ns - 1, kMaxL - o.p);
    if (kmax < 1) return RSVDGB_ERR_UNSUPPORTED;
    const cudaStream_t s = h->stream;
    const int nb_abs = 4 * h->sm_count;
    const int64_t nb = std::max<int64_t>(ialm_blocks(m, n), nb_abs);
    // aux: Z, X (m x n), U (m x kmax), V (n x kmax), d, sig, partial sums, scalars, rSVD info
    size_t off = 0;
    auto take = [&](size_t bytes) {
        off = (size_t)round_up((int64_t)off, 256);
        size_t at = off;
        off += bytes;
        return at;
    };
    const size_t oZ = take((size_t)m * n * 4), oX = take((size_t)m * n * 4), oU = take((size_t)m * kmax * 4),
                 oV = take((size_t)n * kmax * 4), oD = take((size_t)kmax * 4 + 64), oSig = take((size_t)kmax * 4),
                 oPart = take((size_t)nb * 8), oE = take(8), oSq = take(8), oMax = take(4),
                 oInfo = take(sizeof(rsvdgb_info));
    rc = ensure_buffer(h, &h->aux, &h->aux_bytes, off);
    if (rc) return rc;
    char* base = (char*)h->aux;
    float *Z = (float*)(base + oZ), *X = (float*)(base + oX), *U = (float*)(base + oU), *V = (float*)(base + oV),
          *d = (float*)(base + oD), *sig = (float*)(base + oSig);
    double *part = (double*)(base + oPart), *err2 = (double*)(base + oE), *sumsq = (double*)(base + oSq);
    unsigned int* amax = (unsigned int*)(base + oMax);
    rsvdgb_info* dinfo = (rsvdgb_info*)(base + oInfo);

    // max |a_ij| and ||A||_F first: A = 0 or a non-finite A stops here,
    // before any rSVD runs on it; then ||A||_2 from a rank-1 rSVD
    RSVDGB_CUDA_TRY(cudaMemsetAsync(amax, 0, 4, s));
    launch_absmax_sumsq(s, A, lda, m, n, amax, part, nb_abs, sumsq);
    unsigned int h_amax = 0;
    double h_sumsq = 0.0;
    RSVDGB_CUDA_TRY(cudaMemcpyAsync(&h_amax, amax, 4, cudaMemcpyDeviceToHost, s));
    RSVDGB_CUDA_TRY(cudaMemcpyAsync(&h_sumsq, sumsq, 8, cudaMemcpyDeviceToHost, s));
    RSVDGB_CUDA_TRY(cudaStreamSynchronize(s));
    const double normA = std::sqrt(h_sumsq);
    if (!std::isfinite(normA)) return RSVDGB_ERR_NONFINITE;
    if (!(normA > 0.0)) return RSVDGB_ERR_INVALID_ARG;  // A = 0
    float maxabs;
    std::memcpy(&maxabs, &h_amax, 4);
    rc = rsvdgb_rsvd(h, A, m, n, lda, RSVDGB_F32, 1, 1, 1, &o, d, U, kmax, V, kmax, dinfo);
    if (rc) return rc;
    float h_norm2 = 0.f;
    RSVDGB_CUDA_TRY(cudaMemcpyAsync(&h_norm2, d, 4, cudaMemcpyDeviceToHost, s));
    RSVDGB_CUDA_TRY(cudaStreamSynchronize(s));
    const double norm2 = (double)h_norm2;
    if (!(norm2 > 0.0)) return RSVDGB_ERR_BREAKDOWN;
    const double lam = ro.lambda > 0.f ? (double)ro.lambda : 1.0 / std::sqrt((double)std::max(m, n));
    double mu = 1.25 / norm2;
    const double mu_bar = 1e7 * mu;
    const double dual = std::max(norm2, (double)maxabs / lam);
    launch_ialm_init(s, A, lda, m, n, (float)(1.0 / dual), (float)(1.0 / mu), S, lds, Z, X);

    int k = std::min(ro.k0, kmax), svp = 0, it = 0, status = RSVDGB_OK;
    double err = 0.0;
    std::vector<float> hd(kmax), hsig(kmax);
    for (it = 1; it <= ro.maxiter; ++it) {
        rsvdgb_opts oi = o;
        oi.seed = o.seed + (uint64_t)it;
        rc = rsvdgb_rsvd(h, X, m, n, n, RSVDGB_F32, k, k, k, &oi, d, U, kmax, V, kmax, dinfo);
        if (rc) return rc;
        rsvdgb_info hinfo;
        RSVDGB_CUDA_TRY(cudaMemcpyAsync(hd.data(), d, sizeof(float) * k, cudaMemcpyDeviceToHost, s));
        RSVDGB_CUDA_TRY(cudaMemcpyAsync(&hinfo, dinfo, sizeof(hinfo), cudaMemcpyDeviceToHost, s));
        RSVDGB_CUDA_TRY(cudaStreamSynchronize(s));
        if (hinfo.status != RSVDGB_OK) {
            status = hinfo.status;
            break;
        }
        // predicted rank: singular values above 1/mu are kept, shrunk by 1/mu
        const double inv_mu = 1.0 / mu;
        svp = 0;
        for (int t = 0; t < k; ++t) svp += (double)hd[t] > inv_mu;
        int knext = svp < k ? svp + 1 : svp + (int)std::lround(0.05 * (double)ns);
        knext = std::max(1, std::min(knext, kmax));
        for (int t = 0; t < svp; ++t) hsig[t] = (float)std::max((double)hd[t] - inv_mu, 0.0);
        if (svp > 0) RSVDGB_CUDA_TRY(cudaMemcpyAsync(sig, hsig.data(), sizeof(float) * svp, cudaMemcpyHostToDevice, s));
        const double mu_next = std::min(ro.rho * mu, mu_bar);
        launch_ialm_step(s, A, lda, m, n, U, kmax, V, kmax, sig, svp, (float)mu, (float)inv_mu, (float)(1.0 / mu_next),
                         (float)(lam * inv_mu), S, lds, Z, X, part, err2, 0, nullptr, 0);
        double he2 = 0.0;
        RSVDGB_CUDA_TRY(cudaMemcpyAsync(&he2, err2, 8, cudaMemcpyDeviceToHost, s));
        RSVDGB_CUDA_TRY(cudaStreamSynchronize(s));
        err = std::sqrt(he2) / normA;
        mu = mu_next;
        k = knext;
        if (err < (double)ro.tol) break;
    }
    if (it > ro.maxiter) it = ro.maxiter;
    if (L && status == RSVDGB_OK)
        launch_ialm_step(s, A, lda, m, n, U, kmax, V, kmax, sig, svp, 0.f, 0.f, 0.f, 0.f, nullptr, 0, nullptr, nullptr,
                         nullptr, nullptr, 1, L, ldl);
    RSVDGB_CUDA_TRY(cudaGetLastError());
    RSVDGB_CUDA_TRY(cudaStreamSynchronize(s));
    if (res) {
        *res = rsvdgb_rrpca_result{};
        res->iters = it;
        res->rank = svp;
        res->k_next = k;
        res->status = status;
        res->err = err;
        res->mu = mu;
    }
    return status;
}

int rsvdgb_omega(rsvdgb_handle* h, int64_t rows, int l, uint64_t seed, int sdist, float* out, int64_t ld)
{
    int rc = check_handle(h);
    if (rc) return rc;
    if (rows < 1 || l < 1 || !out || ld < l || sdist < 0 || sdist > 2 || !aligned(out, 4))
        return RSVDGB_ERR_INVALID_ARG;
    launch_omega_rowmajor(h->stream, rows, l, seed, sdist, out, ld);
    RSVDGB_CUDA_TRY(cudaGetLastError());
    return RSVDGB_OK;
}

static int pass_common(rsvdgb_handle* h, const void* A, int64_t m, int64_t n, int64_t lda, int dtype, const float* X,
                       int64_t ldx, int l, float* Y, int64_t ldy, int engine, int prec, bool transpose)
{
    int rc = check_handle(h);
    if (rc) return rc;
    if (!A || !X || !Y || m < 1 || n < 1 || l < 1 || lda < n) return RSVDGB_ERR_INVALID_ARG;
    if (dtype != RSVDGB_F32 && dtype != RSVDGB_BF16) return RSVDGB_ERR_INVALID_ARG;
    if (ldx < l || ldy < l) return RSVDGB_ERR_INVALID_ARG;
    if (engine < RSVDGB_ENGINE_AUTO || engine > RSVDGB_ENGINE_TC_TF32) return RSVDGB_ERR_INVALID_ARG;
    if (prec != RSVDGB_PREC_FP32 && prec != RSVDGB_PREC_BF16_SKETCH && prec != RSVDGB_PREC_FP8_SKETCH)
        return RSVDGB_ERR_INVALID_ARG;
    const bool f8 = prec == RSVDGB_PREC_FP8_SKETCH;
    const bool bf = prec == RSVDGB_PREC_BF16_SKETCH || f8;
    const bool want_tc = engine == RSVDGB_ENGINE_TC || engine == RSVDGB_ENGINE_TC_TF32;
    const int64_t M = transpose ? n : m, K = transpose ? m : n;
    const int L = (int)round_up(l, 16);
    const bool tc_ok = l <= 256 && tc_pass_supported(m, n, lda, L, A, dtype == RSVDGB_BF16);
    if ((want_tc || bf) && !tc_ok) return RSVDGB_ERR_UNSUPPORTED;
    if (bf && engine == RSVDGB_ENGINE_SIMT) return RSVDGB_ERR_UNSUPPORTED;
    if (engine == RSVDGB_ENGINE_SIMT || !tc_ok) {
        const int64_t tiles = ceil_div(M, 64) * ceil_div(l, 64);
        const int splits = splits_for(tiles, K, h->sm_count);
        rc = ensure_workspace(h, (size_t)splits * M * ldy * sizeof(float) + 1024);
        if (rc) return rc;
        tall_gemm(h->stream, h->sm_count, transpose, false, false, A, lda, dtype == RSVDGB_BF16, X, ldx, Y, ldy, M, l,
                  K, (float*)h->ws, nullptr);
        RSVDGB_CUDA_TRY(cudaGetLastError());
        return RSVDGB_OK;
    }
    // tensor-core engine: stage X column-major and TF32-split, run, copy back
    const int64_t ldK = round_up(K, 32), ldM = round_up(M, 32);
    const int64_t splits = transpose ? tc_pass_max_splits(m, n, L, h->sm_count) : 1;
    Carve probe(nullptr);
    probe.take<float>(L * ldK);
    probe.take<float>(L * ldK);
    probe.take<float>(L * ldK);
    probe.take<float>(L * ldM);
    const int64_t ld8 = round_up(n, 16), ldt8 = round_up(m, 16), ldp8 = round_up(K, 16);
    const int64_t splits8 = f8 ? f8_pass_max_splits(transpose ? n : m, K, L, h->sm_count) : 0;
    probe.take<float>(std::max(splits, splits8) * L * ldM);
    probe.take<int>(4);
    probe.take<float>(L);
    if (f8) {
        probe.take<uint8_t>((size_t)m * ld8);
        probe.take<uint8_t>((size_t)n * ldt8);
        probe.take<uint8_t>((size_t)L * ldp8);
        probe.take<float>(m);
        probe.take<float>(L);
        probe.take<unsigned int>(L + 1);
    }
    rc = ensure_workspace(h, probe.off + 1024);
    if (rc) return rc;
    Carve c(h->ws);
    float* Xc = c.take<float>(L * ldK);
    float* Xh = c.take<float>(L * ldK);
    float* Xl = c.take<float>(L * ldK);
    float* Yc = c.take<float>(L * ldM);
    float* part = c.take<float>(std::max(splits, splits8) * L * ldM);
    int* status = c.take<int>(4);
    float* pinv = c.take<float>(L);
    uint8_t *A8 = nullptr, *At8 = nullptr, *P8 = nullptr;
    float *rs8 = nullptr, *ts8 = nullptr;
    unsigned int* cm8 = nullptr;
    if (f8) {
        A8 = c.take<uint8_t>((size_t)m * ld8);
        At8 = c.take<uint8_t>((size_t)n * ldt8);
        P8 = c.take<uint8_t>((size_t)L * ldp8);
        rs8 = c.take<float>(m);
        ts8 = c.take<float>(L);
        cm8 = c.take<unsigned int>(L + 1);
        RSVDGB_CUDA_TRY(cudaMemsetAsync(cm8, 0, (L + 1) * sizeof(unsigned int), h->stream));
    }
    unsigned int* amax = (unsigned int*)(status + 1);
    const cudaStream_t s = h->stream;
    RSVDGB_CUDA_TRY(cudaMemsetAsync(status, 0, 2 * sizeof(int), s));
    launch_rowmajor_to_colmajor(s, X, ldx, K, l, L, Xc, ldK);
    int64_t used = 0;
    if (f8) {
        // E4M3 copies of A with row powers of two, the panel quantised per column
        launch_fp8_prep(s, A, lda, dtype == RSVDGB_BF16, m, n, A8, ld8, At8, ldt8, rs8, nullptr, nullptr);
        launch_fp8_panel(s, Xc, ldK, K, l, L, transpose ? rs8 : nullptr, P8, ldp8, ts8, cm8);
        rc = launch_f8_pass(s, h->sm_count, transpose, transpose ? At8 : A8, M, K, transpose ? ldt8 : ld8, P8, ldp8,
                            L, transpose ? nullptr : rs8, ts8, Yc, ldM, part, &used, status);
    } else if (bf) {
        launch_to_bf16(s, Xc, ldK, K, l, L, Xh);
        rc = launch_tc_gemm(s, h->sm_count, transpose, (const float*)A, m, n, lda, Xh, nullptr, ldK, L, Yc, nullptr,
                            nullptr, ldM, part, transpose ? 0 : 1, &used, status, nullptr, 0, 0, 1,
                            dtype == RSVDGB_BF16);
    } else if (engine != RSVDGB_ENGINE_TC_TF32) {
        // scaled FP16x3: max|A| first (a rSVD takes it from its first pass)
        launch_absmax(s, h->sm_count, A, lda, dtype == RSVDGB_BF16, m, n, amax);
        launch_panel_f16(s, Xc, ldK, K, l, L, (uint16_t*)Xh, (uint16_t*)Xl, pinv);
        TcExtra x{};
        x.h16 = 1;
        x.amax_in = amax;
        x.pinv = pinv;
        rc = launch_tc_gemm(s, h->sm_count, transpose, (const float*)A, m, n, lda, Xh, Xl, ldK, L, Yc, nullptr,
                            nullptr, ldM, part, transpose ? 0 : 1, &used, status, nullptr, 0, 0, 0,
                            dtype == RSVDGB_BF16, kExactChunk, nullptr, nullptr, nullptr, &x);
    } else {
        launch_split_tf32(s, Xc, ldK, K, l, L, Xh, Xl);
        rc = launch_tc_gemm(s, h->sm_count, transpose, (const float*)A, m, n, lda, Xh, Xl, ldK, L, Yc, nullptr,
                            nullptr, ldM, part, transpose ? 0 : 1, &used, status, nullptr, 0, 0, 0,
                            dtype == RSVDGB_BF16, kExactChunk);
    }
    if (rc) return rc;
    if (used > 0) launch_reduce_splits(s, part, (int)used, (int64_t)L * ldM, l, M, ldM, Yc, ldM);
    launch_colmajor_to_rowmajor(s, Yc, ldM, M, l, Y, ldy);
    RSVDGB_CUDA_TRY(cudaGetLastError());
    return RSVDGB_OK;
}

int rsvdgb_pass_ax(rsvdgb_handle* h, const void* A, int64_t m, int64_t n, int64_t lda, int dtype, const float* X,
                   int64_t ldx, int l, float* Y, int64_t ldy, int engine, int prec)
{
    return pass_common(h, A, m, n, lda, dtype, X, ldx, l, Y, ldy, engine, prec, false);
}

int rsvdgb_pass_atx(rsvdgb_handle* h, const void* A, int64_t m, int64_t n, int64_t lda, int dtype, const float* X,
                    int64_t ldx, int l, float* Z, int64_t ldz, int engine, int prec)
{
    return pass_common(h, A, m, n, lda, dtype, X, ldx, l, Z, ldz, engine, prec, true);
}

int rsvdgb_rsvd_batched(rsvdgb_handle* h, int batch, const rsvdgb_matrix_desc* descs, int k, const rsvdgb_opts* opts,
                        const rsvdgb_result_desc* outs, rsvdgb_info* infos)
{
    int rc = check_handle(h);
    if (rc) return rc;
    if (batch < 1 || !descs || !outs || k < 1) return RSVDGB_ERR_INVALID_ARG;
    rsvdgb_opts o;
    if (opts)
        o = *opts;
    else
        rsvdgb_default_opts(&o);
    if (o.p < 0 || o.q < 0 || o.q > 8 || o.sdist < 0 || o.sdist > 2) return RSVDGB_ERR_INVALID_ARG;
    if (o.layout != RSVDGB_ROW_MAJOR) return RSVDGB_ERR_UNSUPPORTED;
    for (int b = 0; b < batch; ++b) {
        const rsvdgb_matrix_desc& d = descs[b];
        const rsvdgb_result_desc& r = outs[b];
        if (!d.A || d.m < 1 || d.n < 1 || d.lda < d.n || !aligned(d.A, 4)) return RSVDGB_ERR_INVALID_ARG;
        if (d.dtype != RSVDGB_F32) return RSVDGB_ERR_UNSUPPORTED;
        if (k >= std::min(d.m, d.n)) return RSVDGB_ERR_INVALID_ARG;
        if (std::min<int64_t>((int64_t)k + o.p, std::min(d.m, d.n)) > 32) return RSVDGB_ERR_UNSUPPORTED;
        if (!r.d || (r.U && r.ldu < k) || (r.V && r.ldv < k)) return RSVDGB_ERR_INVALID_ARG;
    }
    return batched_rsvd(&h->batched, h->device, h->sm_count, h->stream, batch, descs, k, o, outs, infos);
}

static int controller_alloc(rsvdgb_handle* h)
{
    if (!h->ctl_params) RSVDGB_CUDA_TRY(cudaMalloc(&h->ctl_params, sizeof(float) * kMlpParams));
    if (!h->ctl_scratch) RSVDGB_CUDA_TRY(cudaMalloc(&h->ctl_scratch, sizeof(float) * 64));
    if (!h->ctl_host) RSVDGB_CUDA_TRY(cudaMallocHost(&h->ctl_host, sizeof(int) * 2));
    return RSVDGB_OK;
}

int rsvdgb_controller_set(rsvdgb_handle* h, const float* params_host)
{
    int rc = check_handle(h);
    if (rc) return rc;
    if (!params_host) return RSVDGB_ERR_INVALID_ARG;
    for (int i = 0; i < kMlpParams; ++i)
        if (!std::isfinite(params_host[i])) return RSVDGB_ERR_INVALID_ARG;
    for (int i = 0; i < kMlpIn; ++i)
        if (!(params_host[kMlpIn + i] > 0.f)) return RSVDGB_ERR_INVALID_ARG;  // sd > 0
    rc = controller_alloc(h);
    if (rc) return rc;
    RSVDGB_CUDA_TRY(cudaMemcpyAsync(h->ctl_params, params_host, sizeof(float) * kMlpParams, cudaMemcpyHostToDevice,
                                    h->stream));
    RSVDGB_CUDA_TRY(cudaStreamSynchronize(h->stream));
    return RSVDGB_OK;
}

int rsvdgb_controller_load(rsvdgb_handle* h, const char* path)
{
    int rc = check_handle(h);
    if (rc) return rc;
    if (!path) return RSVDGB_ERR_INVALID_ARG;
    FILE* f = std::fopen(path, "rb");
    if (!f) return RSVDGB_ERR_INVALID_ARG;
    char magic[8];
    int32_t count = 0;
    std::vector<float> P(kMlpParams);
    const bool ok = std::fread(magic, 1, 8, f) == 8 && std::memcmp(magic, "RSVDMLP1", 8) == 0 &&
                    std::fread(&count, 4, 1, f) == 1 && count == kMlpParams &&
                    std::fread(P.data(), sizeof(float), kMlpParams, f) == (size_t)kMlpParams;
    std::fclose(f);
    if (!ok) return RSVDGB_ERR_INVALID_ARG;
    return rsvdgb_controller_set(h, P.data());
}

int rsvdgb_controller_train(rsvdgb_handle* h, const char* dataset_path, const rsvdgb_train_opts* opts,
                            const char* out_path, float* final_loss)
{
    int rc = check_handle(h);
    if (rc) return rc;
    if (!dataset_path || !out_path) return RSVDGB_ERR_INVALID_ARG;
    rsvdgb_train_opts o;
    if (opts)
        o = *opts;
    else
        rsvdgb_default_train_opts(&o);
    FILE* f = std::fopen(dataset_path, "rb");
    if (!f) return RSVDGB_ERR_INVALID_ARG;
    char magic[8];
    int32_t n = 0, nf = 0;
    bool ok = std::fread(magic, 1, 8, f) == 8 && std::memcmp(magic, "RSVDDS01", 8) == 0 &&
              std::fread(&n, 4, 1, f) == 1 && std::fread(&nf, 4, 1, f) == 1 && n > 0 && nf == kMlpIn;
    std::vector<float> X, Y;
    if (ok) {
        X.resize((size_t)n * kMlpIn);
        Y.resize((size_t)n * kMlpOut);
        ok = std::fread(X.data(), sizeof(float), X.size(), f) == X.size() &&
             std::fread(Y.data(), sizeof(float), Y.size(), f) == Y.size();
    }
    std::fclose(f);
    if (!ok) return RSVDGB_ERR_INVALID_ARG;
    for (float v : X)
        if (!std::isfinite(v)) return RSVDGB_ERR_INVALID_ARG;
    for (float v : Y)
        if (!std::isfinite(v)) return RSVDGB_ERR_INVALID_ARG;
    std::vector<float> P(kMlpParams);
    rc = mlp_train(h->stream, X.data(), Y.data(), n, o.epochs, o.batch, o.lr, o.tau, o.seed, P.data(), final_loss);
    if (rc) return rc;
    FILE* g = std::fopen(out_path, "wb");
    if (!g) return RSVDGB_ERR_INVALID_ARG;
    const int32_t count = kMlpParams;
    ok = std::fwrite("RSVDMLP1", 1, 8, g) == 8 && std::fwrite(&count, 4, 1, g) == 1 &&
         std::fwrite(P.data(), sizeof(float), kMlpParams, g) == (size_t)kMlpParams;
    ok = (std::fclose(g) == 0) && ok;
    if (!ok) return RSVDGB_ERR_INVALID_ARG;
    return rsvdgb_controller_set(h, P.data());
}

int rsvdgb_controller_features(rsvdgb_handle* h, const void* A, int64_t m, int64_t n, int64_t lda, int dtype, int k,
                               const rsvdgb_opts* opts, float* feats)
{
    int rc = check_handle(h);
    if (rc) return rc;
    rsvdgb_opts o;
    if (opts)
        o = *opts;
    else
        rsvdgb_default_opts(&o);
    if (!feats || o.p_max < 2 || o.sdist < 0 || o.sdist > 2) return RSVDGB_ERR_INVALID_ARG;
    Geom g{};
    rc = make_geom(A, m, n, lda, dtype, o.layout, k, o.p_max, o.engine, o.prec, g);
    if (rc) return rc;
    Outputs out{};
    const Learned lc{k, o.p_max, o.q_max, feats};
    return run_fp32(h, g, k, 0, o.sdist, o.seed, out, &lc);
}

int rsvdgb_mlp_forward(rsvdgb_handle* h, const float* P, const float* X, int n, float* out)
{
    int rc = check_handle(h);
    if (rc) return rc;
    if (!P || !X || !out || n < 1) return RSVDGB_ERR_INVALID_ARG;
    launch_mlp_forward(h->stream, P, X, n, out);
    RSVDGB_CUDA_TRY(cudaGetLastError());
    return RSVDGB_OK;
}

int rsvdgb_mlp_grad(rsvdgb_handle* h, const float* P, const float* X, const float* Y, int n, float tau, float* grad,
                    float* loss)
{
    int rc = check_handle(h);
    if (rc) return rc;
    if (!P || !X || !Y || !grad || n < 1 || !(tau > 0.f && tau < 1.f)) return RSVDGB_ERR_INVALID_ARG;
    rc = ensure_workspace(h, sizeof(float) * mlp_grad_scratch_floats(n) + 256);
    if (rc) return rc;
    return launch_mlp_grad(h->stream, P, X, Y, nullptr, n, tau, (float*)h->ws, grad, loss);
}

int rsvdgb_profile_passes(rsvdgb_handle* h, int enable)
{
    int rc = check_handle(h);
    if (rc) return rc;
    cudaStreamSynchronize(h->stream);
    h->prof.on = enable != 0;
    h->prof.used = 0;
    h->prof.bytes = 0.0;
    return RSVDGB_OK;
}

int rsvdgb_profile_read(rsvdgb_handle* h, double* pass_ms, int64_t* pass_launches, double* pass_bytes)
{
    int rc = check_handle(h);
    if (rc) return rc;
    RSVDGB_CUDA_TRY(cudaStreamSynchronize(h->stream));
    double total = 0.0;
    for (size_t i = 0; i < h->prof.used; ++i) {
        float ms = 0.f;
        RSVDGB_CUDA_TRY(cudaEventElapsedTime(&ms, h->prof.ev[2 * i], h->prof.ev[2 * i + 1]));
        total += ms;
    }
    if (pass_ms) *pass_ms = total;
    if (pass_launches) *pass_launches = (int64_t)h->prof.used;
    if (pass_bytes) *pass_bytes = h->prof.bytes;
    return RSVDGB_OK;
}

int rsvdgb_test_pqr_barrier(rsvdgb_handle* h, int64_t spin_ticks)
{
    int rc = check_handle(h);
    if (rc) return rc;
    if (spin_ticks < 1) return RSVDGB_ERR_INVALID_ARG;
    h->test_pqr_absent = 1;
    h->test_spin = spin_ticks;
    return RSVDGB_OK;
}

int64_t rsvdgb_kernel_launches(void) { return launches_so_far(); }

}  // extern "C"
