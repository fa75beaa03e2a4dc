// Learned choice of the power-iteration count q and the oversampling p.
//
// The paper leaves q and p to the user (Sec. 3.4: p = 10 and q = 1 or 2 are
// recommended; a slowly decaying spectrum needs more subspace iterations and
// oversampling).  This controller predicts them per matrix from cheap
// statistics of the first sketch: pass 1 runs with the widest sketch
// l_max = k + p_max, the diagonal of the CholeskyQR factor R of Y = A Omega
// (residual energies of the sketch columns, see features_kernel) and
// ||A||_F^2 give 16 features, and a small MLP (16 -> 64 -> 64 -> 2,
// ReLU, FP32) maps them to (q, log2 p).  Omega's columns are nested in l, so
// the first k + p columns of that sketch are exactly the sketch for the chosen
// p and the run continues from there.  The plain fixed-(q, p) method is the
// fallback when no controller is loaded.
//
// Training (on the GPU, these kernels): pinball loss with quantile tau (0.9
// penalises under-prediction, i.e. a failed accuracy target, more than
// over-prediction), minibatch gradients by hand-written forward and backward
// kernels, Adam.
//
// Parameter layout (FP32, kMlpParams floats): mu[16], sd[16] (input
// standardisation, not trained), W1[64][16], b1[64], W2[64][64], b2[64],
// W3[2][64], b3[2]; the trainable part starts at kOffW1.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <random>
#include <vector>

#include "internal.cuh"

namespace rsvdgb {
namespace {

constexpr int NI = kMlpIn, NH = kMlpHidden, NO = kMlpOut;
constexpr int kOffMu = 0, kOffSd = NI, kOffW1 = 2 * NI;
constexpr int kOffB1 = kOffW1 + NH * NI;
constexpr int kOffW2 = kOffB1 + NH;
constexpr int kOffB2 = kOffW2 + NH * NH;
constexpr int kOffW3 = kOffB2 + NH;
constexpr int kOffB3 = kOffW3 + NO * NH;
static_assert(kOffB3 + NO == kMlpParams, "parameter layout");
constexpr int kTrain = kMlpParams - kOffW1;  // trainable parameters
constexpr int kBS = 64;                      // samples per CTA in the gradient kernel
constexpr int kGradThreads = 256;

__device__ __forceinline__ float relu(float x) { return x > 0.f ? x : 0.f; }

// ---------------------------------------------------------------- features
// 16 scale-free statistics of the first sketch Y (m x lmax) from its
// CholeskyQR factor R (Y = Q R, R row-major lmax x lmax) and ||A||_F^2.
// R_jj^2 is the energy of column j of Y outside the span of columns 1..j-1:
// for the Gaussian sketch it estimates ||A - Q_{j-1} Q_{j-1}^T A||_F^2, the
// error of the rank-(j-1) range finder without oversampling or iterations
// (and R_11^2 estimates ||A||_F^2), so log10(R_jj / R_11) around j = k maps
// out how much oversampling and how many iterations the target needs.
__global__ void features_kernel(const float* __restrict__ R, int lmax, const double* __restrict__ fro2, int64_t m,
                                int64_t n, int k, int p_max, float* __restrict__ f)
{
    // one warp: lane c takes the columns j = c + 1, c + 33, ... of the sums
    // (FP64 per lane, then a shuffle reduction); lane 0 writes the features
    if (blockIdx.x != 0 || threadIdx.x >= 32) return;
    const int lane = threadIdx.x;
    const float tiny = 1e-30f;
    auto rd = [&](int j) {  // |R_jj|, j 1-based, clamped to [1, lmax]
        j = min(max(j, 1), lmax);
        return fmaxf(fabsf(R[(int64_t)(j - 1) * lmax + (j - 1)]), tiny);
    };
    const float r1 = rd(1);
    auto lr = [&](int j) { return log10f(rd(j) / r1); };
    double e_all = 0.0, e_k = 0.0, tr = 0.0;
    for (int j = 1 + lane; j <= lmax; j += 32) {
        const double v = (double)rd(j) * (double)rd(j);
        e_all += v;
        if (j <= k) e_k += v;
        // trace(G) = sum_j ||y_j||^2 = sum over the column j of R of R_ij^2
        for (int i = 1; i <= j; ++i) {
            const double x = (double)R[(int64_t)(i - 1) * lmax + (j - 1)];
            tr += x * x;
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        e_all += __shfl_xor_sync(0xffffffffu, e_all, o);
        e_k += __shfl_xor_sync(0xffffffffu, e_k, o);
        tr += __shfl_xor_sync(0xffffffffu, tr, o);
    }
    if (lane != 0) return;
    const double fa = fro2 ? *fro2 : 0.0;
    f[0] = log10f((float)m);
    f[1] = log10f((float)n);
    f[2] = log10f((float)k);
    f[3] = (float)k / (float)min(m, n);
    f[4] = lr((k + 3) / 4);
    f[5] = lr((k + 1) / 2);
    f[6] = lr((3 * k + 3) / 4);
    f[7] = lr(k);
    f[8] = lr(k + 1);
    f[9] = lr(k + max(p_max / 4, 1));
    f[10] = lr(k + max(p_max / 2, 1));
    f[11] = lr(lmax);
    f[12] = e_all > 0.0 ? (float)(e_k / e_all) : 1.f;
    // sketch energy per column relative to ||A||_F^2 (E ||A w||^2 = ||A||_F^2)
    f[13] = (fa > 0.0 && tr > 0.0) ? log10f((float)(tr / ((double)lmax * fa))) : 0.f;
    f[14] = log10f(rd(min(k, lmax)) / rd(lmax));
    f[15] = (float)p_max / (float)k;
}

// ---------------------------------------------------------------- inference
// out[i] = MLP((X[i] - mu) / sd).
__global__ void __launch_bounds__(NH) mlp_forward_kernel(const float* __restrict__ P, const float* __restrict__ X,
                                                           int n, float* __restrict__ out)
{
    // one CTA per sample, thread j = hidden unit j; every sum runs over its
    // inputs in increasing order, as a single thread would
    __shared__ float x[NI], h1[NH], h2[NH];
    const int i = blockIdx.x, j = threadIdx.x;
    if (i >= n) return;
    if (j < NI) x[j] = (X[(int64_t)i * NI + j] - P[kOffMu + j]) / P[kOffSd + j];
    __syncthreads();
    float a = P[kOffB1 + j];
#pragma unroll
    for (int t = 0; t < NI; ++t) a = fmaf(P[kOffW1 + j * NI + t], x[t], a);
    h1[j] = relu(a);
    __syncthreads();
    float b = P[kOffB2 + j];
#pragma unroll 16
    for (int t = 0; t < NH; ++t) b = fmaf(P[kOffW2 + j * NH + t], h1[t], b);
    h2[j] = relu(b);
    __syncthreads();
    if (j < NO) {
        float o = P[kOffB3 + j];
        for (int t = 0; t < NH; ++t) o = fmaf(P[kOffW3 + j * NH + t], h2[t], o);
        out[(int64_t)i * NO + j] = o;
    }
}

// (q, p) from the network's (q_hat, log2 p_hat), rounded up from kRoundUp
// below the next integer (an under-estimate costs accuracy, an over-estimate
// only time) and clamped; l = k + p is kept <= min(m, n).  A NaN output gives
// (q_max, p_max).
constexpr float kRoundUp = 0.35f;
__global__ void decide_kernel(const float* __restrict__ o, int q_max, int p_min, int p_max, int k, int64_t mn,
                              int* __restrict__ qp)
{
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    const float qh = o[0], lp = o[1];
    int q = (qh == qh) ? (int)floorf(fminf(fmaxf(qh + kRoundUp, 0.f), (float)q_max)) : q_max;
    float pf = (lp == lp) ? exp2f(fminf(fmaxf(lp, 0.f), 16.f)) : (float)p_max;
    int p = (int)floorf(pf + kRoundUp);
    p = max(p_min, min(p, p_max));
    if ((int64_t)p > mn - k) p = (int)(mn - k);
    qp[0] = q;
    qp[1] = p;
}

// ---------------------------------------------------------------- training
// Loss of one sample: sum over the two outputs of the pinball loss
// rho_tau(u) = u (tau - [u < 0]), u = y - y_hat; the batch loss is the mean.
// Each CTA takes kBS samples (idx gives their rows; null = consecutive) and
// writes its share of the gradient of the batch mean (1 / nb scaling).
__global__ void __launch_bounds__(kGradThreads)
    mlp_grad_kernel(const float* __restrict__ P, const float* __restrict__ X, const float* __restrict__ Y,
                    const int* __restrict__ idx, int nb, float tau, float* __restrict__ partial,
                    float* __restrict__ loss_part)
{
    extern __shared__ __align__(16) float gsm[];
    float* Xs = gsm;              // kBS x NI
    float* H1 = Xs + kBS * NI;    // kBS x NH
    float* H2 = H1 + kBS * NH;    // kBS x NH
    float* D2 = H2 + kBS * NH;    // kBS x NH
    float* D1 = D2 + kBS * NH;    // kBS x NH
    float* dO = D1 + kBS * NH;    // kBS x NO
    __shared__ float red[kGradThreads / 32];
    const int tid = threadIdx.x;
    const int s0 = blockIdx.x * kBS;
    const int ns = min(kBS, nb - s0);
    const float inv_nb = 1.f / (float)nb;

    for (int e = tid; e < kBS * NI; e += kGradThreads) {
        const int s = e / NI, t = e % NI;
        float v = 0.f;
        if (s < ns) {
            const int row = idx ? idx[s0 + s] : s0 + s;
            v = (X[(int64_t)row * NI + t] - P[kOffMu + t]) / P[kOffSd + t];
        }
        Xs[e] = v;
    }
    __syncthreads();
    for (int e = tid; e < kBS * NH; e += kGradThreads) {
        const int s = e / NH, j = e % NH;
        float a = P[kOffB1 + j];
#pragma unroll
        for (int t = 0; t < NI; ++t) a = fmaf(P[kOffW1 + j * NI + t], Xs[s * NI + t], a);
        H1[e] = relu(a);
    }
    __syncthreads();
    for (int e = tid; e < kBS * NH; e += kGradThreads) {
        const int s = e / NH, j = e % NH;
        float a = P[kOffB2 + j];
        for (int t = 0; t < NH; ++t) a = fmaf(P[kOffW2 + j * NH + t], H1[s * NH + t], a);
        H2[e] = relu(a);
    }
    __syncthreads();
    float lsum = 0.f;
    for (int e = tid; e < kBS * NO; e += kGradThreads) {
        const int s = e / NO, c = e % NO;
        float g = 0.f;
        if (s < ns) {
            float o = P[kOffB3 + c];
            for (int t = 0; t < NH; ++t) o = fmaf(P[kOffW3 + c * NH + t], H2[s * NH + t], o);
            const int row = idx ? idx[s0 + s] : s0 + s;
            const float u = Y[(int64_t)row * NO + c] - o;
            const float w = (u < 0.f) ? tau - 1.f : tau;
            lsum += u * w;
            g = -w * inv_nb;  // d loss / d o
        }
        dO[e] = g;
    }
    __syncthreads();
    // D2 = (dO W3) * [H2 > 0]
    for (int e = tid; e < kBS * NH; e += kGradThreads) {
        const int s = e / NH, j = e % NH;
        float a = 0.f;
#pragma unroll
        for (int c = 0; c < NO; ++c) a = fmaf(dO[s * NO + c], P[kOffW3 + c * NH + j], a);
        D2[e] = H2[e] > 0.f ? a : 0.f;
    }
    __syncthreads();
    // D1 = (D2 W2) * [H1 > 0]
    for (int e = tid; e < kBS * NH; e += kGradThreads) {
        const int s = e / NH, t = e % NH;
        float a = 0.f;
        for (int j = 0; j < NH; ++j) a = fmaf(D2[s * NH + j], P[kOffW2 + j * NH + t], a);
        D1[e] = H1[e] > 0.f ? a : 0.f;
    }
    __syncthreads();
    // parameter gradients of this CTA's samples
    float* gp = partial + (int64_t)blockIdx.x * kTrain;
    for (int e = tid; e < kTrain; e += kGradThreads) {
        const int pi = e + kOffW1;
        float a = 0.f;
        if (pi < kOffB1) {  // W1[j][t]
            const int j = (pi - kOffW1) / NI, t = (pi - kOffW1) % NI;
            for (int s = 0; s < kBS; ++s) a = fmaf(D1[s * NH + j], Xs[s * NI + t], a);
        } else if (pi < kOffW2) {  // b1[j]
            const int j = pi - kOffB1;
            for (int s = 0; s < kBS; ++s) a += D1[s * NH + j];
        } else if (pi < kOffB2) {  // W2[j][t]
            const int j = (pi - kOffW2) / NH, t = (pi - kOffW2) % NH;
            for (int s = 0; s < kBS; ++s) a = fmaf(D2[s * NH + j], H1[s * NH + t], a);
        } else if (pi < kOffW3) {  // b2[j]
            const int j = pi - kOffB2;
            for (int s = 0; s < kBS; ++s) a += D2[s * NH + j];
        } else if (pi < kOffB3) {  // W3[c][t]
            const int c = (pi - kOffW3) / NH, t = (pi - kOffW3) % NH;
            for (int s = 0; s < kBS; ++s) a = fmaf(dO[s * NO + c], H2[s * NH + t], a);
        } else {  // b3[c]
            const int c = pi - kOffB3;
            for (int s = 0; s < kBS; ++s) a += dO[s * NO + c];
        }
        gp[e] = a;
    }
    // loss share of this CTA (mean over the batch)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) lsum += __shfl_xor_sync(0xffffffffu, lsum, o);
    if ((tid & 31) == 0) red[tid >> 5] = lsum;
    __syncthreads();
    if (tid == 0) {
        float t = 0.f;
        for (int w = 0; w < kGradThreads / 32; ++w) t += red[w];
        loss_part[blockIdx.x] = t * inv_nb;
    }
}

// grad[e] = sum over CTAs of partial[c][e] (fixed order); loss likewise.
__global__ void mlp_grad_reduce_kernel(const float* __restrict__ partial, const float* __restrict__ loss_part,
                                       int ctas, float* __restrict__ grad, float* __restrict__ loss)
{
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e < kTrain) {
        float a = 0.f;
        for (int c = 0; c < ctas; ++c) a += partial[(int64_t)c * kTrain + e];
        grad[e] = a;
    }
    if (e == 0 && loss) {
        float a = 0.f;
        for (int c = 0; c < ctas; ++c) a += loss_part[c];
        *loss = a;
    }
}

// Adam (Kingma and Ba) on the trainable parameters, step t >= 1.
__global__ void adam_kernel(float* __restrict__ P, const float* __restrict__ grad, float* __restrict__ m1,
                            float* __restrict__ m2, int t, float lr, float b1, float b2, float eps)
{
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= kTrain) return;
    const float g = grad[e];
    const float a = b1 * m1[e] + (1.f - b1) * g;
    const float v = b2 * m2[e] + (1.f - b2) * g * g;
    m1[e] = a;
    m2[e] = v;
    const float ah = a / (1.f - powf(b1, (float)t));
    const float vh = v / (1.f - powf(b2, (float)t));
    P[kOffW1 + e] -= lr * ah / (sqrtf(vh) + eps);
}

constexpr size_t kGradSmem = sizeof(float) * (kBS * NI + 4 * kBS * NH + kBS * NO);

}  // namespace

void launch_controller_features(cudaStream_t s, const float* R, int lmax, const double* fro2, int64_t m, int64_t n,
                                int k, int p_max, float* feats)
{
    features_kernel<<<1, 32, 0, s>>>(R, lmax, fro2, m, n, k, p_max, feats);
    count_launches();
}

void launch_mlp_forward(cudaStream_t s, const float* P, const float* X, int n, float* out)
{
    if (n <= 0) return;
    mlp_forward_kernel<<<n, NH, 0, s>>>(P, X, n, out);
    count_launches();
}

void launch_controller_decide(cudaStream_t s, const float* out2, int q_max, int p_min, int p_max, int k, int64_t mn,
                              int* qp)
{
    decide_kernel<<<1, 32, 0, s>>>(out2, q_max, p_min, p_max, k, mn, qp);
    count_launches();
}

size_t mlp_grad_scratch_floats(int nb) { return (size_t)((nb + kBS - 1) / kBS) * (kTrain + 1); }

int launch_mlp_grad(cudaStream_t s, const float* P, const float* X, const float* Y, const int* idx, int nb, float tau,
                    float* scratch, float* grad, float* loss)
{
    if (nb <= 0) return RSVDGB_ERR_INVALID_ARG;
    if (cudaFuncSetAttribute(mlp_grad_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kGradSmem) !=
        cudaSuccess)
        return RSVDGB_ERR_CUDA;
    const int ctas = (nb + kBS - 1) / kBS;
    float* partial = scratch;
    float* loss_part = scratch + (size_t)ctas * kTrain;
    mlp_grad_kernel<<<ctas, kGradThreads, kGradSmem, s>>>(P, X, Y, idx, nb, tau, partial, loss_part);
    mlp_grad_reduce_kernel<<<(kTrain + 255) / 256, 256, 0, s>>>(partial, loss_part, ctas, grad, loss);
    count_launches(2);
    return cudaGetLastError() == cudaSuccess ? RSVDGB_OK : RSVDGB_ERR_CUDA;
}

// Host-driven training loop: seeded He initialisation, standardisation from
// the data, then epochs of shuffled minibatches (grad + Adam per step).
int mlp_train(cudaStream_t s, const float* X_host, const float* Y_host, int n, int epochs, int batch, float lr,
              float tau, uint64_t seed, float* P_host_out, float* final_loss)
{
    if (n < 1 || epochs < 1 || batch < 1 || !(lr > 0.f) || !(tau > 0.f && tau < 1.f)) return RSVDGB_ERR_INVALID_ARG;
    batch = std::min(batch, n);
    std::vector<float> P(kMlpParams, 0.f);
    // standardisation
    for (int t = 0; t < NI; ++t) {
        double mu = 0.0, sq = 0.0;
        for (int i = 0; i < n; ++i) mu += X_host[(size_t)i * NI + t];
        mu /= n;
        for (int i = 0; i < n; ++i) {
            const double d = X_host[(size_t)i * NI + t] - mu;
            sq += d * d;
        }
        const double sd = std::sqrt(sq / n);
        P[kOffMu + t] = (float)mu;
        P[kOffSd + t] = (float)(sd > 1e-6 ? sd : 1.0);
    }
    std::mt19937_64 rng(seed);
    std::normal_distribution<float> nd(0.f, 1.f);
    for (int j = 0; j < NH * NI; ++j) P[kOffW1 + j] = nd(rng) * std::sqrt(2.f / NI);
    for (int j = 0; j < NH * NH; ++j) P[kOffW2 + j] = nd(rng) * std::sqrt(2.f / NH);
    for (int j = 0; j < NO * NH; ++j) P[kOffW3 + j] = nd(rng) * std::sqrt(1.f / NH);
    // output biases start at the label means (q, log2 p)
    for (int c = 0; c < NO; ++c) {
        double a = 0.0;
        for (int i = 0; i < n; ++i) a += Y_host[(size_t)i * NO + c];
        P[kOffB3 + c] = (float)(a / n);
    }

    float *dP = nullptr, *dX = nullptr, *dY = nullptr, *dG = nullptr, *dM1 = nullptr, *dM2 = nullptr, *dS = nullptr,
          *dL = nullptr;
    int* dIdx = nullptr;
    const size_t scratch = mlp_grad_scratch_floats(n);  // also serves the final whole-set loss
    auto cleanup = [&]() {
        cudaFree(dP); cudaFree(dX); cudaFree(dY); cudaFree(dG); cudaFree(dM1); cudaFree(dM2); cudaFree(dS);
        cudaFree(dL); cudaFree(dIdx);
    };
    if (cudaMalloc(&dP, sizeof(float) * kMlpParams) || cudaMalloc(&dX, sizeof(float) * (size_t)n * NI) ||
        cudaMalloc(&dY, sizeof(float) * (size_t)n * NO) || cudaMalloc(&dG, sizeof(float) * kTrain) ||
        cudaMalloc(&dM1, sizeof(float) * kTrain) || cudaMalloc(&dM2, sizeof(float) * kTrain) ||
        cudaMalloc(&dS, sizeof(float) * scratch) || cudaMalloc(&dL, sizeof(float)) ||
        cudaMalloc(&dIdx, sizeof(int) * (size_t)n)) {
        cleanup();
        cudaGetLastError();
        return RSVDGB_ERR_NOMEM;
    }
    cudaMemcpyAsync(dP, P.data(), sizeof(float) * kMlpParams, cudaMemcpyHostToDevice, s);
    cudaMemcpyAsync(dX, X_host, sizeof(float) * (size_t)n * NI, cudaMemcpyHostToDevice, s);
    cudaMemcpyAsync(dY, Y_host, sizeof(float) * (size_t)n * NO, cudaMemcpyHostToDevice, s);
    cudaMemsetAsync(dM1, 0, sizeof(float) * kTrain, s);
    cudaMemsetAsync(dM2, 0, sizeof(float) * kTrain, s);
    std::vector<int> perm(n);
    for (int i = 0; i < n; ++i) perm[i] = i;
    int t = 0;
    int rc = RSVDGB_OK;
    for (int ep = 0; ep < epochs && rc == RSVDGB_OK; ++ep) {
        std::shuffle(perm.begin(), perm.end(), rng);
        // the permutation is consumed by the kernels of this epoch before the
        // next upload (same stream)
        cudaMemcpyAsync(dIdx, perm.data(), sizeof(int) * (size_t)n, cudaMemcpyHostToDevice, s);
        cudaStreamSynchronize(s);
        for (int b0 = 0; b0 + batch <= n; b0 += batch) {
            rc = launch_mlp_grad(s, dP, dX, dY, dIdx + b0, batch, tau, dS, dG, dL);
            if (rc) break;
            ++t;
            adam_kernel<<<(kTrain + 255) / 256, 256, 0, s>>>(dP, dG, dM1, dM2, t, lr, 0.9f, 0.999f, 1e-8f);
            count_launches();
        }
    }
    if (rc == RSVDGB_OK) {
        // loss of the final parameters on the whole set
        rc = launch_mlp_grad(s, dP, dX, dY, nullptr, n, tau, dS, dG, dL);
    }
    cudaMemcpyAsync(P.data(), dP, sizeof(float) * kMlpParams, cudaMemcpyDeviceToHost, s);
    float lh = 0.f;
    cudaMemcpyAsync(&lh, dL, sizeof(float), cudaMemcpyDeviceToHost, s);
    if (cudaStreamSynchronize(s) != cudaSuccess) rc = RSVDGB_ERR_CUDA;
    cleanup();
    if (rc) return rc;
    std::memcpy(P_host_out, P.data(), sizeof(float) * kMlpParams);
    if (final_loss) *final_loss = lh;
    return RSVDGB_OK;
}

}  // namespace rsvdgb
