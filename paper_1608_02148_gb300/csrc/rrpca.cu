// Randomized robust PCA (Algorithm rrpca, Sec. 5): A = L + S by the inexact
// augmented Lagrange multiplier method, one randomized SVD per iteration.
//
// The low-rank part L = U diag(sigma') V^T is never stored during the
// iteration: one fused kernel per iteration forms each tile of L from the
// (thresholded) factors in shared memory and, in the same pass over A,
// updates the sparse part S, the multiplier Z and the next rSVD input
// X = A - S + Z / mu_next, and sums ||A - L - S||_F^2.  Only the final L is
// written out.  The host drives the loop (rank prediction and the stopping
// test need two small device-to-host copies per iteration).
#include "internal.cuh"

#include <vector>

namespace rsvdgb {
namespace {

constexpr int kTile = 64;   // 64 x 64 elements per block
constexpr int kTk = 32;     // rank chunk staged in shared memory

// max |a| (as the bits of a non-negative float) and per-block sum of a^2.
__global__ void __launch_bounds__(256) absmax_sumsq_kernel(const float* __restrict__ A, int64_t lda, int64_t m,
                                                           int64_t n, unsigned int* amax, double* part)
{
    double s = 0.0;
    float mx = 0.f;
    const int64_t total = m * n;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const float a = A[(e / n) * lda + e % n];
        mx = fmaxf(mx, fabsf(a));
        s += (double)a * a;
    }
    for (int o = 16; o > 0; o >>= 1) {
        s += __shfl_xor_sync(0xffffffffu, s, o);
        mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    }
    __shared__ double rs[8];
    __shared__ float rm[8];
    if ((threadIdx.x & 31) == 0) {
        rs[threadIdx.x >> 5] = s;
        rm[threadIdx.x >> 5] = mx;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        float u = 0.f;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
            t += rs[w];
            u = fmaxf(u, rm[w]);
        }
        part[blockIdx.x] = t;
        atomicMax(amax, __float_as_uint(u));  // non-negative floats order as their bits
    }
}

// Z = A / dual; S = 0; X = A - S + Z / mu0.
__global__ void init_kernel(const float* __restrict__ A, int64_t lda, int64_t m, int64_t n, float inv_dual,
                            float inv_mu0, float* __restrict__ S, int64_t lds, float* __restrict__ Z,
                            float* __restrict__ X)
{
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= m * n) return;
    const int64_t i = e / n, j = e % n;
    const float a = A[i * lda + j];
    const float z = a * inv_dual;
    S[i * lds + j] = 0.f;
    Z[e] = z;
    X[e] = fmaf(z, inv_mu0, a);
}

// One IALM iteration over a 64 x 64 tile (256 threads, each 4 rows x 4
// consecutive columns): L = U diag(sig) V^T from kl columns of U (m x ldu)
// and V (n x ldv); with mode 0
//   T = A - L + Z / mu;  S = shrink(T, lam / mu);  R = A - L - S;
//   Z += mu R;  X = A - S + Z / mu_next;  part[block] = sum R^2,
// with mode 1 only L is written (to Lout, ld ldl).
__global__ void __launch_bounds__(256) ialm_kernel(const float* __restrict__ A, int64_t lda, int64_t m, int64_t n,
                                                   const float* __restrict__ U, int64_t ldu,
                                                   const float* __restrict__ V, int64_t ldv,
                                                   const float* __restrict__ sig, int kl, float mu, float inv_mu,
                                                   float inv_mu_next, float thr, float* __restrict__ S, int64_t lds,
                                                   float* __restrict__ Z, float* __restrict__ X,
                                                   double* __restrict__ part, int mode, float* __restrict__ Lout,
                                                   int64_t ldl)
{
    __shared__ float Ut[kTk][kTile];
    __shared__ float Vt[kTk][kTile];
    __shared__ double red[8];
    const int tid = threadIdx.x;
    const int tx = tid & 15, ty = tid >> 4;  // columns 4 tx .. 4 tx + 3, rows ty + 16 a
    const int64_t i0 = (int64_t)blockIdx.y * kTile, j0 = (int64_t)blockIdx.x * kTile;
    float acc[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b] = 0.f;
    for (int t0 = 0; t0 < kl; t0 += kTk) {
        const int tn = min(kTk, kl - t0);
        __syncthreads();
        for (int e = tid; e < kTk * kTile; e += 256) {
            const int t = e / kTile, r = e % kTile;
            const int64_t i = i0 + r, j = j0 + r;
            Ut[t][r] = (t < tn && i < m) ? U[i * ldu + t0 + t] * sig[t0 + t] : 0.f;
            Vt[t][r] = (t < tn && j < n) ? V[j * ldv + t0 + t] : 0.f;
        }
        __syncthreads();
        for (int t = 0; t < tn; ++t) {
            const float4 v = *reinterpret_cast<const float4*>(&Vt[t][4 * tx]);
#pragma unroll
            for (int a = 0; a < 4; ++a) {
                const float u = Ut[t][ty + 16 * a];
                acc[a][0] = fmaf(u, v.x, acc[a][0]);
                acc[a][1] = fmaf(u, v.y, acc[a][1]);
                acc[a][2] = fmaf(u, v.z, acc[a][2]);
                acc[a][3] = fmaf(u, v.w, acc[a][3]);
            }
        }
    }
    float r2 = 0.f;
#pragma unroll
    for (int a = 0; a < 4; ++a) {
        const int64_t i = i0 + ty + 16 * a;
        if (i >= m) continue;
#pragma unroll
        for (int b = 0; b < 4; ++b) {
            const int64_t j = j0 + 4 * tx + b;
            if (j >= n) continue;
            const float L = acc[a][b];
            if (mode == 1) {
                Lout[i * ldl + j] = L;
                continue;
            }
            const float av = A[i * lda + j];
            const int64_t e = i * n + j;
            const float z = Z[e];
            const float tv = fmaf(z, inv_mu, av - L);
            const float s = copysignf(fmaxf(fabsf(tv) - thr, 0.f), tv);
            const float r = av - L - s;
            const float zn = fmaf(mu, r, z);
            S[i * lds + j] = s;
            Z[e] = zn;
            X[e] = fmaf(zn, inv_mu_next, av - s);
            r2 = fmaf(r, r, r2);
        }
    }
    if (mode == 1) return;
    double rd = (double)r2;
    for (int o = 16; o > 0; o >>= 1) rd += __shfl_xor_sync(0xffffffffu, rd, o);
    if ((tid & 31) == 0) red[tid >> 5] = rd;
    __syncthreads();
    if (tid == 0) {
        double t = 0.0;
        for (int w = 0; w < 8; ++w) t += red[w];
        part[(int64_t)blockIdx.y * gridDim.x + blockIdx.x] = t;
    }
}

// Fixed-order sum of count doubles (one block).
__global__ void __launch_bounds__(1024) sum_kernel(const double* __restrict__ part, int64_t count,
                                                   double* __restrict__ out)
{
    __shared__ double red[32];
    double t = 0.0;
    for (int64_t i = threadIdx.x; i < count; i += blockDim.x) t += part[i];
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = t;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
        *out = s;
    }
}

}  // namespace

int64_t ialm_blocks(int64_t m, int64_t n) { return ceil_div(m, kTile) * ceil_div(n, kTile); }

void launch_absmax_sumsq(cudaStream_t s, const float* A, int64_t lda, int64_t m, int64_t n, unsigned int* amax,
                         double* part, int nblocks, double* sumsq)
{
    absmax_sumsq_kernel<<<nblocks, 256, 0, s>>>(A, lda, m, n, amax, part);
    sum_kernel<<<1, 1024, 0, s>>>(part, nblocks, sumsq);
    count_launches(2);
}

void launch_ialm_init(cudaStream_t s, const float* A, int64_t lda, int64_t m, int64_t n, float inv_dual,
                      float inv_mu0, float* S, int64_t lds, float* Z, float* X)
{
    init_kernel<<<(unsigned)ceil_div(m * n, 256), 256, 0, s>>>(A, lda, m, n, inv_dual, inv_mu0, S, lds, Z, X);
    count_launches();
}

void launch_ialm_step(cudaStream_t s, const float* A, int64_t lda, int64_t m, int64_t n, const float* U, int64_t ldu,
                      const float* V, int64_t ldv, const float* sig, int kl, float mu, float inv_mu,
                      float inv_mu_next, float thr, float* S, int64_t lds, float* Z, float* X, double* part,
                      double* err2, int mode, float* Lout, int64_t ldl)
{
    const dim3 grid((unsigned)ceil_div(n, kTile), (unsigned)ceil_div(m, kTile));
    ialm_kernel<<<grid, 256, 0, s>>>(A, lda, m, n, U, ldu, V, ldv, sig, kl, mu, inv_mu, inv_mu_next, thr, S, lds, Z,
                                     X, part, mode, Lout, ldl);
    count_launches();
    if (mode == 0) {
        sum_kernel<<<1, 1024, 0, s>>>(part, (int64_t)grid.x * grid.y, err2);
        count_launches();
    }
}

}  // namespace rsvdgb
