// Test matrix Omega of Sec. 2.3 (Algorithm rqb step 2) on the GPU.
//
// Counter-based: element (i, j) is a pure function of (seed, i, j), so the
// matrix can be generated by any thread in any order, and a wider Omega
// extends a narrower one column by column.
//   key     = (seed mod 2^32, seed >> 32)
//   counter = (r mod 2^32, r >> 32, j, 0),  r = i / 4
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11) turns the counter into
// four 32-bit words x0..x3 for rows 4r..4r+3 of column j.
//   normal     : Box-Muller in double on (x0,x1) and (x2,x3), u = (x + 1/2) 2^-32,
//                rad = sqrt(-2 ln u_a), theta = 2 pi u_b, (rad cos, rad sin)
//   unif       : 2u - 1
//   rademacher : +1 if bit 31 of x_t is clear, else -1
// Values are rounded from double to the nearest float.
#include "internal.cuh"

namespace rsvdgb {
namespace {

__device__ __forceinline__ void philox_round(uint32_t& c0, uint32_t& c1, uint32_t& c2, uint32_t& c3, uint32_t k0,
                                             uint32_t k1)
{
    const uint32_t lo0 = 0xD2511F53u * c0;
    const uint32_t hi0 = __umulhi(0xD2511F53u, c0);
    const uint32_t lo1 = 0xCD9E8D57u * c2;
    const uint32_t hi1 = __umulhi(0xCD9E8D57u, c2);
    const uint32_t n0 = hi1 ^ c1 ^ k0;
    const uint32_t n2 = hi0 ^ c3 ^ k1;
    c0 = n0;
    c1 = lo1;
    c2 = n2;
    c3 = lo0;
}

__device__ __forceinline__ void philox10(uint32_t (&c)[4], uint32_t k0, uint32_t k1)
{
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        philox_round(c[0], c[1], c[2], c[3], k0, k1);
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
}

__device__ __forceinline__ double open_unit(uint32_t x) { return ((double)x + 0.5) * (1.0 / 4294967296.0); }

// Four consecutive rows 4r..4r+3 of column j.
__device__ __forceinline__ void omega4(uint64_t seed, int64_t r, int64_t j, int sdist, float (&v)[4])
{
    uint32_t c[4] = {(uint32_t)((uint64_t)r & 0xffffffffu), (uint32_t)((uint64_t)r >> 32), (uint32_t)j, 0u};
    philox10(c, (uint32_t)(seed & 0xffffffffu), (uint32_t)(seed >> 32));
    if (sdist == RSVDGB_SDIST_NORMAL) {
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const double ua = open_unit(c[2 * h]);
            const double ub = open_unit(c[2 * h + 1]);
            const double rad = sqrt(-2.0 * log(ua));
            const double theta = 6.283185307179586 * ub;
            v[2 * h] = (float)(rad * cos(theta));
            v[2 * h + 1] = (float)(rad * sin(theta));
        }
    } else if (sdist == RSVDGB_SDIST_UNIF) {
#pragma unroll
        for (int t = 0; t < 4; ++t) v[t] = (float)(2.0 * open_unit(c[t]) - 1.0);
    } else {
#pragma unroll
        for (int t = 0; t < 4; ++t) v[t] = (c[t] & 0x80000000u) ? -1.0f : 1.0f;
    }
}

// Column-major output; one thread per (row group r, column j).
__global__ void omega_colmajor_kernel(int64_t rows, int64_t nblk_pad, int l, int l_pad, uint64_t seed, int sdist,
                                      float* __restrict__ out, int64_t ld)
{
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y;
    if (r >= nblk_pad || j >= l_pad) return;
    float v[4] = {0.f, 0.f, 0.f, 0.f};
    if (j < l && 4 * r < rows) omega4(seed, r, j, sdist, v);
#pragma unroll
    for (int t = 0; t < 4; ++t)
        if (4 * r + t >= rows) v[t] = 0.f;
    float4* dst = reinterpret_cast<float4*>(out + (int64_t)j * ld + 4 * r);
    *dst = make_float4(v[0], v[1], v[2], v[3]);
}

__global__ void omega_rowmajor_kernel(int64_t rows, int l, uint64_t seed, int sdist, float* __restrict__ out,
                                      int64_t ld)
{
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y;
    if (4 * r >= rows || j >= l) return;
    float v[4];
    omega4(seed, r, j, sdist, v);
#pragma unroll
    for (int t = 0; t < 4; ++t)
        if (4 * r + t < rows) out[(4 * r + t) * ld + j] = v[t];
}

}  // namespace

void launch_omega(cudaStream_t s, int64_t rows, int64_t rows_pad, int l, int l_pad, uint64_t seed, int sdist,
                  float* out, int64_t ld)
{
    // rows_pad and ld are multiples of 4, so each thread writes one aligned float4.
    const int64_t nblk_pad = rows_pad / 4;
    dim3 block(128);
    dim3 grid((unsigned)ceil_div(nblk_pad, 128), (unsigned)l_pad);
    omega_colmajor_kernel<<<grid, block, 0, s>>>(rows, nblk_pad, l, l_pad, seed, sdist, out, ld); count_launches();
}

void launch_omega_rowmajor(cudaStream_t s, int64_t rows, int l, uint64_t seed, int sdist, float* out, int64_t ld)
{
    dim3 block(128);
    dim3 grid((unsigned)ceil_div(ceil_div(rows, 4), 128), (unsigned)l);
    omega_rowmajor_kernel<<<grid, block, 0, s>>>(rows, l, seed, sdist, out, ld); count_launches();
}

}  // namespace rsvdgb
