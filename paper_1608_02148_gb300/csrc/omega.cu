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
#include "philox.cuh"

namespace rsvdgb {
namespace {

using philox::omega4;

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
