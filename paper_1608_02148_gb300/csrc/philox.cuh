// Counter-based test matrix Omega of Sec. 2.3 (device code).
//
//   key     = (seed mod 2^32, seed >> 32)
//   counter = (r mod 2^32, r >> 32, j, 0),  r = i / 4
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11) turns the counter into
// four 32-bit words x0..x3 for rows 4r..4r+3 of column j.
//   normal     : Box-Muller in double on (x0,x1) and (x2,x3), u = (x + 1/2) 2^-32,
//                rad = sqrt(-2 ln u_a), theta = 2 pi u_b, (rad cos, rad sin)
//   unif       : 2u - 1
//   rademacher : +1 if bit 31 of x_t is clear, else -1
// Values are rounded from double to the nearest float.
#pragma once

#include <stdint.h>

#include "../../include/rsvdgb.h"

namespace rsvdgb {
namespace philox {

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

}  // namespace philox
}  // namespace rsvdgb
