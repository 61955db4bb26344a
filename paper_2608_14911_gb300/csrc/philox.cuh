// Counter-based Philox4x32-10 on the device (Salmon, Moraes, Dror, Shaw,
// "Parallel random numbers: as easy as 1, 2, 3", SC'11), written from the
// published definition: ten rounds of two 32x32->64-bit multiplies
// (0xD2511F53, 0xCD9E8D57) whose halves are permuted and xor-ed with the key,
// the key advancing by the Weyl constants (0x9E3779B9, 0xBB67AE85) between
// rounds.
#pragma once
#include <cuda_runtime.h>

namespace espp {

__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r > 0) {
            k.x += 0x9E3779B9u;
            k.y += 0xBB67AE85u;
        }
        const unsigned int hi0 = __umulhi(0xD2511F53u, c.x), lo0 = 0xD2511F53u * c.x;
        const unsigned int hi1 = __umulhi(0xCD9E8D57u, c.z), lo1 = 0xCD9E8D57u * c.z;
        c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
    }
    return c;
}

// Top 24 bits k of a word -> (2k + 1 - 2^24) * 2^-25: an odd multiple of 2^-25
// in (-1/2, 1/2), exact in float and double, mean 0, variance (1-2^-48)/12.
template <class T>
__device__ __forceinline__ T uniform_centered(unsigned int w) {
    const int odd = 2 * (int)(w >> 8) + 1 - 16777216;
    return (T)odd * (T)2.98023223876953125e-08;
}

// Langevin noise of one particle: key (seed lo, seed hi), counter
// (local id, step lo, step hi, tag 0); words 0..2 -> x, y, z.
template <class T>
__device__ __forceinline__ void langevin_noise(unsigned long long seed, int id, long long step,
                                               T& rx, T& ry, T& rz) {
    const unsigned long long s = (unsigned long long)step;
    const uint4 o = philox4x32_10(make_uint4((unsigned int)id, (unsigned int)(s & 0xffffffffull),
                                             (unsigned int)(s >> 32), 0u),
                                  make_uint2((unsigned int)(seed & 0xffffffffull),
                                             (unsigned int)(seed >> 32)));
    rx = uniform_centered<T>(o.x);
    ry = uniform_centered<T>(o.y);
    rz = uniform_centered<T>(o.z);
}

// DPD pair noise theta_ij = sqrt(12) u (zero mean, unit variance): word 0 of
// Philox4x32-10 with key (seed lo, seed hi) and counter (min id, max id | 2^31,
// step lo, step hi); symmetric in the two ids.
template <class T>
__device__ __forceinline__ T dpd_theta(unsigned long long seed, int a, int b, long long step) {
    const unsigned long long s = (unsigned long long)step;
    const unsigned int lo = (unsigned int)min(a, b), hi = (unsigned int)max(a, b) | 0x80000000u;
    const uint4 o = philox4x32_10(make_uint4(lo, hi, (unsigned int)(s & 0xffffffffull), (unsigned int)(s >> 32)),
                                  make_uint2((unsigned int)(seed & 0xffffffffull), (unsigned int)(seed >> 32)));
    return uniform_centered<T>(o.x);
}

}  // namespace espp
