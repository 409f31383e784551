// Counter-based random numbers for the step kernels: Philox4x32-10 from
// Salmon, Moraes, Dror & Shaw, "Parallel random numbers: as easy as 1, 2, 3"
// (SC'11).  Ten rounds; each round multiplies words 0 and 2 by the two Philox
// constants (high and low halves via __umulhi), mixes in words 1 and 3 and the
// key, and the key advances by the two Weyl constants between rounds.
#pragma once
#include <cstdint>

namespace gn {

struct u32x4 {
    uint32_t x, y, z, w;
};

__device__ __forceinline__ u32x4 philox4x32_10(u32x4 c, uint32_t k0, uint32_t k1)
{
    constexpr uint32_t kMulA = 0xD2511F53u, kMulB = 0xCD9E8D57u;
    constexpr uint32_t kWeylA = 0x9E3779B9u, kWeylB = 0xBB67AE85u;
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint32_t hiA = __umulhi(kMulA, c.x), loA = kMulA * c.x;
        const uint32_t hiB = __umulhi(kMulB, c.z), loB = kMulB * c.z;
        c = u32x4{hiB ^ c.y ^ k0, loB, hiA ^ c.w ^ k1, loA};
        k0 += kWeylA;
        k1 += kWeylB;
    }
    return c;
}

// Stream ids of the draws (the counter's last word).
constexpr uint32_t kStreamBackground = 1u;
constexpr uint32_t kStreamObservation = 2u;

// Draw for (node, index, stream) under a 64-bit seed: counter
// {node, index low word, index high word, stream}, key {seed low, seed high}.
__device__ __forceinline__ u32x4 draw(uint64_t seed, uint32_t node, int64_t index, uint32_t stream)
{
    const uint64_t ui = static_cast<uint64_t>(index);
    return philox4x32_10(u32x4{node, static_cast<uint32_t>(ui), static_cast<uint32_t>(ui >> 32), stream},
                         static_cast<uint32_t>(seed), static_cast<uint32_t>(seed >> 32));
}

// Standard normal by Box-Muller (1958) from the top 23 bits of two words:
// u = (k + 1/2) 2^-23 is exact in FP32 and strictly inside (0, 1).
__device__ __forceinline__ float gauss_from(u32x4 r)
{
    const float u1 = (static_cast<float>(r.x >> 9) + 0.5f) * (1.0f / 8388608.0f);
    const float u2 = (static_cast<float>(r.y >> 9) + 0.5f) * (1.0f / 8388608.0f);
    return sqrtf(-2.0f * logf(u1)) * cospif(2.0f * u2);
}

}  // namespace gn
