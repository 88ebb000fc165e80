// philox.cuh -- Philox4x32-10 counter-based generator on the device
// (Salmon, Moraes, Dror, Shaw, "Parallel Random Numbers: As Easy as 1, 2, 3",
// SC'11). Each draw is a pure function of a 64-bit key and a 128-bit counter,
// so the GA's random decisions are indexed by (generation, slot, gene, purpose)
// and need no stored generator state.
#pragma once
#include <stdint.h>

namespace game {

// Purpose tags: the last counter word keeps the streams of one slot apart.
enum : uint32_t {
  kTagInit = 1,
  kTagTour = 2,
  kTagCross = 3,
  kTagMut = 4,
  kTagGauss0 = 5,
  kTagGauss1 = 6,
  kTagGauss2 = 7,
  kTagImmigrant = 8,
  kTagSurrogate = 9   // initial weights of the fitness surrogate
};

__device__ __forceinline__ uint4 philox4x32_10(uint64_t key, uint32_t c0, uint32_t c1,
                                               uint32_t c2, uint32_t c3) {
  uint32_t k0 = static_cast<uint32_t>(key);
  uint32_t k1 = static_cast<uint32_t>(key >> 32);
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint32_t hi_a = __umulhi(0xD2511F53u, c0);
    const uint32_t lo_a = 0xD2511F53u * c0;
    const uint32_t hi_b = __umulhi(0xCD9E8D57u, c2);
    const uint32_t lo_b = 0xCD9E8D57u * c2;
    c0 = hi_b ^ c1 ^ k0;
    c1 = lo_b;
    c2 = hi_a ^ c3 ^ k1;
    c3 = lo_a;
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
  return make_uint4(c0, c1, c2, c3);
}

// A gene uniform in [-1, 1): the top 24 bits as a signed offset times 2^-23,
// exact in FP32.
__device__ __forceinline__ float uniform_gene(uint32_t w) {
  const int v = static_cast<int>(w >> 8) - (1 << 23);
  return __fmul_rn(__int2float_rn(v), 1.0f / 8388608.0f);
}

// Standard normal from twelve 24-bit uniforms (Irwin-Hall, n = 12, variance
// 1): the centred integer sum is exact, rounded once to FP32 (nearest even)
// and scaled by 2^-24.
__device__ __forceinline__ float irwin_hall12(uint64_t key, uint32_t g, uint32_t s,
                                              uint32_t k) {
  long long sum = 0;
  const uint32_t tags[3] = {kTagGauss0, kTagGauss1, kTagGauss2};
#pragma unroll
  for (int t = 0; t < 3; ++t) {
    const uint4 w = philox4x32_10(key, g, s, k, tags[t]);
    sum += (w.x >> 8) + (w.y >> 8) + (long long)(w.z >> 8) + (w.w >> 8);
  }
  sum -= 6LL * 16777216LL;
  return __fmul_rn(__ll2float_rn(sum), 1.0f / 16777216.0f);
}

}  // namespace game
