// tc_common.cuh -- device helpers shared by the tensor-core fitness kernels
// (single problem and batched): bounded mbarrier waits, the fused
// squared- or absolute-error epilogue step, and operand rounding to BF16 /
// E4M3.
#pragma once
#include <cuda_bf16.h>
#include <cuda_fp8.h>
#include <stdint.h>

#include "game_internal.cuh"
#include "tc_ptx.cuh"

namespace game {
namespace tc {

constexpr uint64_t kTimeoutNs = 2000000000ull;   // 2 s per wait
constexpr uint32_t kSuspendNs = 20000;           // per try_wait suspension (woken early on completion)

// Bounded wait for the phase of the given parity. Waiting threads are
// suspended by the hardware (suspend-time hint) instead of spinning, so they
// take no issue slots from the MMA issuer and the producers on their SM
// sub-partition; each wake-up re-checks the abort flag and the time limit.
static __device__ bool wait_bar(uint32_t bar, uint32_t parity, volatile int* abort_flag, int* status) {
  if (ptx::mbar_try_wait(bar, parity)) return true;
  const uint64_t t0 = ptx::global_timer_ns();
  for (;;) {
    if (ptx::mbar_try_wait_sleep(bar, parity, kSuspendNs)) return true;
    if (*abort_flag) return false;
    if (ptx::global_timer_ns() - t0 > kTimeoutNs) {
      *abort_flag = 1;
      atomicExch(status, (int)kDevTimeout);
      return false;
    }
  }
}

// Waits for this CTA's own asynchronous work (copies, MMAs) regardless of the
// abort flag, still bounded.
static __device__ void wait_bar_drain(uint32_t bar, uint32_t parity, int* status) {
  const uint64_t t0 = ptx::global_timer_ns();
  while (!ptx::mbar_try_wait(bar, parity)) {
    if (ptx::global_timer_ns() - t0 > kTimeoutNs) {
      atomicExch(status, (int)kDevTimeout);
      return;
    }
  }
}

// sse += ((y - bias) - u * acc)^2 over 32 columns, two columns per packed op
// (ABS: += |(y - bias) - u * acc|, the absolute error).
// SCALED = false: u = 1 and the residual is one packed subtraction; true
// (FP8): -u * acc + (y - bias) as one packed FMA (one rounding, as the
// subtraction is for u = 1).
// YS: the targets yc are in shared memory (else global memory, read through
// the read-only path).
template <bool SCALED, bool ABS = false, bool YS = false>
__device__ __forceinline__ void epi_chunk(const uint32_t (&v)[32], const float* yc,
                                          uint64_t bias2, uint64_t negu2, uint64_t& s2) {
#pragma unroll
  for (int e4 = 0; e4 < 8; ++e4) {
    const float4 yv = YS ? reinterpret_cast<const float4*>(yc)[e4]
                         : __ldg(reinterpret_cast<const float4*>(yc) + e4);
    const uint64_t ya = ptx::f2_sub(ptx::f2_pack(yv.x, yv.y), bias2);
    const uint64_t yb = ptx::f2_sub(ptx::f2_pack(yv.z, yv.w), bias2);
    const uint64_t da = ptx::f2_pack(__uint_as_float(v[4 * e4 + 0]), __uint_as_float(v[4 * e4 + 1]));
    const uint64_t db = ptx::f2_pack(__uint_as_float(v[4 * e4 + 2]), __uint_as_float(v[4 * e4 + 3]));
    const uint64_t ra = SCALED ? ptx::f2_fma(negu2, da, ya) : ptx::f2_sub(ya, da);
    const uint64_t rb = SCALED ? ptx::f2_fma(negu2, db, yb) : ptx::f2_sub(yb, db);
    if (ABS) {
      s2 = ptx::f2_add(s2, ptx::f2_abs(ra));
      s2 = ptx::f2_add(s2, ptx::f2_abs(rb));
    } else {
      s2 = ptx::f2_fma(ra, ra, s2);
      s2 = ptx::f2_fma(rb, rb, s2);
    }
  }
}

// Rounds 2 x 8 values to BF16 pairs (hi), and for bf16x3 also the residuals
// v - hi (lo).
__device__ __forceinline__ uint32_t bf16x2_bits(float lo_col, float hi_col) {
  const __nv_bfloat162 b = __floats2bfloat162_rn(lo_col, hi_col);
  return *reinterpret_cast<const uint32_t*>(&b);
}
__device__ __forceinline__ void split_bf16x2(float v0, float v1, uint32_t& hi, uint32_t& lo) {
  const __nv_bfloat162 h = __floats2bfloat162_rn(v0, v1);
  const float2 hf = __bfloat1622float2(h);
  hi = *reinterpret_cast<const uint32_t*>(&h);
  lo = bf16x2_bits(v0 - hf.x, v1 - hf.y);
}
__device__ __forceinline__ uint32_t e4m3x4_bits(float v0, float v1, float v2, float v3) {
  const uint32_t lo = __nv_cvt_float2_to_fp8x2(make_float2(v0, v1), __NV_SATFINITE, __NV_E4M3);
  const uint32_t hi = __nv_cvt_float2_to_fp8x2(make_float2(v2, v3), __NV_SATFINITE, __NV_E4M3);
  return lo | (hi << 16);
}

}  // namespace tc
}  // namespace game
