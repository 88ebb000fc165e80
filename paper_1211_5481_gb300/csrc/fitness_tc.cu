// fitness_tc.cu -- fitness of a population with the contraction on the
// 5th-generation tensor cores (tcgen05, BF16 operands, FP32 accumulation in
// tensor memory), the squared-error reduction fused into the epilogue.
//
// Math (paper Section 3): Out_p(m) = a_{p,0} + sum_c a_{p,c+1} phi_c(x_m)
// (Eq. 2), fit_p = (1/M) sum_m (y_m - Out_p(m))^2 (Eq. 3, MSE). The
// expansion phi does not depend on the chromosome, so for a tile of BN
// patterns the sum over c is a dense product D[p][m] = A[p][:] . PHI[m][:]
// with A = genes 1..K-1 (chromosomes on MMA-M = 128 TMEM lanes) and PHI the
// tile's expansion (patterns on MMA-N).
//
// Persistent CTAs, one per SM, each walking pattern tiles t = blockIdx.x +
// i * gridDim.x. Warp roles:
//   warp 0       A producer: bulk-copies 16 KB gene blocks (chromosome tile c,
//                K-block kb) from the pre-swizzled operand image into a
//                4-stage ring.
//   warp 1       MMA issuer (one thread) and tensor-memory owner; two FP32
//                accumulators of BN columns, so the epilogue of chromosome
//                tile c overlaps the MMAs of tile c+1.
//   warp 2       X producer: bulk-copies the next pattern tile's features.
//   warps 4-7    epilogue: tcgen05.ld of the accumulator (thread = chromosome,
//                TMEM lane), r = (y_m - a_0) - D, sse += r^2 over the tile's
//                patterns in FP32, then added into an FP64 per-CTA partial.
//   warps 8-11   expansion: the basis recurrences in registers from the
//                staged features, converted to BF16 and stored in the
//                K-major SWIZZLE_128B operand layout, one K-block (64
//                columns) at a time so the next tile's expansion overwrites a
//                K-block as soon as the last MMA reading it has completed.
// PHI and D never leave the SM. All waits are bounded (2 s): on expiry the
// kernel raises a status word, abandons its loops, waits for its own bulk
// copies and MMAs in flight, frees tensor memory and returns.
#include "basis.cuh"
#include "game_internal.cuh"
#include "tc_ptx.cuh"

namespace game {

namespace {

constexpr int kStages = 4;
constexpr uint32_t kABytes = 128 * 128;   // one (chromosome tile, K-block) gene block
constexpr int kWarps = 12;
constexpr int kThreads = kWarps * 32;
constexpr int kEpiThreads = 128;          // warps 4..7
constexpr int kBasisThreads = 128;        // warps 8..11
constexpr uint64_t kTimeoutNs = 2000000000ull;
constexpr int kMaxSmem = 232448;          // 227 KB opt-in per CTA
constexpr int kMinSmem = 120 * 1024;

struct TcArgs {
  int64_t M;
  int N, d, basis, Kp;
  int BN, KB, C, nmma_last, ntiles, Ppad, tmem_cols;
  const float* Xt;
  const float* y;
  const uint8_t* popA;
  const float* a0;
  double* part;
  int* status;
};

__host__ __device__ inline int phi_bytes(int KB, int BN) { return KB * BN * 128; }
__host__ __device__ inline int xs_bytes(int N, int BN) { return N * BN * 4; }
__host__ __device__ inline int num_bars(int KB) { return 2 * kStages + 2 * KB + 7; }
__host__ __device__ inline int smem_total(int KB, int BN, int N) {
  return 1024 + phi_bytes(KB, BN) + kStages * (int)kABytes + xs_bytes(N, BN) + 8 +
         num_bars(KB) * 8 + 16;
}

__device__ bool wait_bar(uint32_t bar, uint32_t parity, volatile int* abort_flag, int* status) {
  if (ptx::mbar_try_wait(bar, parity)) return true;
  const uint64_t t0 = ptx::global_timer_ns();
  for (uint32_t n = 0;; ++n) {
    if (ptx::mbar_try_wait(bar, parity)) return true;
    if ((n & 15) == 15) {
      if (*abort_flag) return false;
      if (ptx::global_timer_ns() - t0 > kTimeoutNs) {
        *abort_flag = 1;
        atomicExch(status, (int)kDevTimeout);
        return false;
      }
    }
  }
}

// Waits for this CTA's own asynchronous work (copies, MMAs) regardless of the
// abort flag, still bounded.
__device__ void wait_bar_drain(uint32_t bar, uint32_t parity, int* status) {
  const uint64_t t0 = ptx::global_timer_ns();
  while (!ptx::mbar_try_wait(bar, parity)) {
    if (ptx::global_timer_ns() - t0 > kTimeoutNs) {
      atomicExch(status, (int)kDevTimeout);
      return;
    }
  }
}

__global__ void __launch_bounds__(kThreads, 1) fitness_tc_kernel(const TcArgs a) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* base = reinterpret_cast<uint8_t*>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~static_cast<uintptr_t>(1023));
  const int BN = a.BN, KB = a.KB, N = a.N;
  uint8_t* phi = base;
  uint8_t* ast = phi + phi_bytes(KB, BN);
  float* xs = reinterpret_cast<float*>(ast + kStages * kABytes);
  uint64_t* bars = reinterpret_cast<uint64_t*>(
      (reinterpret_cast<uintptr_t>(xs + (size_t)N * BN) + 7) & ~static_cast<uintptr_t>(7));
  uint64_t* a_full = bars;
  uint64_t* a_empty = a_full + kStages;
  uint64_t* phi_full = a_empty + kStages;
  uint64_t* phi_free = phi_full + KB;
  uint64_t* acc_full = phi_free + KB;
  uint64_t* acc_empty = acc_full + 2;
  uint64_t* x_full = acc_empty + 2;
  uint64_t* x_empty = x_full + 1;
  uint64_t* drain = x_empty + 1;
  uint32_t* tmem_holder = reinterpret_cast<uint32_t*>(drain + 1);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_holder + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (int s = 0; s < kStages; ++s) {
      ptx::mbar_init(ptx::smem_addr(&a_full[s]), 1);
      ptx::mbar_init(ptx::smem_addr(&a_empty[s]), 1);
    }
    for (int kb = 0; kb < KB; ++kb) {
      ptx::mbar_init(ptx::smem_addr(&phi_full[kb]), kBasisThreads);
      ptx::mbar_init(ptx::smem_addr(&phi_free[kb]), 1);
    }
    for (int b = 0; b < 2; ++b) {
      ptx::mbar_init(ptx::smem_addr(&acc_full[b]), 1);
      ptx::mbar_init(ptx::smem_addr(&acc_empty[b]), kEpiThreads);
    }
    ptx::mbar_init(ptx::smem_addr(x_full), 1);
    ptx::mbar_init(ptx::smem_addr(x_empty), kBasisThreads);
    ptx::mbar_init(ptx::smem_addr(drain), 1);
    *abort_flag = 0;
    ptx::fence_mbar_init();
    ptx::fence_proxy_async_smem();
  }
  if (warp == 1) {
    ptx::tmem_alloc(ptx::smem_addr(tmem_holder), (uint32_t)a.tmem_cols);
    ptx::tmem_relinquish();
  }
  ptx::tc_fence_before();
  __syncthreads();
  ptx::tc_fence_after();
  const uint32_t tmem = *tmem_holder;

  const int G = gridDim.x;
  const int my_tiles = (a.ntiles - (int)blockIdx.x + G - 1) / G;
  const int XW = BN < 128 ? BN : 128;   // patterns per feature row in xs

  if (warp == 0) {
    // ---------------- A producer ----------------
    if (lane == 0) {
      uint32_t q = 0;
      bool ok = true;
      for (int it = 0; it < my_tiles && ok; ++it)
        for (int c = 0; c < a.C && ok; ++c)
          for (int kb = 0; kb < KB && ok; ++kb) {
            const uint32_t s = q % kStages, u = q / kStages;
            ok = wait_bar(ptx::smem_addr(&a_empty[s]), (u & 1) ^ 1, abort_flag, a.status);
            if (!ok) break;
            ptx::mbar_arrive_expect_tx(ptx::smem_addr(&a_full[s]), kABytes);
            ptx::bulk_g2s(ptx::smem_addr(ast + s * kABytes),
                          a.popA + (size_t)(c * KB + kb) * kABytes, kABytes,
                          ptx::smem_addr(&a_full[s]));
            ++q;
          }
      // own copies in flight: the last phase armed on each stage
      for (uint32_t s = 0; s < kStages && s < q; ++s) {
        const uint32_t uses = (q - s + kStages - 1) / kStages;
        wait_bar_drain(ptx::smem_addr(&a_full[s]), (uses - 1) & 1, a.status);
      }
    }
  } else if (warp == 1) {
    // ---------------- MMA issuer ----------------
    if (lane == 0) {
      const uint32_t idesc = ptx::idesc_bf16_f32(128, BN);
      const uint32_t phi_base = ptx::smem_addr(phi), ast_base = ptx::smem_addr(ast);
      uint32_t q = 0, acc_it = 0;
      bool ok = true;
      for (int it = 0; it < my_tiles && ok; ++it) {
        for (int c = 0; c < a.C && ok; ++c) {
          const uint32_t buf = acc_it & 1, u = acc_it >> 1;
          ok = wait_bar(ptx::smem_addr(&acc_empty[buf]), (u & 1) ^ 1, abort_flag, a.status);
          if (!ok) break;
          ptx::tc_fence_after();
          const uint32_t d_tmem = tmem + buf * (uint32_t)BN;
          for (int kb = 0; kb < KB; ++kb) {
            if (c == 0) {
              ok = wait_bar(ptx::smem_addr(&phi_full[kb]), it & 1, abort_flag, a.status);
              if (!ok) break;
              ptx::tc_fence_after();
            }
            const uint32_t s = q % kStages;
            ok = wait_bar(ptx::smem_addr(&a_full[s]), (q / kStages) & 1, abort_flag, a.status);
            if (!ok) break;
            ptx::tc_fence_after();
            const int nm = (kb == KB - 1) ? a.nmma_last : 4;
            for (int kk = 0; kk < nm; ++kk) {
              const uint64_t adesc = ptx::desc_kmajor_sw128(ast_base + s * kABytes + kk * 32);
              const uint64_t bdesc =
                  ptx::desc_kmajor_sw128(phi_base + (uint32_t)(kb * BN * 128) + kk * 32);
              ptx::mma_bf16(d_tmem, adesc, bdesc, idesc, (kb | kk) != 0);
            }
            ptx::mma_commit(ptx::smem_addr(&a_empty[s]));
            if (c == a.C - 1) ptx::mma_commit(ptx::smem_addr(&phi_free[kb]));
            ++q;
          }
          if (!ok) break;
          ptx::mma_commit(ptx::smem_addr(&acc_full[buf]));
          ++acc_it;
        }
      }
      // every MMA issued above has completed once this arrives
      ptx::mma_commit(ptx::smem_addr(drain));
      wait_bar_drain(ptx::smem_addr(drain), 0, a.status);
    }
  } else if (warp == 2) {
    // ---------------- X producer ----------------
    if (lane == 0) {
      int issued = 0;
      for (int it = 0; it < my_tiles; ++it) {
        const int64_t t = (int64_t)blockIdx.x + (int64_t)it * G;
        if (!wait_bar(ptx::smem_addr(x_empty), (it & 1) ^ 1, abort_flag, a.status)) break;
        const uint32_t bytes = (uint32_t)xs_bytes(N, BN);
        ptx::mbar_arrive_expect_tx(ptx::smem_addr(x_full), bytes);
        const int64_t m0 = t * BN;
        if (BN >= kPatBlock) {
          ptx::bulk_g2s(ptx::smem_addr(xs), a.Xt + m0 * N, bytes, ptx::smem_addr(x_full));
        } else {
          const int64_t blk = m0 / kPatBlock;
          const int off = (int)(m0 % kPatBlock);
          for (int i = 0; i < N; ++i)
            ptx::bulk_g2s(ptx::smem_addr(xs + i * BN),
                          a.Xt + (blk * N + i) * kPatBlock + off, (uint32_t)BN * 4,
                          ptx::smem_addr(x_full));
        }
        ++issued;
      }
      if (issued > 0) wait_bar_drain(ptx::smem_addr(x_full), (issued - 1) & 1, a.status);
    }
  } else if (warp >= 4 && warp < 8) {
    // ---------------- epilogue ----------------
    const int qw = warp & 3;
    const int row = qw * 32 + lane;
    const uint32_t lane_addr = (uint32_t)(qw * 32) << 16;
    double* part_row = a.part + (size_t)blockIdx.x * a.Ppad;
    uint32_t acc_it = 0;
    bool ok = true;
    for (int it = 0; it < my_tiles && ok; ++it) {
      const int64_t m0 = ((int64_t)blockIdx.x + (int64_t)it * G) * BN;
      const int64_t rem = a.M - m0;
      const int valid = rem <= 0 ? 0 : (rem >= BN ? BN : (int)rem);
      const float* yt = a.y + m0;
      for (int c = 0; c < a.C; ++c) {
        const uint32_t buf = acc_it & 1, u = acc_it >> 1;
        ok = wait_bar(ptx::smem_addr(&acc_full[buf]), u & 1, abort_flag, a.status);
        if (!ok) break;
        ptx::tc_fence_after();
        const int chrom = c * 128 + row;
        const float bias = a.a0[chrom];
        float s0 = 0.f, s1 = 0.f;
        for (int col0 = 0; col0 < valid; col0 += 32) {
          uint32_t v[32];
          ptx::tmem_ld32(tmem + lane_addr + buf * (uint32_t)BN + (uint32_t)col0, v);
          if (col0 + 32 <= valid) {
#pragma unroll
            for (int e4 = 0; e4 < 8; ++e4) {
              const float4 yv = __ldg(reinterpret_cast<const float4*>(yt + col0) + e4);
              const float r0 = (yv.x - bias) - __uint_as_float(v[4 * e4 + 0]);
              const float r1 = (yv.y - bias) - __uint_as_float(v[4 * e4 + 1]);
              const float r2 = (yv.z - bias) - __uint_as_float(v[4 * e4 + 2]);
              const float r3 = (yv.w - bias) - __uint_as_float(v[4 * e4 + 3]);
              s0 = fmaf(r0, r0, s0);
              s1 = fmaf(r1, r1, s1);
              s0 = fmaf(r2, r2, s0);
              s1 = fmaf(r3, r3, s1);
            }
          } else {
            const int lim = valid - col0;
#pragma unroll
            for (int e = 0; e < 32; ++e) {
              if (e < lim) {
                const float r = (yt[col0 + e] - bias) - __uint_as_float(v[e]);
                s0 = fmaf(r, r, s0);
              }
            }
          }
        }
        ptx::tc_fence_before();
        ptx::mbar_arrive(ptx::smem_addr(&acc_empty[buf]));
        const double tile_sse = (double)s0 + (double)s1;
        part_row[chrom] = (it == 0) ? tile_sse : part_row[chrom] + tile_sse;
        ++acc_it;
      }
    }
  } else if (warp >= 8) {
    // ---------------- expansion (basis) ----------------
    const int bt = threadIdx.x - 8 * 32;
    bool ok = true;
    for (int it = 0; it < my_tiles && ok; ++it) {
      ok = wait_bar(ptx::smem_addr(x_full), it & 1, abort_flag, a.status);
      if (!ok) break;
      for (int kb = 0; kb < KB; ++kb) {
        if (it > 0) {
          ok = wait_bar(ptx::smem_addr(&phi_free[kb]), (it - 1) & 1, abort_flag, a.status);
          if (!ok) break;
        }
        uint8_t* phik = phi + (size_t)kb * BN * 128;
        for (int task = bt; task < BN * 8; task += kBasisThreads) {
          const int r = task % BN, qd = task / BN;
          const float* xr = xs + (r >> 7) * N * XW + (r % XW);
          float v[8];
          basis_run<8>(a.basis, a.d, a.Kp, xr, XW, kb * 64 + qd * 8, v);
          uint32_t w[4];
#pragma unroll
          for (int h = 0; h < 4; ++h) {
            const __nv_bfloat162 b2 = __floats2bfloat162_rn(v[2 * h], v[2 * h + 1]);
            w[h] = *reinterpret_cast<const uint32_t*>(&b2);
          }
          *reinterpret_cast<uint4*>(phik + r * 128 + ((qd ^ (r & 7)) << 4)) =
              make_uint4(w[0], w[1], w[2], w[3]);
        }
        ptx::fence_proxy_async_smem();
        ptx::mbar_arrive(ptx::smem_addr(&phi_full[kb]));
      }
      if (!ok) break;
      ptx::mbar_arrive(ptx::smem_addr(x_empty));
    }
  }

  ptx::tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    ptx::tc_fence_after();
    ptx::tmem_dealloc(tmem, (uint32_t)a.tmem_cols);
  }
}

}  // namespace

TcPlan plan_tc(const Shape& s, int P, int num_sms) {
  TcPlan pl{};
  pl.KB = ceil_div(s.Kp, 64);
  pl.C = ceil_div(P, 128);
  pl.ok = false;
  const int cands[4] = {256, 128, 64, 32};
  for (int i = 0; i < 4; ++i) {
    const int BN = cands[i];
    const int sm = smem_total(pl.KB, BN, s.N);
    if (sm <= kMaxSmem) {
      pl.BN = BN;
      // at least half an SM's shared memory: one CTA per SM, so the tensor
      // memory allocation never waits on a co-resident CTA
      pl.smem_bytes = sm < kMinSmem ? kMinSmem : sm;
      pl.ok = true;
      break;
    }
  }
  if (!pl.ok) return pl;
  const int ntiles = (int)(s.Mpad / pl.BN);
  pl.grid = ntiles < num_sms ? ntiles : num_sms;
  int cols = 32;
  while (cols < 2 * pl.BN) cols <<= 1;
  pl.tmem_cols = cols;
  pl.rows = pl.grid;
  return pl;
}

cudaError_t launch_fitness_tc(const TcPlan& pl, const Shape& s, const float* Xt,
                              const float* y, const uint8_t* popA, const float* a0, int P,
                              int Ppad, double* part, int* status, cudaStream_t st) {
  (void)P;
  if (!pl.ok) return cudaErrorInvalidValue;
  TcArgs a;
  a.M = s.M;
  a.N = s.N;
  a.d = s.d;
  a.basis = s.basis;
  a.Kp = s.Kp;
  a.BN = pl.BN;
  a.KB = pl.KB;
  a.C = pl.C;
  const int last_cols = s.Kp - 64 * (pl.KB - 1);
  a.nmma_last = (last_cols + 15) / 16;
  a.ntiles = (int)(s.Mpad / pl.BN);
  a.Ppad = Ppad;
  a.tmem_cols = pl.tmem_cols;
  a.Xt = Xt;
  a.y = y;
  a.popA = popA;
  a.a0 = a0;
  a.part = part;
  a.status = status;
  cudaError_t e = cudaFuncSetAttribute(fitness_tc_kernel,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       pl.smem_bytes);
  if (e != cudaSuccess) return e;
  fitness_tc_kernel<<<pl.grid, kThreads, pl.smem_bytes, st>>>(a);
  return cudaGetLastError();
}

}  // namespace game
