// fitness_tc.cu -- fitness of a population with the contraction on the
// 5th-generation tensor cores (tcgen05, FP32 accumulation in tensor memory),
// the squared-error reduction fused into the epilogue.
//
// Operand forms (template parameter F):
//   BF16      genes and expansion rounded to BF16, one kind::f16 MMA per K=16.
//   bf16x3    split products: x = hi + lo with hi = bf16(x), lo = bf16(x - hi)
//             for both operands, and per K=16 step three MMAs into the same
//             accumulator, A_hi PHI_hi + A_hi PHI_lo + A_lo PHI_hi (the lo*lo
//             term, below 2^-16 of the product, is dropped).
//   FP8 E4M3  kind::f8f6f4, K = 32 per MMA, 128 columns per K-block. Column k
//             of the expansion is scaled by colinv_k = 448 / max_m |phi_k| into
//             E4M3's range; the genes carry colscale_k = 1 / colinv_k and a
//             per-chromosome factor 1 / u_p (u_p = max_k |a_pk colscale_k| / 448),
//             which the epilogue restores: Out = a_0 + u_p * D.
//
// Math (paper Section 3): Out_p(m) = a_{p,0} + sum_c a_{p,c+1} phi_c(x_m)
// (Eq. 2), fit_p = (1/M) sum_m (y_m - Out_p(m))^2 (Eq. 3, MSE). The
// expansion phi does not depend on the chromosome, so for a tile of BN
// patterns the sum over c is a dense product D[p][m] = A[p][:] . PHI[m][:]
// with A = genes 1..K-1 (chromosomes on MMA-M = 128 TMEM lanes) and PHI the
// tile's expansion (patterns on MMA-N).
//
// Persistent CTAs, one per SM, each walking pattern tiles t = blockIdx.x +
// i * gridDim.x. Warp roles (16 warps):
//   warp 0       A producer: bulk-copies 16 KB gene blocks (chromosome tile c,
//                K-block kb of 64 columns) from the pre-swizzled operand
//                image into a ring of 3-4 stages.
//   warp 1       MMA issuer (one thread) and tensor-memory owner; two FP32
//                accumulators of BN columns, so the epilogue of chromosome
//                tile c overlaps the MMAs of tile c+1. The tcgen05 queue
//                drains fast, so the issuing path is kept minimal: precomputed
//                descriptors, unrolled groups of four K=16 MMAs, K-blocks taken
//                in pairs (singly for the first chromosome tile of a pattern
//                tile, so that its MMAs start as soon as one slot is full).
//   warp 2       X producer: bulk-copies the next pattern tile's features
//                (staged mode only, below).
//   warps 4-11   epilogue: tcgen05.ld of the accumulator (thread = chromosome
//                = TMEM lane; warps 4-7 take the first half of the columns,
//                8-11 the second), r = (y_m - a_0) - D, sse += r^2 in packed
//                FP32 pairs, then added to an FP64 partial per (CTA, half).
//   warps 12-15  expansion: each thread owns fixed pattern rows; per 8-column
//                chunk (a table built once per launch says where the chunk
//                starts in the feature / degree sequence) the basis
//                recurrence runs in registers, is rounded to BF16 and stored
//                in the K-major SWIZZLE_128B operand layout.
// Expansion slots: the K-blocks of the tiles go, in order, into a ring of NS
// K-block slots (use q = i * KB + kb takes slot q % NS); a slot is rewritten
// as soon as the last MMA reading its previous use has completed. With
// NS = KB this is one buffer per K-block; spare slots (NS > KB) let the next
// tile's first K-blocks be written while this tile's MMAs still run.
// Features: staged (the X producer bulk-copies the tile's feature blocks
// into shared memory, the expansion reads them there) or, for the BF16 form
// with Chebyshev runs of 8 degrees at 128 / 256 patterns, read by the
// expansion threads from global memory (L2, prefetched two tiles ahead),
// one K-block ahead of use; the shared memory this frees holds the spare
// slots. Both modes produce identical expansion values.
// PHI and D never leave the SM. All waits are bounded (2 s): on expiry the
// kernel raises a status word, abandons its loops, waits for its own bulk
// copies and MMAs in flight, frees tensor memory and returns.
#include <cuda_fp8.h>

#include <atomic>

#include "basis.cuh"
#include "game_internal.cuh"
#include "tc_common.cuh"
#include "tc_ptx.cuh"


namespace game {

namespace {

using namespace tc;

constexpr uint32_t kABytes = 128 * 128;   // one (chromosome tile, K-block) gene block
constexpr int kWarps = 16;
constexpr int kThreads = kWarps * 32;
constexpr int kEpiWarp0 = 4;
constexpr int kEpiThreads = 256;          // warps 4..11
constexpr int kBasisWarp0 = 12;
constexpr int kBasisThreads = 128;        // warps 12..15
constexpr int kMaxSmem = 232448;          // 227 KB opt-in per CTA
constexpr int kMinSmem = 120 * 1024;

struct TcArgs {
  int64_t M;
  int N, d, basis, Kp;
  int BN, KB, C, stages, nmma_last, ntiles, Ppad, tmem_cols;
  int NS;       // expansion K-block slots (KB .. 2 KB): slots beyond KB let the
                // next tile's first K-blocks be written while this tile's MMAs run
  int xstage;   // 1: the tile's features are bulk-copied into shared memory;
                // 0: read from global memory (L2) by the expansion warps
  int ystage;   // 1 (with xstage 0): warp 2 bulk-copies each tile's targets into
                // a two-slot shared buffer the epilogue reads
  int slack;    // bytes reserved for aligning the dynamic shared memory to 1024
  const float* Xt;
  const float* y;
  const uint8_t* popA;
  const float* a0;
  const float* uscale;   // FP8 only
  const float* colinv;   // FP8 only, [KB * 128]
  double* part;
  int* status;
  uint64_t stall_ns;   // test hook: > 0 makes the MMA issuer first wait this long on a
                       // barrier phase that nothing completes, then abandon the launch
};

struct SmemPlan {
  int phi, ast, xs, ys, cs, tab, bars, total;
};

__host__ __device__ inline int num_bars(int NS, int stages) { return 2 * stages + 2 * NS + 11; }

// Byte offsets of the shared-memory regions from the 1024-aligned base;
// total includes `slack` bytes for aligning the base.
__host__ __device__ inline SmemPlan smem_plan(int KB, int NS, int BN, int N, int stages, int F,
                                              int xstage, int ystage, int slack) {
  SmemPlan s;
  s.phi = 0;
  s.ast = s.phi + NS * form_nphi(F) * BN * 128;
  s.xs = s.ast + stages * form_na(F) * (int)kABytes;
  s.ys = s.xs + (xstage ? N * BN * 4 : 0);
  s.cs = s.ys + (ystage ? 2 * BN * 4 : 0);
  s.tab = s.cs + (F == kFormFP8 ? KB * 128 * 4 : 0);
  s.bars = (s.tab + KB * (form_cols(F) / 8) * 4 + 7) & ~7;
  s.total = s.bars + num_bars(NS, stages) * 8 + 16 + slack;
  return s;
}

// TRI: the 192-pattern tile (three expansion rows per thread), instantiated
// for the BF16 form only, so the 128- and 256-pattern code stays lean.
// ABS: the epilogue sums absolute residuals (MAE) instead of squared ones.
template <int F, bool TRI, bool ABS>
__global__ void __launch_bounds__(kThreads, 1) fitness_tc_kernel(const TcArgs a) {
  constexpr int NA = form_na(F), NPHI = form_nphi(F), CPK = form_cols(F) / 8;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* base = reinterpret_cast<uint8_t*>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~static_cast<uintptr_t>(1023));
  const int BN = a.BN, KB = a.KB, N = a.N, S = a.stages, NS = a.NS;
  // the plan reserves a.slack bytes for aligning the base: a base that needs
  // more (the host plans from a probe of where dynamic shared memory starts)
  // ends the launch before any shared memory is touched
  const uint32_t pad = (1024u - (ptx::smem_addr(smem_raw) & 1023u)) & 1023u;
  if (pad > (uint32_t)a.slack) {
    if (threadIdx.x == 0) atomicExch(a.status, (int)kDevSmemBase);
    return;
  }
  const SmemPlan sp = smem_plan(KB, NS, BN, N, S, F, a.xstage, a.ystage, a.slack);
  uint8_t* phi = base + sp.phi;
  uint8_t* ast = base + sp.ast;
  float* xs = reinterpret_cast<float*>(base + sp.xs);
  float* ys = reinterpret_cast<float*>(base + sp.ys);
  float* cs = reinterpret_cast<float*>(base + sp.cs);
  uint32_t* tab = reinterpret_cast<uint32_t*>(base + sp.tab);
  uint64_t* bars = reinterpret_cast<uint64_t*>(base + sp.bars);
  uint64_t* a_full = bars;
  uint64_t* a_empty = a_full + S;
  uint64_t* phi_full = a_empty + S;
  uint64_t* phi_free = phi_full + NS;
  uint64_t* acc_full = phi_free + NS;
  uint64_t* acc_empty = acc_full + 2;
  uint64_t* x_full = acc_empty + 2;
  uint64_t* x_empty = x_full + 1;
  uint64_t* drain = x_empty + 1;
  uint64_t* y_full = drain + 1;   // [2]
  uint64_t* y_empty = y_full + 2;  // [2]
  uint32_t* tmem_holder = reinterpret_cast<uint32_t*>(y_empty + 2);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_holder + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (int s = 0; s < S; ++s) {
      ptx::mbar_init(ptx::smem_addr(&a_full[s]), 1);
      ptx::mbar_init(ptx::smem_addr(&a_empty[s]), 1);
    }
    for (int sl = 0; sl < NS; ++sl) {
      ptx::mbar_init(ptx::smem_addr(&phi_full[sl]), kBasisThreads);
      ptx::mbar_init(ptx::smem_addr(&phi_free[sl]), 1);
    }
    for (int b = 0; b < 2; ++b) {
      ptx::mbar_init(ptx::smem_addr(&acc_full[b]), 1);
      ptx::mbar_init(ptx::smem_addr(&acc_empty[b]), kEpiThreads);
    }
    ptx::mbar_init(ptx::smem_addr(x_full), 1);
    ptx::mbar_init(ptx::smem_addr(x_empty), kBasisThreads);
    ptx::mbar_init(ptx::smem_addr(drain), 1);
    for (int b = 0; b < 2; ++b) {
      ptx::mbar_init(ptx::smem_addr(&y_full[b]), 1);
      ptx::mbar_init(ptx::smem_addr(&y_empty[b]), kEpiThreads);
    }
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
  // xs holds the tile's features as 128-pattern blocks [BN/128][N][128] when BN
  // is a multiple of 128, else as one block [N][BN]
  const bool xblocks = BN % 128 == 0;
  const int XW = xblocks ? 128 : BN;    // patterns per feature row in xs

  if (warp == 0) {
    // ---------------- A producer ----------------
    if (lane == 0) {
      uint32_t q = 0, s = 0, ph = 0;   // issue count, stage, stage phase
      bool ok = true;
      for (int it = 0; it < my_tiles && ok; ++it)
        for (int c = 0; c < a.C && ok; ++c)
          for (int kb = 0; kb < KB && ok; ++kb) {
            ok = wait_bar(ptx::smem_addr(&a_empty[s]), ph ^ 1, abort_flag, a.status);
            if (!ok) break;
            ptx::mbar_arrive_expect_tx(ptx::smem_addr(&a_full[s]), NA * kABytes);
            ptx::bulk_g2s(ptx::smem_addr(ast + s * NA * kABytes),
                          a.popA + (size_t)(c * KB + kb) * NA * kABytes, NA * kABytes,
                          ptx::smem_addr(&a_full[s]));
            ++q;
            if (++s == (uint32_t)S) {
              s = 0;
              ph ^= 1;
            }
          }
      // own copies in flight: the last phase armed on each stage
      for (uint32_t st = 0; st < (uint32_t)S && st < q; ++st) {
        const uint32_t uses = (q - st + S - 1) / S;
        wait_bar_drain(ptx::smem_addr(&a_full[st]), (uses - 1) & 1, a.status);
      }
    }
  } else if (warp == 1) {
    // ---------------- MMA issuer ----------------
    // The tcgen05 MMA queue drains quickly, so this thread's path between
    // MMAs is kept short: descriptors are precomputed (a stage, a K-block or
    // a K=16 step only moves the 14-bit start-address field), K-blocks are
    // taken in pairs (both operand waits first, then up to eight MMAs back
    // to back, then the commits), and the inner groups are unrolled.
    if (lane == 0) {
      const uint32_t idesc =
          F == kFormFP8 ? ptx::idesc_e4m3_f32(128, BN) : ptx::idesc_bf16_f32(128, BN);
      const uint64_t adesc0 = ptx::desc_kmajor_sw128(ptx::smem_addr(ast));
      const uint64_t bdesc0 = ptx::desc_kmajor_sw128(ptx::smem_addr(phi));
      const uint32_t a_step = (uint32_t)(NA * kABytes) >> 4;       // one A stage
      const uint32_t b_step = (uint32_t)(NPHI * BN * 128) >> 4;    // one expansion K-block
      const uint32_t a_lo = kABytes >> 4;                          // bf16x3: lo gene block
      const uint32_t b_lo = (uint32_t)(BN * 128) >> 4;             // bf16x3: lo expansion
      const uint32_t a_full0 = ptx::smem_addr(a_full), a_empty0 = ptx::smem_addr(a_empty);
      const uint32_t phi_full0 = ptx::smem_addr(phi_full), phi_free0 = ptx::smem_addr(phi_free);
      const uint32_t acc_full0 = ptx::smem_addr(acc_full), acc_empty0 = ptx::smem_addr(acc_empty);
      const int nlast = a.nmma_last;
      uint32_t s = 0, ph = 0, acc_it = 0;   // A stage and its phase, accumulator count
      bool ok = true;
      if (a.stall_ns) {
        // test hook: the drain barrier's first phase completes only at the
        // final commit below, so this wait runs out; the launch is then
        // abandoned as on any expired wait (status word, abort flag)
        const uint64_t t0 = ptx::global_timer_ns();
        while (ok && !ptx::mbar_try_wait_sleep(ptx::smem_addr(drain), 0, kSuspendNs)) {
          if (ptx::global_timer_ns() - t0 > a.stall_ns) {
            *abort_flag = 1;
            atomicExch(a.status, (int)kDevTimeout);
            ok = false;
          }
        }
      }
      // one K step (32 bytes of each operand row): one MMA, three for bf16x3
      auto kstep = [&](uint32_t d_tmem, uint64_t ad, uint64_t bd, uint32_t acc) {
        if (F == kFormFP8) {
          ptx::mma_f8(d_tmem, ad, bd, idesc, acc);
        } else {
          ptx::mma_bf16(d_tmem, ad, bd, idesc, acc);
          if (F == kFormBF16x3) {
            ptx::mma_bf16(d_tmem, ad, bd + b_lo, idesc, 1u);
            ptx::mma_bf16(d_tmem, ad + a_lo, bd, idesc, 1u);
          }
        }
      };
      // issues the MMAs of one K-block (nm of 4 K steps)
      auto kblock = [&](uint32_t d_tmem, uint32_t st, int kb, int slot, int nm) {
        const uint64_t ad = adesc0 + st * a_step;
        const uint64_t bd = bdesc0 + (uint32_t)slot * b_step;
        if (nm == 4) {
          kstep(d_tmem, ad, bd, kb != 0);
          kstep(d_tmem, ad + 2u, bd + 2u, 1u);
          kstep(d_tmem, ad + 4u, bd + 4u, 1u);
          kstep(d_tmem, ad + 6u, bd + 6u, 1u);
        } else {
          for (int kk = 0; kk < nm; ++kk)
            kstep(d_tmem, ad + 2u * kk, bd + 2u * kk, (kb | kk) != 0);
        }
      };
      for (int it = 0; it < my_tiles && ok; ++it) {
        for (int c = 0; c < a.C && ok; ++c) {
          const uint32_t buf = acc_it & 1, u = acc_it >> 1;
          ok = wait_bar(acc_empty0 + 8 * buf, (u & 1) ^ 1, abort_flag, a.status);
          if (!ok) break;
          ptx::tc_fence_after();
          const uint32_t d_tmem = tmem + buf * (uint32_t)BN;
          // the first chromosome tile of a pattern tile takes K-blocks one at a
          // time, so its MMAs start as soon as the first expansion slot is full
          for (int kb = 0; kb < KB && ok; kb += (c != 0 && kb + 1 < KB) ? 2 : 1) {
            const bool two = c != 0 && kb + 1 < KB;
            uint32_t s1 = s + 1, ph1 = ph;
            if (s1 == (uint32_t)S) {
              s1 = 0;
              ph1 ^= 1;
            }
            // expansion slots of the two K-blocks: use q = it KB + kb of slot q % NS
            const int q0 = it * KB + kb, q1 = q0 + 1;
            const int sl0 = q0 % NS, sl1 = q1 % NS;
            // operands of both K-blocks first
            if (c == 0) {
              ok = wait_bar(phi_full0 + 8 * sl0, (q0 / NS) & 1, abort_flag, a.status);
              if (ok && two)
                ok = wait_bar(phi_full0 + 8 * sl1, (q1 / NS) & 1, abort_flag, a.status);
            }
            if (ok) ok = wait_bar(a_full0 + 8 * s, ph, abort_flag, a.status);
            if (ok && two) ok = wait_bar(a_full0 + 8 * s1, ph1, abort_flag, a.status);
            if (!ok) break;
            kblock(d_tmem, s, kb, sl0, (kb == KB - 1) ? nlast : 4);
            if (two) kblock(d_tmem, s1, kb + 1, sl1, (kb + 1 == KB - 1) ? nlast : 4);
            ptx::mma_commit(a_empty0 + 8 * s);
            if (two) ptx::mma_commit(a_empty0 + 8 * s1);
            if (c == a.C - 1) {
              ptx::mma_commit(phi_free0 + 8 * sl0);
              if (two) ptx::mma_commit(phi_free0 + 8 * sl1);
            }
            s = s1;
            ph = ph1;
            if (two) {
              if (++s == (uint32_t)S) {
                s = 0;
                ph ^= 1;
              }
            }
          }
          if (!ok) break;
          ptx::mma_commit(acc_full0 + 8 * buf);
          ++acc_it;
        }
      }
      // every MMA issued above has completed once this arrives
      ptx::mma_commit(ptx::smem_addr(drain));
      wait_bar_drain(ptx::smem_addr(drain), 0, a.status);
    }
  } else if (warp == 2) {
    // ---------------- X producer (staged features only) ----------------
    if (lane == 0 && a.xstage) {
      int issued = 0;
      for (int it = 0; it < my_tiles; ++it) {
        const int64_t t = (int64_t)blockIdx.x + (int64_t)it * G;
        if (!wait_bar(ptx::smem_addr(x_empty), (it & 1) ^ 1, abort_flag, a.status)) break;
        const uint32_t bytes = (uint32_t)(N * BN * 4);
        ptx::mbar_arrive_expect_tx(ptx::smem_addr(x_full), bytes);
        const int64_t m0 = t * BN;
        if (xblocks) {
          ptx::bulk_g2s(ptx::smem_addr(xs), a.Xt + m0 * N, bytes, ptx::smem_addr(x_full));
        } else {
          // per feature, the tile's run of patterns, in pieces that stay inside
          // one 128-pattern block (starts and lengths are multiples of 32
          // patterns, so every piece is 16-byte aligned)
          for (int i = 0; i < N; ++i) {
            int64_t m = m0;
            int done = 0;
            while (done < BN) {
              const int off = (int)(m % kPatBlock);
              const int seg = (kPatBlock - off) < (BN - done) ? (kPatBlock - off) : (BN - done);
              ptx::bulk_g2s(ptx::smem_addr(xs + i * BN + done),
                            a.Xt + ((m / kPatBlock) * N + i) * kPatBlock + off,
                            (uint32_t)seg * 4, ptx::smem_addr(x_full));
              done += seg;
              m += seg;
            }
          }
        }
        // the next tile's feature blocks into L2, so its copy (issued once the
        // expansion has released this one) reads L2 instead of HBM
        if (it + 1 < my_tiles) {
          const int64_t m1 = (t + G) * BN;
          const int64_t b0 = m1 / kPatBlock, b1 = (m1 + BN - 1) / kPatBlock;
          ptx::bulk_prefetch_l2(a.Xt + b0 * N * kPatBlock,
                                (uint32_t)((b1 - b0 + 1) * N * kPatBlock * 4));
        }
        ++issued;
      }
      if (issued > 0) wait_bar_drain(ptx::smem_addr(x_full), (issued - 1) & 1, a.status);
    }
    // ---------------- Y producer (features read from L2) ----------------
    // each tile's targets into slot it & 1, released by the 256 epilogue
    // threads after the tile's last chromosome tile
    if (lane == 0 && a.ystage) {
      int issued = 0;
      for (int it = 0; it < my_tiles; ++it) {
        const int b = it & 1;
        if (!wait_bar(ptx::smem_addr(&y_empty[b]), ((it >> 1) & 1) ^ 1, abort_flag, a.status))
          break;
        const int64_t m0 = ((int64_t)blockIdx.x + (int64_t)it * G) * BN;
        ptx::mbar_arrive_expect_tx(ptx::smem_addr(&y_full[b]), (uint32_t)BN * 4);
        ptx::bulk_g2s(ptx::smem_addr(ys + b * BN), a.y + m0, (uint32_t)BN * 4,
                      ptx::smem_addr(&y_full[b]));
        ++issued;
      }
      // own copies in flight: the last phase armed on each slot
      for (int b = 0; b < 2 && b < issued; ++b) {
        const int uses = (issued - b + 1) / 2;
        wait_bar_drain(ptx::smem_addr(&y_full[b]), (uint32_t)(uses - 1) & 1u, a.status);
      }
    }
  } else if (warp >= kEpiWarp0 && warp < kBasisWarp0) {
    // ---------------- epilogue ----------------
    const int qw = warp & 3;
    const int half = (warp - kEpiWarp0) >> 2;
    const int row = qw * 32 + lane;
    const int NH = BN >= 64 ? 2 : 1;          // column halves in use
    const int HW = BN / NH;                   // columns per half (>= 32)
    const int col_lo = half * HW;
    const uint32_t lane_addr = (uint32_t)(qw * 32) << 16;
    double* part_row = a.part + (size_t)(2 * blockIdx.x + half) * a.Ppad;
    uint32_t acc_it = 0;
    bool ok = true;
    for (int it = 0; it < my_tiles && ok; ++it) {
      const int64_t m0 = ((int64_t)blockIdx.x + (int64_t)it * G) * BN;
      const int64_t rem = a.M - m0 - col_lo;
      const int valid = (half >= NH || rem <= 0) ? 0 : (rem >= HW ? HW : (int)rem);
      const bool ysm = a.ystage != 0;
      if (ysm) {
        ok = wait_bar(ptx::smem_addr(&y_full[it & 1]), (it >> 1) & 1, abort_flag, a.status);
        if (!ok) break;
      }
      const float* yt = ysm ? ys + (it & 1) * BN + col_lo : a.y + m0 + col_lo;
      for (int c = 0; c < a.C; ++c) {
        const uint32_t buf = acc_it & 1, u = acc_it >> 1;
        ok = wait_bar(ptx::smem_addr(&acc_full[buf]), u & 1, abort_flag, a.status);
        if (!ok) break;
        ptx::tc_fence_after();
        const int chrom = c * 128 + row;
        const float bias = a.a0[chrom];
        const uint64_t bias2 = ptx::f2_pack(bias, bias);
        const float negu = F == kFormFP8 ? -a.uscale[chrom] : -1.f;
        const uint64_t negu2 = ptx::f2_pack(negu, negu);
        uint64_t s2 = 0;   // two FP32 partial sums (even / odd columns)
        float s_tail = 0.f;
        const uint32_t tbase = tmem + lane_addr + buf * (uint32_t)BN + (uint32_t)col_lo;
        const int nfull = valid / 32;
        if (nfull > 0) {
          // double-buffered: the load of chunk k+1 is in flight while chunk k
          // is reduced
          uint32_t va[32], vb[32];
          ptx::tmem_ld32_issue(tbase, va);
          ptx::tmem_ld32_wait(va);
          for (int k = 0; k < nfull; k += 2) {
            const bool has_b = k + 1 < nfull;
            if (has_b) ptx::tmem_ld32_issue(tbase + (uint32_t)(k + 1) * 32, vb);
            if (ysm) epi_chunk<F == kFormFP8, ABS, true>(va, yt + k * 32, bias2, negu2, s2);
            else epi_chunk<F == kFormFP8, ABS>(va, yt + k * 32, bias2, negu2, s2);
            if (has_b) {
              ptx::tmem_ld32_wait(vb);
              const bool has_a = k + 2 < nfull;
              if (has_a) ptx::tmem_ld32_issue(tbase + (uint32_t)(k + 2) * 32, va);
              if (ysm) epi_chunk<F == kFormFP8, ABS, true>(vb, yt + (k + 1) * 32, bias2, negu2, s2);
              else epi_chunk<F == kFormFP8, ABS>(vb, yt + (k + 1) * 32, bias2, negu2, s2);
              if (has_a) ptx::tmem_ld32_wait(va);
            }
          }
        }
        if (nfull * 32 < valid) {   // ragged last chunk of the last tile
          uint32_t v[32];
          ptx::tmem_ld32(tbase + (uint32_t)nfull * 32, v);
          const int lim = valid - nfull * 32;
#pragma unroll
          for (int e = 0; e < 32; ++e) {
            if (e < lim) {
              const float r = fmaf(negu, __uint_as_float(v[e]), yt[nfull * 32 + e] - bias);
              s_tail = ABS ? s_tail + fabsf(r) : fmaf(r, r, s_tail);
            }
          }
        }
        ptx::tc_fence_before();
        ptx::mbar_arrive(ptx::smem_addr(&acc_empty[buf]));
        const float2 sp2 = ptx::f2_unpack(s2);
        const double tile_sse = (double)sp2.x + (double)sp2.y + (double)s_tail;
        part_row[chrom] = (it == 0) ? tile_sse : part_row[chrom] + tile_sse;
        ++acc_it;
      }
      if (ysm && ok) ptx::mbar_arrive(ptx::smem_addr(&y_empty[it & 1]));
    }
  } else if (warp >= kBasisWarp0) {
    // ---------------- expansion (basis) ----------------
    const int bt = threadIdx.x - kBasisWarp0 * 32;
    for (int cid = bt; cid < KB * CPK; cid += kBasisThreads)
      tab[cid] = chunk_desc(cid, a.basis, a.d, a.Kp);
    if (F == kFormFP8)
      for (int k = bt; k < KB * 128; k += kBasisThreads) cs[k] = a.colinv[k];
    ptx::named_bar(1, kBasisThreads);
    // thread -> rows r0 + RW * rr (rr < R) and 16-byte units q0, q0 + QS, ...:
    // BN = 128, 256: 128 rows per pass, R = BN / 128; BN = 192: 64 rows per
    // pass, R = 3, two unit groups; BN < 128: BN rows, R = 1, 128 / BN groups
    const int RW = TRI ? 64 : (BN < 128 ? BN : 128);
    const int R = TRI ? 3 : BN / RW;
    const int QS = 128 / RW;
    const int r0 = bt % RW, q0 = bt / RW;
    auto xrow_of = [&](int r) -> const float* {
      return xblocks ? xs + (r >> 7) * N * 128 + (r & 127) : xs + r;
    };
    const bool cheb = a.basis == GAME_BASIS_CHEB;
    // the 8 values of one chunk for row rA (va) and, when hasB, row rB (vb).
    // A Chebyshev chunk inside one feature's run of degrees (the common case:
    // degree 8) takes two interleaved recurrences and one descriptor decode,
    // with no per-value branches.
    auto gen_rows = [&](uint32_t desc, const float* xrow0, const float* xrow1, bool hasB,
                        float (&va)[8], float (&vb)[8]) {
      if (cheb && (desc & kChunkRun) && ((desc >> 24) & 15u) == 8u) {
        const int i = (int)(desc & 0xFFFFu);
        const int j0 = (int)((desc >> 16) & 31u);
        const float xa = xrow0[i * XW];
        const float xb = hasB ? xrow1[i * XW] : 0.f;
        const float a2 = xa + xa, b2 = xb + xb;
        float ta = xa, tam = 1.f, tb = xb, tbm = 1.f;
        for (int st = 1; st < j0; ++st) {
          const float na = fmaf(a2, ta, -tam), nb = fmaf(b2, tb, -tbm);
          tam = ta;
          ta = na;
          tbm = tb;
          tb = nb;
        }
        va[0] = ta;
        vb[0] = tb;
#pragma unroll
        for (int e = 1; e < 8; ++e) {
          const float na = fmaf(a2, ta, -tam), nb = fmaf(b2, tb, -tbm);
          tam = ta;
          ta = na;
          tbm = tb;
          tb = nb;
          va[e] = ta;
          vb[e] = tb;
        }
      } else if (cheb && a.d >= 4 && !(desc & kChunkZero)) {
        if (hasB) cheb_cross2(desc, a.d, N, xrow0, xrow1, XW, true, va, vb);
        else cheb_cross1(desc, a.d, N, xrow0, XW, va);
      } else {
        gen_chunk(desc, a.basis, a.d, N, xrow0, XW, va);
        if (hasB) gen_chunk(desc, a.basis, a.d, N, xrow1, XW, vb);
      }
    };
    auto store16 = [&](uint8_t* img, int r, int qd, uint32_t w0, uint32_t w1, uint32_t w2,
                       uint32_t w3) {
      *reinterpret_cast<uint4*>(img + r * 128 + ((qd ^ (r & 7)) << 4)) =
          make_uint4(w0, w1, w2, w3);
    };
    // one 16-byte unit qd of K-block kb for rows rA and (when hasB) rB
    auto emit_pair = [&](uint8_t* phik, int kb, int qd, int rA, const float* xa, int rB,
                         const float* xb, bool hasB) {
      float va[8], vb[8];
      if (F == kFormFP8) {
        // 16 columns: chunks 2 qd and 2 qd + 1, scaled into E4M3's range
        float vc[8], vd[8];
        gen_rows(tab[kb * CPK + 2 * qd], xa, xb, hasB, va, vb);
        gen_rows(tab[kb * CPK + 2 * qd + 1], xa, xb, hasB, vc, vd);
        const float* sc = cs + kb * 128 + qd * 16;
        float s16[16];
#pragma unroll
        for (int e = 0; e < 16; ++e) s16[e] = sc[e];
        store16(phik, rA, qd, e4m3x4_bits(va[0] * s16[0], va[1] * s16[1], va[2] * s16[2], va[3] * s16[3]),
                e4m3x4_bits(va[4] * s16[4], va[5] * s16[5], va[6] * s16[6], va[7] * s16[7]),
                e4m3x4_bits(vc[0] * s16[8], vc[1] * s16[9], vc[2] * s16[10], vc[3] * s16[11]),
                e4m3x4_bits(vc[4] * s16[12], vc[5] * s16[13], vc[6] * s16[14], vc[7] * s16[15]));
        if (hasB)
          store16(phik, rB, qd,
                  e4m3x4_bits(vb[0] * s16[0], vb[1] * s16[1], vb[2] * s16[2], vb[3] * s16[3]),
                  e4m3x4_bits(vb[4] * s16[4], vb[5] * s16[5], vb[6] * s16[6], vb[7] * s16[7]),
                  e4m3x4_bits(vd[0] * s16[8], vd[1] * s16[9], vd[2] * s16[10], vd[3] * s16[11]),
                  e4m3x4_bits(vd[4] * s16[12], vd[5] * s16[13], vd[6] * s16[14], vd[7] * s16[15]));
      } else {
        gen_rows(tab[kb * CPK + qd], xa, xb, hasB, va, vb);
        if (F == kFormBF16) {
          store16(phik, rA, qd, bf16x2_bits(va[0], va[1]), bf16x2_bits(va[2], va[3]),
                  bf16x2_bits(va[4], va[5]), bf16x2_bits(va[6], va[7]));
          if (hasB)
            store16(phik, rB, qd, bf16x2_bits(vb[0], vb[1]), bf16x2_bits(vb[2], vb[3]),
                    bf16x2_bits(vb[4], vb[5]), bf16x2_bits(vb[6], vb[7]));
        } else {
          uint8_t* phik_lo = phik + BN * 128;
          uint32_t h[4], l[4];
#pragma unroll
          for (int e = 0; e < 4; ++e) split_bf16x2(va[2 * e], va[2 * e + 1], h[e], l[e]);
          store16(phik, rA, qd, h[0], h[1], h[2], h[3]);
          store16(phik_lo, rA, qd, l[0], l[1], l[2], l[3]);
          if (hasB) {
#pragma unroll
            for (int e = 0; e < 4; ++e) split_bf16x2(vb[2 * e], vb[2 * e + 1], h[e], l[e]);
            store16(phik, rB, qd, h[0], h[1], h[2], h[3]);
            store16(phik_lo, rB, qd, l[0], l[1], l[2], l[3]);
          }
        }
      }
    };
    // the thread's rows (feature pointers fixed for the launch), in pairs
    const int r1 = r0 + RW, r2 = r0 + 2 * RW;
    const float* xr0 = xrow_of(r0);
    const float* xr1 = R >= 2 ? xrow_of(r1) : xr0;
    const float* xr2 = R == 3 ? xrow_of(r2) : xr0;
    auto emit_unit = [&](uint8_t* phik, int kb, int qd) {
      emit_pair(phik, kb, qd, r0, xr0, r1, xr1, R >= 2);
      if (TRI) emit_pair(phik, kb, qd, r2, xr2, r2, xr2, false);
    };
    // The BF16 form at 128 / 256 patterns (the main workloads) stores each row
    // as it is generated: measured 3% faster for the whole kernel than the
    // generic pair path above (fewer values live between the recurrences
    // and the stores).
    auto emit = [&](uint8_t* phik, uint32_t desc, int qd, int r, const float* xr) {
      float v[8];
      gen_chunk(desc, a.basis, a.d, N, xr, XW, v);
      uint32_t w[4];
#pragma unroll
      for (int h = 0; h < 4; ++h) {
        const __nv_bfloat162 b2 = __floats2bfloat162_rn(v[2 * h], v[2 * h + 1]);
        w[h] = *reinterpret_cast<const uint32_t*>(&b2);
      }
      *reinterpret_cast<uint4*>(phik + r * 128 + ((qd ^ (r & 7)) << 4)) =
          make_uint4(w[0], w[1], w[2], w[3]);
    };
    // both rows of a Chebyshev chunk that stays in one feature's run of
    // degrees (the common case: degree 8): two interleaved recurrences, one
    // descriptor decode, no per-value branches
    auto emit_run2x = [&](uint8_t* phik, uint32_t desc, int qd, float xa, float xb) {
      const int j0 = (int)((desc >> 16) & 31u);
      const float a2 = xa + xa, b2 = xb + xb;
      float ta = xa, tam = 1.f, tb = xb, tbm = 1.f;
      for (int st = 1; st < j0; ++st) {
        const float na = fmaf(a2, ta, -tam), nb = fmaf(b2, tb, -tbm);
        tam = ta;
        ta = na;
        tbm = tb;
        tb = nb;
      }
      float va[8], vb[8];
      va[0] = ta;
      vb[0] = tb;
#pragma unroll
      for (int e = 1; e < 8; ++e) {
        const float na = fmaf(a2, ta, -tam), nb = fmaf(b2, tb, -tbm);
        tam = ta;
        ta = na;
        tbm = tb;
        tb = nb;
        va[e] = ta;
        vb[e] = tb;
      }
      uint32_t wa[4], wb[4];
#pragma unroll
      for (int h = 0; h < 4; ++h) {
        const __nv_bfloat162 pa = __floats2bfloat162_rn(va[2 * h], va[2 * h + 1]);
        const __nv_bfloat162 pb = __floats2bfloat162_rn(vb[2 * h], vb[2 * h + 1]);
        wa[h] = *reinterpret_cast<const uint32_t*>(&pa);
        wb[h] = *reinterpret_cast<const uint32_t*>(&pb);
      }
      *reinterpret_cast<uint4*>(phik + r0 * 128 + ((qd ^ (r0 & 7)) << 4)) =
          make_uint4(wa[0], wa[1], wa[2], wa[3]);
      if (R == 2)
        *reinterpret_cast<uint4*>(phik + r1 * 128 + ((qd ^ (r1 & 7)) << 4)) =
            make_uint4(wb[0], wb[1], wb[2], wb[3]);
    };
    // Degree 8: chunk qd of K-block kb is feature kb 8 + qd's run of degrees
    // 1..8 (zero past the last feature). Four chunks of both rows at a time:
    // eight independent recurrences with no branch between them; the values
    // are emit_run2x's, bit for bit.
    auto emit_kblock_d8 = [&](uint8_t* phik, int kb, const float (&xa)[8], const float (&xb)[8]) {
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        uint32_t wa[4][4], wb[4][4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const float xa0 = xa[h * 4 + u], xb0 = xb[h * 4 + u];
          const float a2 = xa0 + xa0, b2 = xb0 + xb0;
          float ta = xa0, tam = 1.f, tb = xb0, tbm = 1.f;
          float va[8], vb[8];
          va[0] = ta;
          vb[0] = tb;
#pragma unroll
          for (int e = 1; e < 8; ++e) {
            const float na = fmaf(a2, ta, -tam), nb = fmaf(b2, tb, -tbm);
            tam = ta;
            ta = na;
            tbm = tb;
            tb = nb;
            va[e] = ta;
            vb[e] = tb;
          }
#pragma unroll
          for (int e = 0; e < 4; ++e) {
            wa[u][e] = bf16x2_bits(va[2 * e], va[2 * e + 1]);
            wb[u][e] = bf16x2_bits(vb[2 * e], vb[2 * e + 1]);
          }
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int qd = h * 4 + u;
          const bool zero = kb * 8 + qd >= N;
          *reinterpret_cast<uint4*>(phik + r0 * 128 + ((qd ^ (r0 & 7)) << 4)) =
              zero ? make_uint4(0u, 0u, 0u, 0u)
                   : make_uint4(wa[u][0], wa[u][1], wa[u][2], wa[u][3]);
          if (R == 2)
            *reinterpret_cast<uint4*>(phik + r1 * 128 + ((qd ^ (r1 & 7)) << 4)) =
                zero ? make_uint4(0u, 0u, 0u, 0u)
                     : make_uint4(wb[u][0], wb[u][1], wb[u][2], wb[u][3]);
        }
      }
    };
    // both rows of a Chebyshev chunk that crosses feature runs (d >= 4)
    auto emit_cheb_cross2 = [&](uint8_t* phik, uint32_t desc, int qd) {
      float va[8], vb[8];
      if (R == 2) cheb_cross2(desc, a.d, N, xr0, xr1, XW, true, va, vb);
      else cheb_cross1(desc, a.d, N, xr0, XW, va);
      uint32_t wa[4], wb[4];
#pragma unroll
      for (int h = 0; h < 4; ++h) {
        wa[h] = bf16x2_bits(va[2 * h], va[2 * h + 1]);
        wb[h] = bf16x2_bits(vb[2 * h], vb[2 * h + 1]);
      }
      *reinterpret_cast<uint4*>(phik + r0 * 128 + ((qd ^ (r0 & 7)) << 4)) =
          make_uint4(wa[0], wa[1], wa[2], wa[3]);
      if (R == 2)
        *reinterpret_cast<uint4*>(phik + r1 * 128 + ((qd ^ (r1 & 7)) << 4)) =
            make_uint4(wb[0], wb[1], wb[2], wb[3]);
    };
    auto emit_cheb_run2 = [&](uint8_t* phik, uint32_t desc, int qd) {
      const int i = (int)(desc & 0xFFFFu);
      emit_run2x(phik, desc, qd, xr0[i * XW], R == 2 ? xr1[i * XW] : 0.f);
    };
    // waits until expansion slot q % NS may be written (use q / NS)
    auto slot_free = [&](int q) -> bool {
      const int use = q / NS;
      return use == 0 ||
             wait_bar(ptx::smem_addr(&phi_free[q % NS]), (use - 1) & 1, abort_flag, a.status);
    };
    bool ok = true;
    const bool staged = !(F == kFormBF16 && !TRI) || a.xstage;
    if (!staged) {
      // Features from global memory (L2), for the BF16 form, the Chebyshev
      // basis with d a multiple of 8 (every chunk one feature's run of 8
      // degrees) and BN a multiple of 128: the x of a K-block's 8 chunks
      // are loaded one K-block ahead; thread 0 prefetches the next tile's
      // feature blocks into L2.
      auto xptr = [&](int itn, int r) -> const float* {
        const int64_t m = ((int64_t)blockIdx.x + (int64_t)itn * G) * BN + r;
        return a.Xt + (m >> 7) * (int64_t)N * kPatBlock + (m & (kPatBlock - 1));
      };
      auto prefetch_tile = [&](int itn) {
        const int64_t m1 = ((int64_t)blockIdx.x + (int64_t)itn * G) * BN;
        ptx::bulk_prefetch_l2(a.Xt + (m1 / kPatBlock) * N * kPatBlock,
                              (uint32_t)((BN / kPatBlock) * N * kPatBlock * 4));
      };
      float na[8], nb[8];
      auto load_kb = [&](int itn, int kbn) {
        const float* p0 = xptr(itn, r0);
        const float* p1 = xptr(itn, r1);
#pragma unroll
        for (int q = 0; q < 8; ++q) {
          const int i = (int)(tab[kbn * 8 + q] & 0xFFFFu);
          na[q] = __ldg(p0 + i * kPatBlock);
          nb[q] = R == 2 ? __ldg(p1 + i * kPatBlock) : 0.f;
        }
      };
      if (bt == 0) {
        if (my_tiles > 0) prefetch_tile(0);
        if (my_tiles > 1) prefetch_tile(1);
      }
      if (my_tiles > 0) load_kb(0, 0);
      for (int it = 0; it < my_tiles && ok; ++it) {
        if (bt == 0 && it + 2 < my_tiles) prefetch_tile(it + 2);
        for (int kb = 0; kb < KB; ++kb) {
          float xa[8], xb[8];
#pragma unroll
          for (int q = 0; q < 8; ++q) {
            xa[q] = na[q];
            xb[q] = nb[q];
          }
          if (kb + 1 < KB) load_kb(it, kb + 1);
          else if (it + 1 < my_tiles) load_kb(it + 1, 0);
          const int q = it * KB + kb;
          ok = slot_free(q);
          if (!ok) break;
          uint8_t* phik = phi + (size_t)(q % NS) * BN * 128;
          if (a.d == 8) {
            emit_kblock_d8(phik, kb, xa, xb);
          } else {
#pragma unroll
          for (int qd = 0; qd < 8; ++qd) {
            const uint32_t desc = tab[kb * 8 + qd];
            if (desc & kChunkZero) {
              *reinterpret_cast<uint4*>(phik + r0 * 128 + ((qd ^ (r0 & 7)) << 4)) =
                  make_uint4(0u, 0u, 0u, 0u);
              if (R == 2)
                *reinterpret_cast<uint4*>(phik + r1 * 128 + ((qd ^ (r1 & 7)) << 4)) =
                    make_uint4(0u, 0u, 0u, 0u);
            } else {
              emit_run2x(phik, desc, qd, xa[qd], xb[qd]);
            }
          }
          }
          ptx::fence_proxy_async_smem();
          ptx::mbar_arrive(ptx::smem_addr(&phi_full[q % NS]));
        }
      }
    }
    for (int it = 0; it < my_tiles && ok && staged; ++it) {
      ok = wait_bar(ptx::smem_addr(x_full), it & 1, abort_flag, a.status);
      if (!ok) break;
      for (int kb = 0; kb < KB; ++kb) {
        const int q = it * KB + kb;
        ok = slot_free(q);
        if (!ok) break;
        uint8_t* phik = phi + (size_t)(q % NS) * NPHI * BN * 128;
        if (F == kFormBF16 && !TRI) {
          for (int qd = q0; qd < 8; qd += QS) {
            const uint32_t desc = tab[kb * 8 + qd];
            if (cheb && (desc & kChunkRun) && ((desc >> 24) & 15u) == 8u) {
              emit_cheb_run2(phik, desc, qd);
            } else if (cheb && a.d >= 4 && !(desc & kChunkZero)) {
              emit_cheb_cross2(phik, desc, qd);
            } else {
              emit(phik, desc, qd, r0, xr0);
              if (R == 2) emit(phik, desc, qd, r1, xr1);
            }
          }
        } else {
          for (int qd = q0; qd < 8; qd += QS) emit_unit(phik, kb, qd);
        }
        ptx::fence_proxy_async_smem();
        ptx::mbar_arrive(ptx::smem_addr(&phi_full[q % NS]));
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

TcPlan plan_tc_single(const Shape& s, int P, int num_sms, int form);

// The one-SM kernel where it runs 256-pattern tiles; where its shared memory
// forces narrower tiles, the BF16 form (with at least two chromosome tiles)
// takes the paired-SM kernel, whose CTAs each hold half of a 256-pattern
// tile's expansion. Measured on the large classification set (256-pattern
// one-SM tiles): one-SM 0.50 ms, pairs 0.54 ms per evaluation; on the
// surrogate workload (K' = 288, N = 48: one-SM 192-pattern tiles): one-SM
// 6.57 ms, pairs 5.33 ms.
namespace {
int g_base_pad = 1024;
__global__ void smem_base_probe_kernel(int* out) {
  extern __shared__ uint8_t probe_smem[];
  if (threadIdx.x == 0) *out = (int)((1024u - (ptx::smem_addr(probe_smem) & 1023u)) & 1023u);
}
}  // namespace

static std::atomic<int> g_slack_override{0};
void set_smem_base_pad(int pad) { g_base_pad = pad < 0 ? 1024 : (pad > 1024 ? 1024 : pad); }
int smem_base_pad() {
  const int o = g_slack_override.load();
  return o > 0 ? o : g_base_pad;
}
void set_smem_slack_override(int slack) { g_slack_override.store(slack); }
void note_smem_base_pad(int pad) {
  static std::atomic<int> seen{-1};   // largest padding probed so far
  int cur = seen.load();
  while (pad > cur && !seen.compare_exchange_weak(cur, pad)) {
  }
  set_smem_base_pad(seen.load());
}
cudaError_t launch_smem_base_probe(int* out, cudaStream_t st) {
  smem_base_probe_kernel<<<1, 32, 16, st>>>(out);
  return cudaGetLastError();
}

TcPlan plan_tc(const Shape& s, int P, int num_sms, int form) {
  const TcPlan one = plan_tc_single(s, P, num_sms, form);
  if (form == kFormBF16 && P > 128 && !(one.ok && one.BN == 256)) {
    const TcPlan pp = plan_tc_pair(s, P, num_sms);
    if (pp.ok) return pp;
  }
  return one;
}

TcPlan plan_tc_single(const Shape& s, int P, int num_sms, int form) {
  TcPlan pl{};
  pl.form = form;
  pl.KB = ceil_div(s.Kp, form_cols(form));
  pl.C = ceil_div(P, 128);
  pl.ok = false;
  const int cands[5] = {256, 192, 128, 64, 32};   // 192: BF16 form only
  // bf16x3 doubles both operands, so it may fall back to two gene stages
  const int min_stages = form == kFormBF16x3 ? 2 : 3;
  // BF16 with Chebyshev runs of 8 degrees at 256 / 128 patterns: features
  // read from L2 instead of staged, which frees room for spare expansion
  // slots (the next tile's first K-blocks are written during this tile)
  const bool runs = form == kFormBF16 && s.basis == GAME_BASIS_CHEB && s.d % 8 == 0;
  const int slack = smem_base_pad();
  pl.slack = slack;
  auto take = [&](int BN, int NS, int stages, int xstage, int ystage, int sm) {
    pl.BN = BN;
    pl.NS = NS;
    pl.stages = stages;
    pl.xstage = xstage;
    pl.ystage = ystage;
    // at least half an SM's shared memory: one CTA per SM, so the tensor
    // memory allocation never waits on a co-resident CTA
    pl.smem_bytes = sm < kMinSmem ? kMinSmem : sm;
    pl.ok = true;
  };
  for (int i = 0; i < 5 && !pl.ok; ++i) {
    if (cands[i] == 192 && form != kFormBF16) continue;
    // (features from L2, the targets also staged where they fit: the
    // feature producer is idle then)
    if (runs && cands[i] % 128 == 0)
      for (int stages = 4; stages >= min_stages && !pl.ok; --stages)
        for (int spare = pl.KB; spare >= 1 && !pl.ok; --spare)
          for (int ystage = 1; ystage >= 0 && !pl.ok; --ystage) {
            const int sm = smem_plan(pl.KB, pl.KB + spare, cands[i], s.N, stages, form, 0,
                                     ystage, slack).total;
            if (sm <= kMaxSmem) take(cands[i], pl.KB + spare, stages, 0, ystage, sm);
          }
    for (int stages = 4; stages >= min_stages && !pl.ok; --stages) {
      const int sm = smem_plan(pl.KB, pl.KB, cands[i], s.N, stages, form, 1, 0, slack).total;
      if (sm <= kMaxSmem) take(cands[i], pl.KB, stages, 1, 0, sm);
    }
  }
  if (!pl.ok) return pl;
  const int ntiles = ceil_div(s.M, pl.BN);   // Mpad (a multiple of 768) covers them
  pl.grid = ntiles < num_sms ? ntiles : num_sms;
  int cols = 32;
  while (cols < 2 * pl.BN) cols <<= 1;
  pl.tmem_cols = cols;
  pl.rows = 2 * pl.grid;   // one partial row per (CTA, column half)
  return pl;
}

template <bool ABS>
using TcKernel = void (*)(const TcArgs);

template <bool ABS>
TcKernel<ABS> pick_kernel(const TcPlan& pl) {
  return pl.form == kFormBF16x3 ? fitness_tc_kernel<kFormBF16x3, false, ABS>
         : pl.form == kFormFP8  ? fitness_tc_kernel<kFormFP8, false, ABS>
         : pl.BN == 192         ? fitness_tc_kernel<kFormBF16, true, ABS>
                                : fitness_tc_kernel<kFormBF16, false, ABS>;
}

cudaError_t launch_fitness_tc(const TcPlan& pl, const Shape& s, const float* Xt,
                              const float* y, const uint8_t* popA, const float* a0,
                              const float* uscale, const float* colinv, int P, int Ppad,
                              double* part, int* status, int err, cudaStream_t st) {
  (void)P;
  if (!pl.ok) return cudaErrorInvalidValue;
  if (pl.pair) return launch_fitness_tc_pair(pl, s, Xt, y, popA, a0, Ppad, part, status, err, st);
  TcArgs a;
  a.M = s.M;
  a.N = s.N;
  a.d = s.d;
  a.basis = s.basis;
  a.Kp = s.Kp;
  a.BN = pl.BN;
  a.KB = pl.KB;
  a.C = pl.C;
  a.stages = pl.stages;
  a.NS = pl.NS;
  a.xstage = pl.xstage;
  a.ystage = pl.ystage;
  a.slack = pl.slack;
  const int cols = form_cols(pl.form);
  const int last_cols = s.Kp - cols * (pl.KB - 1);
  a.nmma_last = (last_cols + cols / 4 - 1) / (cols / 4);
  a.ntiles = ceil_div(s.M, pl.BN);
  a.Ppad = Ppad;
  a.tmem_cols = pl.tmem_cols;
  a.Xt = Xt;
  a.y = y;
  a.popA = popA;
  a.a0 = a0;
  a.uscale = uscale;
  a.colinv = colinv;
  a.part = part;
  a.status = status;
  a.stall_ns = hook_take_stall_ns();
  if (pl.form == kFormFP8 && (!uscale || !colinv)) return cudaErrorInvalidValue;
  if (pl.BN == 192 && pl.form != kFormBF16) return cudaErrorInvalidValue;
  if (pl.NS < pl.KB || pl.NS > 2 * pl.KB) return cudaErrorInvalidValue;
  if (!pl.xstage && (pl.form != kFormBF16 || pl.BN % 128 != 0 || s.basis != GAME_BASIS_CHEB ||
                     s.d % 8 != 0))
    return cudaErrorInvalidValue;
  void (*kern)(const TcArgs) = err == GAME_ERR_MAE ? pick_kernel<true>(pl) : pick_kernel<false>(pl);
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       pl.smem_bytes);
  if (e != cudaSuccess) return e;
  kern<<<pl.grid, kThreads, pl.smem_bytes, st>>>(a);
  return cudaGetLastError();
}

}  // namespace game
