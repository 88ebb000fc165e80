// batch_tc.cu -- fitness of many independent GAME problems in one persistent
// tensor-core launch (BF16 operands, FP32 accumulation in tensor memory, the
// squared-error sum fused into the epilogue).
//
// The math per problem is that of fitness_tc.cu (paper Section 3, Eq. 2 and
// Eq. 3 with the MSE): for a tile of BN patterns, D[p][m] = A[p][:] . PHI[m][:]
// with the genes on MMA-M (128 TMEM lanes) and the tile's expansion on MMA-N.
//
// Work items are (problem r, pattern tile t), each with the problem's own
// N, d, basis, K' and tile width BN_r (chosen per problem by the autotuner in
// batch.cu). CTAs are persistent, one per SM, and walk a fixed list of items
// (sched[cta_begin[b] .. cta_begin[b+1])) built on the host by a greedy
// longest-first assignment. The shared-memory regions are sized for the
// largest item of the batch; within an item the layout follows the item's own
// BN and K-block count. Because items use different numbers of K-blocks, the
// phases of the per-K-block barriers are tracked as bit masks (one bit per
// K-block, flipped at each use) instead of the item counter.
//
// Each role copies an item's problem descriptor into registers once (the
// inline-asm memory clobbers of the pipeline would otherwise force a reload
// from global memory after every copy, MMA and barrier operation).
//
// Roles as in fitness_tc.cu: warp 0 gene-block producer, warp 1 MMA issuer
// and TMEM owner, warp 2 feature producer, warps 4-11 epilogue, warps 12-15
// expansion. Each item writes its FP64 partial sums to its own rows,
// part[part_base_r + t Ppad_r + p], so the result does not depend
// on which CTA took the item; the batched reduce adds a problem's rows in
// tile order. All waits are bounded (2 s) as in fitness_tc.cu.
#include "basis.cuh"
#include "game_internal.cuh"
#include "tc_common.cuh"
#include "tc_ptx.cuh"

namespace game {

namespace {

using namespace tc;

constexpr uint32_t kABytes = 128 * 128;
constexpr int kWarps = 16;
constexpr int kThreads = kWarps * 32;
// Items carry 1-2 chromosome tiles, so the expansion, not the epilogue, is
// the busy role: 4 epilogue warps (each thread one chromosome row, all of a
// tile's columns) and 8 expansion warps.
constexpr int kEpiWarp0 = 4;
constexpr int kEpiThreads = 128;
constexpr int kBasisWarp0 = 8;
constexpr int kBasisThreads = 256;
constexpr int kStages = 4;

struct BSmem {
  int phi, ast, xs, tab, bars, total;
};

__host__ __device__ inline BSmem bsmem_plan(int phi_bytes, int x_bytes, int KBmax) {
  BSmem s;
  s.phi = 0;
  s.ast = phi_bytes;
  s.xs = s.ast + kStages * (int)kABytes;
  s.tab = s.xs + x_bytes;
  s.bars = (s.tab + 2 * KBmax * 8 * 4 + 7) & ~7;   // two chunk tables
  s.total = s.bars + (2 * kStages + 2 * KBmax + 7) * 8 + 16 + 1024;
  return s;
}

__global__ void __launch_bounds__(kThreads, 1) fitness_batch_kernel(const BatchArgs a) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* base = reinterpret_cast<uint8_t*>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~static_cast<uintptr_t>(1023));
  const int KBmax = a.KBmax;
  const BSmem sp = bsmem_plan(a.phi_bytes, a.x_bytes, KBmax);
  uint8_t* phi = base + sp.phi;
  uint8_t* ast = base + sp.ast;
  float* xs = reinterpret_cast<float*>(base + sp.xs);
  uint32_t* tab = reinterpret_cast<uint32_t*>(base + sp.tab);
  uint64_t* bars = reinterpret_cast<uint64_t*>(base + sp.bars);
  uint64_t* a_full = bars;
  uint64_t* a_empty = a_full + kStages;
  uint64_t* phi_full = a_empty + kStages;
  uint64_t* phi_free = phi_full + KBmax;
  uint64_t* acc_full = phi_free + KBmax;
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
    for (int kb = 0; kb < KBmax; ++kb) {
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

  const int it0 = a.cta_begin[blockIdx.x], it1 = a.cta_begin[blockIdx.x + 1];

  if (warp == 0) {
    // ---------------- gene-block producer ----------------
    if (lane == 0) {
      uint32_t q = 0, s = 0, ph = 0;
      bool ok = true;
      for (int it = it0; it < it1 && ok; ++it) {
        const BatchRun R = a.runs[a.items[a.sched[it]].x];
        for (int c = 0; c < R.C && ok; ++c)
          for (int kb = 0; kb < R.KB && ok; ++kb) {
            ok = wait_bar(ptx::smem_addr(&a_empty[s]), ph ^ 1, abort_flag, a.status);
            if (!ok) break;
            ptx::mbar_arrive_expect_tx(ptx::smem_addr(&a_full[s]), kABytes);
            ptx::bulk_g2s(ptx::smem_addr(ast + s * kABytes),
                          R.popA + (size_t)(c * R.KB + kb) * kABytes, kABytes,
                          ptx::smem_addr(&a_full[s]));
            ++q;
            if (++s == (uint32_t)kStages) {
              s = 0;
              ph ^= 1;
            }
          }
      }
      for (uint32_t st = 0; st < (uint32_t)kStages && st < q; ++st) {
        const uint32_t uses = (q - st + kStages - 1) / kStages;
        wait_bar_drain(ptx::smem_addr(&a_full[st]), (uses - 1) & 1, a.status);
      }
    }
  } else if (warp == 1) {
    // ---------------- MMA issuer ----------------
    if (lane == 0) {
      const uint64_t adesc0 = ptx::desc_kmajor_sw128(ptx::smem_addr(ast));
      const uint64_t bdesc0 = ptx::desc_kmajor_sw128(ptx::smem_addr(phi));
      const uint32_t a_step = kABytes >> 4;
      const uint32_t a_full0 = ptx::smem_addr(a_full), a_empty0 = ptx::smem_addr(a_empty);
      const uint32_t phi_full0 = ptx::smem_addr(phi_full), phi_free0 = ptx::smem_addr(phi_free);
      const uint32_t acc_full0 = ptx::smem_addr(acc_full), acc_empty0 = ptx::smem_addr(acc_empty);
      uint32_t s = 0, ph = 0, acc_it = 0;
      uint32_t full_par = 0;   // bit kb: parity of the next phi_full[kb] phase
      bool ok = true;
      for (int it = it0; it < it1 && ok; ++it) {
        const BatchRun R = a.runs[a.items[a.sched[it]].x];
        const int KB = R.KB, C = R.C, BN = R.BN, nlast = R.nmma_last;
        const uint32_t idesc = ptx::idesc_bf16_f32(128, BN);
        const uint32_t b_step = (uint32_t)(BN * 128) >> 4;
        auto kblock = [&](uint32_t d_tmem, uint32_t st, int kb, int nm) {
          const uint64_t ad = adesc0 + st * a_step;
          const uint64_t bd = bdesc0 + (uint32_t)kb * b_step;
          for (int kk = 0; kk < nm; ++kk)
            ptx::mma_bf16(d_tmem, ad + 2u * kk, bd + 2u * kk, idesc, (kb | kk) != 0);
        };
        for (int c = 0; c < C && ok; ++c) {
          const uint32_t buf = acc_it & 1, u = acc_it >> 1;
          ok = wait_bar(acc_empty0 + 8 * buf, (u & 1) ^ 1, abort_flag, a.status);
          if (!ok) break;
          ptx::tc_fence_after();
          const uint32_t d_tmem = tmem + buf * (uint32_t)a.bn_max;
          for (int kb = 0; kb < KB && ok; ++kb) {
            if (c == 0) ok = wait_bar(phi_full0 + 8 * kb, (full_par >> kb) & 1u, abort_flag,
                                      a.status);
            if (ok) ok = wait_bar(a_full0 + 8 * s, ph, abort_flag, a.status);
            if (!ok) break;
            kblock(d_tmem, s, kb, kb == KB - 1 ? nlast : 4);
            ptx::mma_commit(a_empty0 + 8 * s);
            if (c == C - 1) ptx::mma_commit(phi_free0 + 8 * kb);
            if (++s == (uint32_t)kStages) {
              s = 0;
              ph ^= 1;
            }
          }
          if (!ok) break;
          ptx::mma_commit(acc_full0 + 8 * buf);
          ++acc_it;
        }
        full_par ^= (KB >= 32) ? 0xFFFFFFFFu : ((1u << KB) - 1u);
      }
      ptx::mma_commit(ptx::smem_addr(drain));
      wait_bar_drain(ptx::smem_addr(drain), 0, a.status);
    }
  } else if (warp == 2) {
    // ---------------- feature producer ----------------
    if (lane == 0) {
      int issued = 0;
      for (int it = it0; it < it1; ++it) {
        const int2 item = a.items[a.sched[it]];
        const BatchRun R = a.runs[item.x];
        if (!wait_bar(ptx::smem_addr(x_empty), (issued & 1) ^ 1, abort_flag, a.status)) break;
        const int BN = R.BN, N = R.N;
        const uint32_t bytes = (uint32_t)(N * BN * 4);
        ptx::mbar_arrive_expect_tx(ptx::smem_addr(x_full), bytes);
        const int64_t m0 = (int64_t)item.y * BN;
        if (BN >= kPatBlock) {
          ptx::bulk_g2s(ptx::smem_addr(xs), R.Xt + m0 * N, bytes, ptx::smem_addr(x_full));
        } else {
          const int64_t blk = m0 / kPatBlock;
          const int off = (int)(m0 % kPatBlock);
          for (int i = 0; i < N; ++i)
            ptx::bulk_g2s(ptx::smem_addr(xs + i * BN), R.Xt + (blk * N + i) * kPatBlock + off,
                          (uint32_t)BN * 4, ptx::smem_addr(x_full));
        }
        // the next item's feature blocks into L2, so its copy reads L2
        if (it + 1 < it1) {
          const int2 nx = a.items[a.sched[it + 1]];
          const BatchRun R2 = a.runs[nx.x];
          const int64_t m1 = (int64_t)nx.y * R2.BN;
          const int64_t b0 = m1 / kPatBlock, b1 = (m1 + R2.BN - 1) / kPatBlock;
          ptx::bulk_prefetch_l2(R2.Xt + b0 * R2.N * kPatBlock,
                                (uint32_t)((b1 - b0 + 1) * R2.N * kPatBlock * 4));
        }
        ++issued;
      }
      if (issued > 0) wait_bar_drain(ptx::smem_addr(x_full), (issued - 1) & 1, a.status);
    }
  } else if (warp >= kEpiWarp0 && warp < kBasisWarp0) {
    // ---------------- epilogue ----------------
    const int qw = warp & 3;

    const int row = qw * 32 + lane;
    const uint32_t lane_addr = (uint32_t)(qw * 32) << 16;
    const uint64_t negu2 = ptx::f2_pack(-1.f, -1.f);
    uint32_t acc_it = 0;
    bool ok = true;
    for (int it = it0; it < it1 && ok; ++it) {
      const int2 item = a.items[a.sched[it]];
      const BatchRun R = a.runs[item.x];
      const int BN = R.BN;
      const int HW = BN;   // all of the tile's columns
      const int col_lo = 0;
      const int64_t m0 = (int64_t)item.y * BN;
      const int64_t rem = R.M - m0 - col_lo;
      const int valid = rem <= 0 ? 0 : (rem >= HW ? HW : (int)rem);
      const float* yt = R.y + m0 + col_lo;
      double* prow = a.part + R.part_base + (int64_t)item.y * R.Ppad;
      for (int c = 0; c < R.C; ++c) {
        const uint32_t buf = acc_it & 1, u = acc_it >> 1;
        ok = wait_bar(ptx::smem_addr(&acc_full[buf]), u & 1, abort_flag, a.status);
        if (!ok) break;
        ptx::tc_fence_after();
        const int chrom = c * 128 + row;
        const float bias = R.a0[chrom];
        const uint64_t bias2 = ptx::f2_pack(bias, bias);
        uint64_t s2 = 0;
        float s_tail = 0.f;
        const uint32_t tbase = tmem + lane_addr + buf * (uint32_t)a.bn_max + (uint32_t)col_lo;
        const int nfull = valid / 32;
        if (nfull > 0) {
          uint32_t va[32], vb[32];
          ptx::tmem_ld32_issue(tbase, va);
          ptx::tmem_ld32_wait(va);
          for (int k = 0; k < nfull; k += 2) {
            const bool has_b = k + 1 < nfull;
            if (has_b) ptx::tmem_ld32_issue(tbase + (uint32_t)(k + 1) * 32, vb);
            epi_chunk<false>(va, yt + k * 32, bias2, negu2, s2);
            if (has_b) {
              ptx::tmem_ld32_wait(vb);
              const bool has_a = k + 2 < nfull;
              if (has_a) ptx::tmem_ld32_issue(tbase + (uint32_t)(k + 2) * 32, va);
              epi_chunk<false>(vb, yt + (k + 1) * 32, bias2, negu2, s2);
              if (has_a) ptx::tmem_ld32_wait(va);
            }
          }
        }
        if (nfull * 32 < valid) {
          uint32_t v[32];
          ptx::tmem_ld32(tbase + (uint32_t)nfull * 32, v);
          const int lim = valid - nfull * 32;
#pragma unroll
          for (int e = 0; e < 32; ++e) {
            if (e < lim) {
              const float r = (yt[nfull * 32 + e] - bias) - __uint_as_float(v[e]);
              s_tail = fmaf(r, r, s_tail);
            }
          }
        }
        ptx::tc_fence_before();
        ptx::mbar_arrive(ptx::smem_addr(&acc_empty[buf]));
        const float2 sp2 = ptx::f2_unpack(s2);
        prow[chrom] = (double)sp2.x + (double)sp2.y + (double)s_tail;
        ++acc_it;
      }
    }
  } else if (warp >= kBasisWarp0) {
    // ---------------- expansion (basis) ----------------
    // The chunk table is rebuilt per item (double-buffered by item parity,
    // one named barrier per item). After an abort the threads keep walking
    // the item list and passing that barrier, doing no waits or stores, so
    // every basis thread executes the same barriers.
    // K-block kb of an item sits at kb * BN * 128, so when BN changes from one
    // item to the next a new K-block can overlap any K-block of the previous
    // layout: then every outstanding phi_free phase is awaited before the
    // first store (the CTA's items are sorted by problem, so this is rare).
    const int bt = threadIdx.x - kBasisWarp0 * 32;
    uint32_t pending = 0;    // bit kb: a filled K-block whose phi_free phase is outstanding
    uint32_t free_par = 0;   // bit kb: parity of the next phi_free[kb] phase
    int items_done = 0, prev_bn = 0;
    bool dead = false;
    auto await_free = [&](int kb) {
      dead = !wait_bar(ptx::smem_addr(&phi_free[kb]), (free_par >> kb) & 1u, abort_flag,
                       a.status);
      free_par ^= 1u << kb;
      pending &= ~(1u << kb);
    };
    for (int it = it0; it < it1; ++it) {
      const int2 item = a.items[a.sched[it]];
      const BatchRun R = a.runs[item.x];
      const int BN = R.BN, N = R.N, KB = R.KB;
      uint32_t* tb = tab + (items_done & 1) * (KBmax * 8);
      for (int cid = bt; cid < KB * 8; cid += kBasisThreads)
        tb[cid] = chunk_desc(cid, R.basis, R.d, R.Kp);
      ptx::named_bar(1, kBasisThreads);
      // one row per thread (256 threads, BN <= 256 rows), 256 / BN unit groups
      const int XW = BN < 128 ? BN : 128;       // patterns per feature row in xs
      const int RW = BN;
      const int QS = kBasisThreads / RW;
      const int r0 = bt % RW, q0 = bt / RW;
      const float* xrow0 = xs + (r0 >> 7) * N * XW + (r0 % XW);
      if (!dead) dead = !wait_bar(ptx::smem_addr(x_full), items_done & 1, abort_flag, a.status);
      if (BN != prev_bn)
        for (int kb = 0; kb < KBmax && !dead; ++kb)
          if ((pending >> kb) & 1u) await_free(kb);
      prev_bn = BN;
      for (int kb = 0; kb < KB && !dead; ++kb) {
        if ((pending >> kb) & 1u) {
          await_free(kb);
          if (dead) break;
        }
        uint8_t* phik = phi + (size_t)kb * BN * 128;
        for (int qd = q0; qd < 8; qd += QS) {
          const uint32_t desc = tb[kb * 8 + qd];
          float va[8];
          gen_chunk(desc, R.basis, R.d, N, xrow0, XW, va);
          *reinterpret_cast<uint4*>(phik + r0 * 128 + ((qd ^ (r0 & 7)) << 4)) =
              make_uint4(bf16x2_bits(va[0], va[1]), bf16x2_bits(va[2], va[3]),
                         bf16x2_bits(va[4], va[5]), bf16x2_bits(va[6], va[7]));
        }
        ptx::fence_proxy_async_smem();
        ptx::mbar_arrive(ptx::smem_addr(&phi_full[kb]));
        pending |= 1u << kb;
      }
      if (!dead) ptx::mbar_arrive(ptx::smem_addr(x_empty));
      ++items_done;
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

int batch_smem_bytes(int phi_bytes, int x_bytes, int KBmax) {
  return bsmem_plan(phi_bytes, x_bytes, KBmax).total;
}

cudaError_t prepare_fitness_batch(int smem_bytes) {
  if (smem_bytes > 232448) return cudaErrorInvalidValue;
  return cudaFuncSetAttribute(fitness_batch_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              smem_bytes);
}

cudaError_t launch_fitness_batch(const BatchArgs& a, int grid, int smem_bytes, cudaStream_t st) {
  if (a.KBmax > 32 || smem_bytes > 232448) return cudaErrorInvalidValue;
  fitness_batch_kernel<<<grid, kThreads, smem_bytes, st>>>(a);
  return cudaGetLastError();
}

}  // namespace game
