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
// batch.cu). CTAs are persistent, one per SM, and take items from one list
// (recs, widest tiles first, longest first within a width) through a global
// counter: warp 2 takes them into the CTA's queue, where every role reads
// them in the same order; each role loads its next item's record while it
// works on the current one. The shared-memory regions are sized for the
// largest item of the batch; within an item the layout follows the item's own
// BN and its expansion slots (one per K-block, or a ring of RK slots). Because
// items use different numbers of slots, the phases of the per-slot barriers
// are tracked as bit masks (one bit per slot, flipped at each use) instead of
// the item counter.
//
// Roles: warp 0 gene-block producer, warp 1 MMA issuer and TMEM owner, warp 2
// scheduler and L2 prefetcher, warps 4-7 epilogue (targets staged in shared memory one item
// ahead), warps 8-15 expansion. The expansion is the busy role (items carry
// 1-2 chromosome tiles, so each expansion value feeds few MMAs): each
// expansion thread streams one pattern row over a contiguous range of whole
// features, with the basis and the degree compile-time constants
// (FeatureGroup in basis.cuh), its features streamed from global memory
// through a per-thread ring of asynchronous copies. Each item writes its FP64
// partial sums to its own row, part[part_base_r + t Ppad_r + p], so the
// result does not depend on which CTA took the item; the batched reduce adds
// a problem's rows in tile order. All waits are bounded (2 s) as in
// fitness_tc.cu.
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
constexpr int kStages = 3;
constexpr int kYSlot = 256;   // targets of one item (floats), two slots
constexpr int kRing = 16;     // features in flight per expansion thread
constexpr int kQueue = 8;     // items scheduled ahead of the slowest role
// readers of each queue slot: gene producer, MMA issuer, the epilogue (one
// thread, which hands the index to the others), every expansion thread
constexpr int kQueueReaders = 3 + kBasisThreads;

struct BSmem {
  int phi, ast, ys, ring, bars, total;
};

__host__ __device__ inline BSmem bsmem_plan(int phi_bytes, int KBmax) {
  BSmem s;
  s.phi = 0;
  s.ast = phi_bytes;
  s.ys = s.ast + kStages * (int)kABytes;
  s.ring = s.ys + 2 * kYSlot * 4;
  s.bars = s.ring + kRing * kBasisThreads * 4;
  s.total = s.bars + (2 * kStages + 2 * KBmax + 5 + 2 * kQueue) * 8 + 16 + 4 * (kQueue + 2) + 1024;
  return s;
}

// The expansion role's state carried from item to item, and its constants.
//
// K-block kb of an item lives in slot kb; for ring items (RK < KB, one
// accumulator group) in slot kb & (RK - 1), RK a power of two, so a ring item
// uses a slot several times. Every expansion thread arrives once per K-block
// on its slot's phi_full barrier (count 256), after its last store into that
// K-block (at once for a K-block it does not write), and each arrival leaves
// the slot pending: before the thread next stores into, or arrives on, that
// slot it awaits the slot's phi_free phase (the MMAs' release). Each slot
// thus holds at most one pending phase per thread, every phase is awaited
// exactly once and in order, and the parity bits stay exact. No thread
// awaits a release that needs its own later arrivals: a plain item uses each
// slot once, so its own releases are awaited only by the next item; a ring
// item has one accumulator group, whose MMAs release a K-block as soon as
// they have used it. With several threads per row, a thread whose range
// starts past the ring's first pass waits there for the MMAs of the row's
// earlier K-blocks: slower, never stuck, as every wait is for the MMAs of a
// lower K-block, whose arrivals come first in each thread's order.
struct ExpState {
  uint32_t pending;    // bit k: arrived on phi_full[k], its phi_free phase not yet awaited
  uint32_t free_par;   // bit k: parity of the next phi_free[k] phase
  int dead;            // a wait failed (time limit or another role's abort)
};
struct ExpEnv {
  uint32_t phi;                    // shared-memory addresses: expansion K-blocks,
  uint32_t ring;                   // the feature ring,
  uint32_t phi_full0, phi_free0;   // the barrier arrays
  volatile int* abort_flag;
  int* status;
};

__device__ __forceinline__ void await_mask(ExpState& es, const ExpEnv& env, uint32_t m) {
  m &= es.pending;
  while (m != 0u && !es.dead) {
    const int k = __ffs(m) - 1;
    m &= m - 1u;
    es.dead = !wait_bar(env.phi_free0 + 8u * (uint32_t)k, (es.free_par >> k) & 1u,
                        env.abort_flag, env.status);
    es.free_par ^= 1u << k;
    es.pending &= ~(1u << k);
  }
}

// One thread's place in one item: pattern row r0 of the tile, stores in
// increasing column order (16 bytes = 8 columns at a time, into the K-major
// 128-byte-swizzled K-block layout the MMA reads).
struct RowCursor {
  ExpState& es;
  const ExpEnv& env;
  int BN, r0, colmax;   // colmax = KB * 64
  int rmask;            // K-block kb in slot kb & rmask (all ones unless a ring)
  int next_arr;         // next K-block to arrive on
  int awaited;          // the slot of K-block `awaited` (and of every lower one) is awaited

  // before the first store into, or arrival on, K-block kb: the previous
  // phase of its slot
  __device__ __forceinline__ void await_for(int kb) {
    const uint32_t m = es.pending & (1u << (kb & rmask));
    if (m != 0u) await_mask(es, env, m);
    awaited = kb;
  }
  __device__ __forceinline__ void arrive(int kb) {
    const int sl = kb & rmask;
    ptx::mbar_arrive(env.phi_full0 + 8u * (uint32_t)sl);
    es.pending |= 1u << sl;
  }
  // arrive on K-blocks [next_arr, kbe)
  __device__ __forceinline__ void arrive_below(int kbe) {
    if (kbe <= next_arr || es.dead) return;
    ptx::fence_proxy_async_smem();
    for (int k = next_arr; k < kbe; ++k) {
      if (k > awaited) await_for(k);
      if (es.dead) return;
      arrive(k);
      next_arr = k + 1;
    }
  }
  // es.dead changes only inside a wait, which is checked right after; once
  // set, the rest of the thread's group still writes its own in-bounds
  // shared-memory cells and arrives at most once per K-block, and the
  // caller's loop stops at the next group
  __device__ __forceinline__ void store(int col, uint4 val) {
    if (col >= colmax) return;
    const int kb = col >> 6;
    if (kb > awaited) {
      await_for(kb);
      if (es.dead) return;
    }
    ptx::st_shared_v4(env.phi + (uint32_t)((kb & rmask) * BN * 128 + r0 * 128) +
                          (uint32_t)((((col >> 3) & 7) ^ (r0 & 7)) << 4), val);
    if (((col + 8) & 63) == 0) {
      ptx::fence_proxy_async_smem();
      arrive(kb);
      next_arr = kb + 1;
    }
  }
};

// sse += ((y - bias) - acc)^2 over 32 columns with the targets in shared
// memory (the arithmetic of epi_chunk<false>: one packed subtraction and one
// packed FMA per two columns)
__device__ __forceinline__ void epi_chunk_smem(const uint32_t (&v)[32], const float* yc,
                                               uint64_t bias2, uint64_t& s2) {
#pragma unroll
  for (int e4 = 0; e4 < 8; ++e4) {
    const float4 yv = reinterpret_cast<const float4*>(yc)[e4];
    const uint64_t ya = ptx::f2_sub(ptx::f2_pack(yv.x, yv.y), bias2);
    const uint64_t yb = ptx::f2_sub(ptx::f2_pack(yv.z, yv.w), bias2);
    const uint64_t da = ptx::f2_pack(__uint_as_float(v[4 * e4 + 0]), __uint_as_float(v[4 * e4 + 1]));
    const uint64_t db = ptx::f2_pack(__uint_as_float(v[4 * e4 + 2]), __uint_as_float(v[4 * e4 + 3]));
    const uint64_t ra = ptx::f2_sub(ya, da);
    const uint64_t rb = ptx::f2_sub(yb, db);
    s2 = ptx::f2_fma(ra, ra, s2);
    s2 = ptx::f2_fma(rb, rb, s2);
  }
}

__device__ __forceinline__ uint4 pack8(const float* v) {
  return make_uint4(bf16x2_bits(v[0], v[1]), bf16x2_bits(v[2], v[3]), bf16x2_bits(v[4], v[5]),
                    bf16x2_bits(v[6], v[7]));
}

// Asynchronous copies of features i0 .. i0 + F - 1 (those below N) of the row
// at xp (stride kPatBlock) into the thread's ring slots slot0 .. slot0 + F - 1
// (slot k of thread bt at ring + (k kBasisThreads + bt) 4: a warp's copies of
// one feature fill 128 consecutive bytes).
template <int F>
__device__ __forceinline__ void issue_group(const float* xp, int i0, int N, uint32_t slot_addr) {
#pragma unroll
  for (int f = 0; f < F; ++f)
    if (i0 + f < N)
      ptx::cp_async4(slot_addr + (uint32_t)(f * kBasisThreads * 4), xp + (size_t)(i0 + f) * kPatBlock);
}

// The thread's share of one item with (basis, degree) known at compile time:
// the row's feature groups split into QS contiguous ranges (thread q0 takes
// range q0); the last range's thread also writes the zero columns from the
// end of the last group to the end of the last K-block. U groups are
// generated together (FeatureGroup::U: at least 8 independent recurrences),
// then stored. The thread's features stream through its own ring of kRing
// shared-memory slots by asynchronous copies, PD = kRing / (U F) steps ahead
// of the generator (one commit group per step; the refill of a step's slots
// is issued after the step's values have been generated from them). Not
// inlined: each (basis, degree) gets its own register allocation.
template <int BASIS, int D>
__device__ __noinline__ ExpState expand_item(ExpState es, const ExpEnv env, const float* xp,
                                             int N, int KB, int RK, int BN, int r0, int q0,
                                             int QS, int bt) {
  using FG = FeatureGroup<BASIS, D>;
  constexpr int U = FG::U, UF = FG::U * FG::F, UG = FG::U * FG::G;
  constexpr int PD = kRing / UF;   // UF divides 16
  RowCursor rc{es, env, BN, r0, KB * 64, RK < KB ? RK - 1 : -1, 0, -1};
  const int ng = (N + FG::F - 1) / FG::F;
  const int gb = q0 * ng / QS, ge = (q0 + 1) * ng / QS;
  const int cs = gb * FG::G < rc.colmax ? gb * FG::G : rc.colmax;
  const uint32_t ring_t = env.ring + (uint32_t)bt * 4u;
  for (int k = 0; k < PD; ++k) {
    if (gb + k * U < ge)
      issue_group<UF>(xp, (gb + k * U) * FG::F, N, ring_t + (uint32_t)(k * UF * kBasisThreads * 4));
    ptx::cp_async_commit();
  }
  rc.arrive_below(cs >> 6);
  for (int g = gb, k = 0; g < ge && !es.dead; g += U) {
    ptx::cp_async_wait<PD - 1>();
    const uint32_t slot = ring_t + (uint32_t)(k * UF * kBasisThreads * 4);
    float xc[UF];
#pragma unroll
    for (int f = 0; f < UF; ++f)
      xc[f] = (g * FG::F + f < N) ? ptx::ld_shared_f32(slot + (uint32_t)(f * kBasisThreads * 4))
                                  : 0.f;
    uint32_t pk[UG / 2];
    features_bf16<BASIS, D, UF>(xc, N - g * FG::F, pk);
    if (g + PD * U < ge) issue_group<UF>(xp, (g + PD * U) * FG::F, N, slot);
    ptx::cp_async_commit();
    const int gcol = g * FG::G;
#pragma unroll
    for (int q = 0; q < U * FG::CH; ++q)
      if (g + q / FG::CH < ge)   // groups past the range belong to the next thread
        rc.store(gcol + 8 * q, make_uint4(pk[4 * q], pk[4 * q + 1], pk[4 * q + 2], pk[4 * q + 3]));
    k = (k + 1 == PD) ? 0 : k + 1;
  }
  ptx::cp_async_wait<0>();
  if (q0 == QS - 1)
    for (int col = ng * FG::G; col < rc.colmax; col += 8) rc.store(col, make_uint4(0, 0, 0, 0));
  rc.arrive_below(KB);
  return es;
}

// Any other degree: per K-block, the thread's CPT = 8 / QS chunks of its row
// from the generic chunk generator.
__device__ __noinline__ ExpState expand_item_generic(ExpState es, const ExpEnv env,
                                                     const float* xp, const BatchItem R, int r0,
                                                     int q0, int QS) {
  RowCursor rc{es, env, R.BN, r0, R.KB * 64, R.RK < R.KB ? R.RK - 1 : -1, 0, -1};
  const int CPT = 8 / QS;
  for (int kb = 0; kb < R.KB && !es.dead; ++kb) {
    for (int qd = q0 * CPT; qd < (q0 + 1) * CPT; ++qd) {
      float va[8];
      gen_chunk(chunk_desc(kb * 8 + qd, R.basis, R.d, R.Kp), R.basis, R.d, R.N, xp, kPatBlock, va);
      rc.store(kb * 64 + qd * 8, pack8(va));
    }
    rc.arrive_below(kb + 1);
  }
  return es;
}

template <int BASIS>
__device__ __forceinline__ ExpState expand_dispatch(ExpState es, const ExpEnv& env,
                                                    const float* xp, const BatchItem& R, int r0,
                                                    int q0, int QS, int bt) {
  const int N = R.N, KB = R.KB, RK = R.RK, BN = R.BN;
  switch (R.d) {
    case 1: return expand_item<BASIS, 1>(es, env, xp, N, KB, RK, BN, r0, q0, QS, bt);
    case 2: return expand_item<BASIS, 2>(es, env, xp, N, KB, RK, BN, r0, q0, QS, bt);
    case 3: return expand_item<BASIS, 3>(es, env, xp, N, KB, RK, BN, r0, q0, QS, bt);
    case 4: return expand_item<BASIS, 4>(es, env, xp, N, KB, RK, BN, r0, q0, QS, bt);
    case 5: return expand_item<BASIS, 5>(es, env, xp, N, KB, RK, BN, r0, q0, QS, bt);
    case 6: return expand_item<BASIS, 6>(es, env, xp, N, KB, RK, BN, r0, q0, QS, bt);
    case 7: return expand_item<BASIS, 7>(es, env, xp, N, KB, RK, BN, r0, q0, QS, bt);
    case 8: return expand_item<BASIS, 8>(es, env, xp, N, KB, RK, BN, r0, q0, QS, bt);
    case 9: return expand_item<BASIS, 9>(es, env, xp, N, KB, RK, BN, r0, q0, QS, bt);
    case 10: return expand_item<BASIS, 10>(es, env, xp, N, KB, RK, BN, r0, q0, QS, bt);
    default: return expand_item_generic(es, env, xp, R, r0, q0, QS);
  }
}

// One role's reader of the CTA's item queue (filled by the scheduler thread
// from the global item counter). pop() returns the next item's index, -1
// once the items are exhausted or when the wait failed (time limit or
// abort).
struct ItemQueue {
  uint32_t full0, empty0;      // shared-memory addresses of q_full[0], q_empty[0]
  const volatile int* idx;     // the slots' item indices
  volatile int* abort_flag;
  int* status;
  int seq;
  __device__ __forceinline__ int pop() {
    const int slot = seq % kQueue;
    const uint32_t par = (uint32_t)(seq / kQueue) & 1u;
    ++seq;
    if (!wait_bar(full0 + 8u * (uint32_t)slot, par, abort_flag, status)) return -1;
    const int v = idx[slot];
    ptx::mbar_arrive(empty0 + 8u * (uint32_t)slot);
    return v;
  }
};

// L2 prefetch of one item's features and targets (16-byte aligned: tile
// starts are multiples of 32 patterns).
__device__ __forceinline__ void prefetch_item(const BatchItem& R) {
  const int64_t m0 = R.m0;
  if (R.BN >= kPatBlock) {
    const int64_t b0 = m0 / kPatBlock, b1 = (m0 + R.BN - 1) / kPatBlock;
    ptx::bulk_prefetch_l2(R.Xt + b0 * R.N * kPatBlock,
                          (uint32_t)((b1 - b0 + 1) * R.N * kPatBlock * 4));
  } else {
    const int64_t blk = m0 / kPatBlock;
    const int off = (int)(m0 % kPatBlock);
    for (int i = 0; i < R.N; ++i)
      ptx::bulk_prefetch_l2(R.Xt + (blk * R.N + i) * kPatBlock + off, (uint32_t)R.BN * 4);
  }
  ptx::bulk_prefetch_l2(R.y + m0, (uint32_t)R.BN * 4);
}

__global__ void __launch_bounds__(kThreads, 1) fitness_batch_kernel(const BatchArgs a) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* base = reinterpret_cast<uint8_t*>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~static_cast<uintptr_t>(1023));
  const int KBmax = a.KBmax;
  const BSmem sp = bsmem_plan(a.phi_bytes, KBmax);
  uint8_t* phi = base + sp.phi;
  uint8_t* ast = base + sp.ast;
  float* ys = reinterpret_cast<float*>(base + sp.ys);
  float* ring = reinterpret_cast<float*>(base + sp.ring);
  uint64_t* bars = reinterpret_cast<uint64_t*>(base + sp.bars);
  uint64_t* a_full = bars;
  uint64_t* a_empty = a_full + kStages;
  uint64_t* phi_full = a_empty + kStages;
  uint64_t* phi_free = phi_full + KBmax;
  uint64_t* acc_full = phi_free + KBmax;
  uint64_t* acc_empty = acc_full + 2;
  uint64_t* drain = acc_empty + 2;
  uint64_t* q_full = drain + 1;
  uint64_t* q_empty = q_full + kQueue;
  uint32_t* tmem_holder = reinterpret_cast<uint32_t*>(q_empty + kQueue);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_holder + 1);
  volatile int* qidx = abort_flag + 1;       // [kQueue] item index per queue slot
  volatile int* ebc = qidx + kQueue;         // [2] item indices handed to the epilogue threads

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
    ptx::mbar_init(ptx::smem_addr(drain), 1);
    *abort_flag = 0;
    for (int q = 0; q < kQueue; ++q) {
      ptx::mbar_init(ptx::smem_addr(&q_full[q]), 1);
      ptx::mbar_init(ptx::smem_addr(&q_empty[q]), kQueueReaders);
    }
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

  ItemQueue iq{ptx::smem_addr(q_full), ptx::smem_addr(q_empty), qidx, abort_flag, a.status, 0};

  if (warp == 0) {
    // ---------------- gene-block producer ----------------
    if (lane == 0) {
      uint32_t q = 0, s = 0, ph = 0;
      bool ok = true;
      BatchItem nxt;
      int idx_n = iq.pop();
      if (idx_n >= 0) nxt = a.recs[idx_n];
      for (int idx = idx_n; idx >= 0 && ok; idx = idx_n) {
        const BatchItem R = nxt;
        idx_n = iq.pop();
        if (idx_n >= 0) nxt = a.recs[idx_n];
        // the MMA order: groups of CG chromosome tiles, K-blocks, tiles of the group
        for (int c0 = 0; c0 < R.C && ok; c0 += R.CG)
          for (int kb = 0; kb < R.KB && ok; ++kb)
            for (int c = c0; c < c0 + R.CG && c < R.C && ok; ++c) {
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
  } else if (warp == 2) {
    // ---------------- scheduler ----------------
    // Takes items from the global counter into the CTA's queue, up to kQueue
    // ahead of the slowest role, and prefetches each one's features and
    // targets into L2 as it takes it; after the last item, index -1.
    if (lane == 0) {
      for (int seq = 0;; ++seq) {
        const int slot = seq % kQueue;
        if (!wait_bar(ptx::smem_addr(&q_empty[slot]), ((uint32_t)(seq / kQueue) & 1u) ^ 1u,
                      abort_flag, a.status))
          break;
        int k = atomicAdd(a.work, 1);
        if (k >= a.nitems) k = -1;
        qidx[slot] = k;
        ptx::mbar_arrive(ptx::smem_addr(&q_full[slot]));
        if (k < 0) break;
        prefetch_item(a.recs[k]);
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
      uint32_t full_par = 0;   // bit k: parity of the next phi_full[k] phase
      bool ok = true;
      BatchItem nxt;
      int idx_n = iq.pop();
      if (idx_n >= 0) nxt = a.recs[idx_n];
      for (int idx = idx_n; idx >= 0 && ok; idx = idx_n) {
        const BatchItem R = nxt;
        idx_n = iq.pop();
        if (idx_n >= 0) nxt = a.recs[idx_n];
        const int KB = R.KB, C = R.C, BN = R.BN, CG = R.CG, nlast = R.nmma_last;
        const uint32_t idesc = ptx::idesc_bf16_f32(128, BN);
        const uint32_t b_step = (uint32_t)(BN * 128) >> 4;
        const int rmask = R.RK < KB ? R.RK - 1 : -1;   // K-block kb in slot kb & rmask
        auto kblock = [&](uint32_t d_tmem, uint32_t st, int kb, int slot, int nm) {
          const uint64_t ad = adesc0 + st * a_step;
          const uint64_t bd = bdesc0 + (uint32_t)slot * b_step;
          for (int kk = 0; kk < nm; ++kk)
            ptx::mma_bf16(d_tmem, ad + 2u * kk, bd + 2u * kk, idesc, (kb | kk) != 0);
        };
        // Chromosome tiles in groups of CG, each group's accumulators side by
        // side in one accumulator set; per group the K-blocks are the outer
        // loop, so with one group (C <= 256 / BN) a K-block is released as
        // soon as every tile has used it and the next item's expansion
        // follows this item's MMAs K-block by K-block. K-block kb sits in
        // slot kb (ring items, one group by construction: kb mod RK, the
        // expansion refilling slots within the item).
        for (int c0 = 0; c0 < C && ok; c0 += CG) {
          const int c1 = c0 + CG < C ? c0 + CG : C;
          const bool last_group = c1 == C;
          const uint32_t set = acc_it & 1, u = acc_it >> 1;
          ok = wait_bar(acc_empty0 + 8 * set, (u & 1) ^ 1, abort_flag, a.status);
          if (!ok) break;
          ptx::tc_fence_after();
          const uint32_t d_set = tmem + set * (uint32_t)a.set_cols;
          for (int kb = 0; kb < KB && ok; ++kb) {
            const int slot = kb & rmask;
            if (c0 == 0) {
              ok = wait_bar(phi_full0 + 8 * slot, (full_par >> slot) & 1u, abort_flag, a.status);
              full_par ^= 1u << slot;
            }
            for (int c = c0; c < c1 && ok; ++c) {
              ok = wait_bar(a_full0 + 8 * s, ph, abort_flag, a.status);
              if (!ok) break;
              kblock(d_set + (uint32_t)((c - c0) * BN), s, kb, slot, kb == KB - 1 ? nlast : 4);
              ptx::mma_commit(a_empty0 + 8 * s);
              if (++s == (uint32_t)kStages) {
                s = 0;
                ph ^= 1;
              }
            }
            if (ok && last_group) ptx::mma_commit(phi_free0 + 8 * slot);
          }
          if (!ok) break;
          ptx::mma_commit(acc_full0 + 8 * set);
          ++acc_it;
        }
      }
      ptx::mma_commit(ptx::smem_addr(drain));
      wait_bar_drain(ptx::smem_addr(drain), 0, a.status);
    }
  } else if (warp >= kEpiWarp0 && warp < kBasisWarp0) {
    // ---------------- epilogue ----------------
    // Each item's targets are staged in shared memory by the epilogue threads
    // themselves, one item ahead (two slots): thread e loads targets e and
    // e + 128 of the next item while this item's tiles are reduced, stores
    // them afterwards, and the 128 threads meet at named barrier 1. Thread 0
    // alone reads the item queue and hands each index to the others through
    // ebc[] across that barrier, so all 128 walk the same items and pass the
    // same barriers, also after an abort (a thread whose wait failed skips
    // the waits and the work of the remaining items).
    const int qw = warp & 3;
    const int row = qw * 32 + lane;
    const uint32_t lane_addr = (uint32_t)(qw * 32) << 16;
    auto load_y = [&](const BatchItem& R, float& y0, float& y1) {
      const float* yg = R.y + R.m0;
      y0 = row < R.BN ? __ldg(yg + row) : 0.f;
      y1 = row + 128 < R.BN ? __ldg(yg + row + 128) : 0.f;
    };
    if (row == 0) ebc[0] = iq.pop();
    ptx::named_bar(1, kEpiThreads);
    int idx = ebc[0];
    BatchItem nxt;
    if (idx >= 0) {
      nxt = a.recs[idx];
      float y0, y1;
      load_y(nxt, y0, y1);
      ys[row] = y0;
      ys[row + 128] = y1;
    }
    if (row == 0) ebc[1] = idx >= 0 ? iq.pop() : -1;
    ptx::named_bar(1, kEpiThreads);
    uint32_t acc_it = 0;
    bool ok = true;
    for (int k = 0; idx >= 0; ++k) {
      const BatchItem R = nxt;
      const int idx_n = ebc[(k + 1) & 1];
      float yn0 = 0.f, yn1 = 0.f;
      if (idx_n >= 0) {
        nxt = a.recs[idx_n];
        load_y(nxt, yn0, yn1);
      }
      const float* yt = ys + (k & 1) * kYSlot;
      const int valid = R.valid;
      double* prow = R.prow;
      uint32_t set = 0;
      for (int c = 0; c < R.C && ok; ++c) {
        const int cg = c % R.CG;   // place in the accumulator set
        if (cg == 0) {
          set = acc_it & 1;
          ok = wait_bar(ptx::smem_addr(&acc_full[set]), (acc_it >> 1) & 1, abort_flag, a.status);
          if (!ok) break;
          ptx::tc_fence_after();
        }
        const int chrom = c * 128 + row;
        const float bias = R.a0[chrom];
        const uint64_t bias2 = ptx::f2_pack(bias, bias);
        uint64_t s2 = 0;
        float s_tail = 0.f;
        const uint32_t tbase =
            tmem + lane_addr + set * (uint32_t)a.set_cols + (uint32_t)(cg * R.BN);
        const int nfull = valid / 32;
        if (nfull > 0) {
          uint32_t va[32], vb[32];
          ptx::tmem_ld32_issue(tbase, va);
          ptx::tmem_ld32_wait(va);
          for (int k = 0; k < nfull; k += 2) {
            const bool has_b = k + 1 < nfull;
            if (has_b) ptx::tmem_ld32_issue(tbase + (uint32_t)(k + 1) * 32, vb);
            epi_chunk_smem(va, yt + k * 32, bias2, s2);
            if (has_b) {
              ptx::tmem_ld32_wait(vb);
              const bool has_a = k + 2 < nfull;
              if (has_a) ptx::tmem_ld32_issue(tbase + (uint32_t)(k + 2) * 32, va);
              epi_chunk_smem(vb, yt + (k + 1) * 32, bias2, s2);
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
        if (cg == R.CG - 1 || c == R.C - 1) {   // the set's last tile: release it
          ptx::tc_fence_before();
          ptx::mbar_arrive(ptx::smem_addr(&acc_empty[set]));
          ++acc_it;
        }
        const float2 sp2 = ptx::f2_unpack(s2);
        prow[chrom] = (double)sp2.x + (double)sp2.y + (double)s_tail;
      }
      float* ynext = ys + ((k + 1) & 1) * kYSlot;
      ynext[row] = yn0;
      ynext[row + 128] = yn1;
      if (row == 0) ebc[k & 1] = idx_n >= 0 ? iq.pop() : -1;   // item k + 2
      ptx::named_bar(1, kEpiThreads);
      idx = idx_n;
    }
  } else if (warp >= kBasisWarp0) {
    // ---------------- expansion (basis) ----------------
    // Slot k of an item sits at k * BN * 128, so when BN changes from one
    // item to the next a new slot can overlap any slot of the previous
    // layout: then every outstanding phi_free phase is awaited before the
    // first store (the item list runs by tile width, so this happens at most
    // three times per CTA).
    const int bt = threadIdx.x - kBasisWarp0 * 32;
    ExpState es{0u, 0u, 0};
    const ExpEnv env{ptx::smem_addr(phi), ptx::smem_addr(ring), ptx::smem_addr(phi_full),
                     ptx::smem_addr(phi_free), abort_flag, a.status};
    int prev_bn = 0;
    BatchItem nxt;
    int idx_n = iq.pop();
    if (idx_n >= 0) nxt = a.recs[idx_n];
    for (int idx = idx_n; idx >= 0 && !es.dead; idx = idx_n) {
      const BatchItem R = nxt;
      idx_n = iq.pop();
      if (idx_n >= 0) nxt = a.recs[idx_n];
      const int BN = R.BN;
      if (BN != prev_bn) await_mask(es, env, 0xFFFFFFFFu);
      prev_bn = BN;
      // BN rows, QS = 256 / BN threads per row (thread bt: row bt % BN, range bt / BN)
      const int QS = kBasisThreads / BN, r0 = bt % BN, q0 = bt / BN;
      const int64_t m = R.m0 + r0;
      const float* xp = R.Xt + (m / kPatBlock) * R.N * kPatBlock + (m % kPatBlock);
      es = (R.basis == GAME_BASIS_CHEB)
               ? expand_dispatch<GAME_BASIS_CHEB>(es, env, xp, R, r0, q0, QS, bt)
               : expand_dispatch<GAME_BASIS_TRIG>(es, env, xp, R, r0, q0, QS, bt);
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

int batch_smem_bytes(int phi_bytes, int KBmax) {
  return bsmem_plan(phi_bytes, KBmax).total;
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
