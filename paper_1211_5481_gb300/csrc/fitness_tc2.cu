// fitness_tc2.cu -- the BF16 fitness contraction on pairs of SMs
// (tcgen05 cta_group::2), the squared- or absolute-error reduction fused into
// the epilogue.
//
// Math (paper Section 3): Out_p(m) = a_{p,0} + sum_c a_{p,c+1} phi_c(x_m)
// (Eq. 2), fit_p = (1/M) sum_m (y_m - Out_p(m))^2 (Eq. 3, MSE). For a tile of
// 256 patterns the sum over c is the dense product D[p][m] = A[p][:] . PHI[m][:].
//
// A cluster of two CTAs (one per SM of a pair) computes D for 256 chromosomes
// (MMA-M, 128 per CTA: the rows of each CTA's tensor memory) x 256 patterns
// (MMA-N) with one tcgen05.mma.cta_group::2 per K = 16 step, issued by one
// thread of the even CTA: each CTA holds in its shared memory the genes of
// its 128 chromosomes and the expansion of its 128 patterns (half of B), so
// per MMA each SM reads half the operand bytes of a one-SM 128 x 256 MMA,
// and each SM expands only its own 128 patterns of a tile.
//
// Warp roles in each CTA (16 warps):
//   warp 0       gene producer: bulk copies of this CTA's 16 KB gene blocks
//                (chromosome tile 2c + rank, K-block kb) into a ring of stages.
//   warp 1       even CTA: MMA issuer (one thread); both CTAs: tensor-memory
//                allocation of the pair (512 columns: two accumulators of 256).
//   warp 2       feature producer (staged features only): this CTA's
//                128-pattern feature block of the next tile.
//   warp 3       odd CTA: relays the completion of its gene copies to the even
//                CTA's stage barrier (the copy's own barrier is local).
//   warps 4-11   epilogue: tcgen05.ld of this CTA's 128 accumulator rows
//                (warps 4-7 the first 128 pattern columns, 8-11 the second),
//                r = (y_m - a_0) - D, sse += r^2 in packed FP32 pairs, FP64
//                partials per (cluster, column half).
//   warps 12-15  expansion: thread = one of this CTA's 128 patterns; per 8-column
//                chunk the basis recurrence in registers, BF16, stored in the
//                K-major SWIZZLE_128B layout, into a ring of K-block slots.
// Barriers: the MMA issuer waits on the even CTA's barriers only; the odd
// CTA's producers reach them by cluster-scope arrivals (one per warp for the
// expansion and the epilogue, one relay per gene stage); every MMA commit is
// multicast to the same barrier in both CTAs, so each CTA's producers and
// epilogue wait on their own copies. All waits are bounded (2 s): on expiry a
// CTA raises the status word, abandons its loops, drains its own copies (the
// even CTA its MMAs), and both CTAs meet at the final cluster barrier before
// the pair's tensor memory is freed.
#include "basis.cuh"
#include "game_internal.cuh"
#include "tc_common.cuh"
#include "tc_ptx.cuh"

namespace game {

namespace {

using namespace tc;

constexpr uint32_t kABytes = 128 * 128;   // one CTA's gene block: 128 chromosomes x 64 genes
constexpr int kWarps = 16;
constexpr int kThreads = kWarps * 32;
constexpr int kEpiWarp0 = 4;
constexpr int kBasisWarp0 = 12;
constexpr int kBasisThreads = 128;
constexpr int kRows = 128;                // patterns of a tile held by one CTA
constexpr int kBN = 2 * kRows;            // patterns per tile (MMA N)
constexpr int kMaxSmem = 232448;          // 227 KB opt-in per CTA
constexpr int kMinSmem = 120 * 1024;      // one CTA per SM
constexpr uint32_t kPhiArrivals = 8;      // expansion warps of both CTAs
constexpr uint32_t kAccArrivals = 16;     // epilogue warps of both CTAs

struct Tc2Args {
  int64_t M;
  int N, d, basis, Kp;
  int KB, Cp, NS, stages, nmma_last, ntiles, Ppad, xstage;
  const float* Xt;
  const float* y;
  const uint8_t* popA;
  const float* a0;
  double* part;
  int* status;
  uint64_t stall_ns;   // test hook (see fitness_tc.cu)
};

struct Smem2 {
  int phi, ast, xs, tab, bars, total;
};

__host__ __device__ inline int num_bars2(int NS, int S) { return 2 * S + 2 * NS + 7; }

__host__ __device__ inline Smem2 smem_plan2(int KB, int NS, int N, int S, int xstage) {
  Smem2 s;
  s.phi = 0;
  s.ast = NS * kRows * 128;
  s.xs = s.ast + S * (int)kABytes;
  s.tab = s.xs + (xstage ? N * kRows * 4 : 0);
  s.bars = (s.tab + KB * 8 * 4 + 7) & ~7;
  s.total = s.bars + num_bars2(NS, S) * 8 + 16 + 1024;   // + alignment slack
  return s;
}

// The 8 expansion values of chunk `desc` for one pattern whose features are
// xrow[i * xstride]: the same values as gen_chunk, with the Chebyshev run of
// one feature's degrees and the crossing chunks of d >= 4 on their
// branch-free generators.
__device__ __forceinline__ void gen8(uint32_t desc, int basis, int d, int N, const float* xrow,
                                     int xstride, float (&v)[8]) {
  if (basis == GAME_BASIS_CHEB && (desc & kChunkRun) && ((desc >> 24) & 15u) == 8u) {
    const int i = (int)(desc & 0xFFFFu);
    const int j0 = (int)((desc >> 16) & 31u);
    const float x = xrow[i * xstride];
    const float x2 = x + x;
    float t = x, tm = 1.f;
    for (int st = 1; st < j0; ++st) {
      const float n = fmaf(x2, t, -tm);
      tm = t;
      t = n;
    }
    v[0] = t;
#pragma unroll
    for (int e = 1; e < 8; ++e) {
      const float n = fmaf(x2, t, -tm);
      tm = t;
      t = n;
      v[e] = t;
    }
  } else if (basis == GAME_BASIS_CHEB && d >= 4 && !(desc & kChunkZero)) {
    cheb_cross1(desc, d, N, xrow, xstride, v);
  } else {
    gen_chunk(desc, basis, d, N, xrow, xstride, v);
  }
}

__device__ __forceinline__ void store_bf16x8(uint8_t* phik, int r, int qd, const float (&v)[8]) {
  *reinterpret_cast<uint4*>(phik + r * 128 + ((qd ^ (r & 7)) << 4)) =
      make_uint4(bf16x2_bits(v[0], v[1]), bf16x2_bits(v[2], v[3]), bf16x2_bits(v[4], v[5]),
                 bf16x2_bits(v[6], v[7]));
}

// Two Chebyshev runs of 8 degrees (chunks of the features xa and xb, first
// degrees ja and jb), interleaved: two independent recurrences.
__device__ __forceinline__ void cheb_run_pair(float xa, int ja, float xb, int jb, float (&va)[8],
                                              float (&vb)[8]) {
  const float a2 = xa + xa, b2 = xb + xb;
  float ta = xa, tam = 1.f, tb = xb, tbm = 1.f;
  for (int st = 1; st < ja; ++st) {
    const float n = fmaf(a2, ta, -tam);
    tam = ta;
    ta = n;
  }
  for (int st = 1; st < jb; ++st) {
    const float n = fmaf(b2, tb, -tbm);
    tbm = tb;
    tb = n;
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
}

template <bool ABS>
__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(kThreads, 1)
    fitness_tc2_kernel(const Tc2Args a) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* base = reinterpret_cast<uint8_t*>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~static_cast<uintptr_t>(1023));
  const int KB = a.KB, N = a.N, S = a.stages, NS = a.NS;
  const Smem2 sp = smem_plan2(KB, NS, N, S, a.xstage);
  uint8_t* phi = base + sp.phi;
  uint8_t* ast = base + sp.ast;
  float* xs = reinterpret_cast<float*>(base + sp.xs);
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
  uint32_t* tmem_holder = reinterpret_cast<uint32_t*>(drain + 1);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_holder + 1);

  const uint32_t rank = ptx::cluster_ctarank();
  const bool lead = rank == 0;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (int s = 0; s < S; ++s) {
      // the even CTA's stage completes on its own copy and the odd CTA's relay
      ptx::mbar_init(ptx::smem_addr(&a_full[s]), lead ? 2 : 1);
      ptx::mbar_init(ptx::smem_addr(&a_empty[s]), 1);
    }
    for (int sl = 0; sl < NS; ++sl) {
      ptx::mbar_init(ptx::smem_addr(&phi_full[sl]), kPhiArrivals);
      ptx::mbar_init(ptx::smem_addr(&phi_free[sl]), 1);
    }
    for (int b = 0; b < 2; ++b) {
      ptx::mbar_init(ptx::smem_addr(&acc_full[b]), 1);
      ptx::mbar_init(ptx::smem_addr(&acc_empty[b]), kAccArrivals);
    }
    ptx::mbar_init(ptx::smem_addr(x_full), 1);
    ptx::mbar_init(ptx::smem_addr(x_empty), kBasisThreads);
    ptx::mbar_init(ptx::smem_addr(drain), 1);
    *abort_flag = 0;
    ptx::fence_mbar_init();
    ptx::fence_proxy_async_smem();
  }
  if (warp == 1) {
    ptx::tmem_alloc2(ptx::smem_addr(tmem_holder), 512u);
    ptx::tmem_relinquish2();
  }
  ptx::tc_fence_before();
  __syncthreads();
  ptx::cluster_sync();   // the peer's barriers exist before any arrival on them
  ptx::tc_fence_after();
  const uint32_t tmem = *tmem_holder;

  const int ncl = (int)(gridDim.x >> 1), cl = (int)(blockIdx.x >> 1);
  const int my_tiles = (a.ntiles - cl + ncl - 1) / ncl;
  const int Cp = a.Cp;

  if (warp == 0) {
    // ---------------- gene producer (both CTAs) ----------------
    if (lane == 0) {
      uint32_t q = 0, s = 0, ph = 0;
      bool ok = true;
      for (int it = 0; it < my_tiles && ok; ++it)
        for (int c = 0; c < Cp && ok; ++c)
          for (int kb = 0; kb < KB && ok; ++kb) {
            ok = wait_bar(ptx::smem_addr(&a_empty[s]), ph ^ 1, abort_flag, a.status);
            if (!ok) break;
            ptx::mbar_arrive_expect_tx(ptx::smem_addr(&a_full[s]), kABytes);
            ptx::bulk_g2s(ptx::smem_addr(ast + s * kABytes),
                          a.popA + ((size_t)(2 * c + (int)rank) * KB + kb) * kABytes, kABytes,
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
    // ---------------- MMA issuer (even CTA) ----------------
    if (lane == 0 && lead) {
      const uint32_t idesc = ptx::idesc_bf16_f32(2 * kRows, kBN);
      const uint64_t adesc0 = ptx::desc_kmajor_sw128(ptx::smem_addr(ast));
      const uint64_t bdesc0 = ptx::desc_kmajor_sw128(ptx::smem_addr(phi));
      const uint32_t a_step = kABytes >> 4;
      const uint32_t b_step = (uint32_t)(kRows * 128) >> 4;
      const uint32_t a_full0 = ptx::smem_addr(a_full), a_empty0 = ptx::smem_addr(a_empty);
      const uint32_t phi_full0 = ptx::smem_addr(phi_full), phi_free0 = ptx::smem_addr(phi_free);
      const uint32_t acc_full0 = ptx::smem_addr(acc_full), acc_empty0 = ptx::smem_addr(acc_empty);
      const uint16_t both = 3;
      const int nlast = a.nmma_last;
      uint32_t s = 0, ph = 0, acc_it = 0;
      bool ok = true;
      if (a.stall_ns) {
        // test hook: the drain barrier's first phase completes only at the
        // final commit below, so this wait runs out
        const uint64_t t0 = ptx::global_timer_ns();
        while (ok && !ptx::mbar_try_wait_sleep(ptx::smem_addr(drain), 0, kSuspendNs)) {
          if (ptx::global_timer_ns() - t0 > a.stall_ns) {
            *abort_flag = 1;
            atomicExch(a.status, (int)kDevTimeout);
            ok = false;
          }
        }
      }
      auto kblock = [&](uint32_t d_tmem, uint32_t st, int kb, int slot, int nm) {
        const uint64_t ad = adesc0 + st * a_step;
        const uint64_t bd = bdesc0 + (uint32_t)slot * b_step;
        if (nm == 4) {
          ptx::mma_bf16_pair(d_tmem, ad, bd, idesc, kb != 0);
          ptx::mma_bf16_pair(d_tmem, ad + 2u, bd + 2u, idesc, 1u);
          ptx::mma_bf16_pair(d_tmem, ad + 4u, bd + 4u, idesc, 1u);
          ptx::mma_bf16_pair(d_tmem, ad + 6u, bd + 6u, idesc, 1u);
        } else {
          for (int kk = 0; kk < nm; ++kk)
            ptx::mma_bf16_pair(d_tmem, ad + 2u * kk, bd + 2u * kk, idesc, (kb | kk) != 0);
        }
      };
      for (int it = 0; it < my_tiles && ok; ++it) {
        for (int c = 0; c < Cp && ok; ++c) {
          const uint32_t buf = acc_it & 1, u = acc_it >> 1;
          ok = wait_bar(acc_empty0 + 8 * buf, (u & 1) ^ 1, abort_flag, a.status);
          if (!ok) break;
          ptx::tc_fence_after();
          const uint32_t d_tmem = tmem + buf * (uint32_t)kBN;
          for (int kb = 0; kb < KB && ok; kb += (c != 0 && kb + 1 < KB) ? 2 : 1) {
            const bool two = c != 0 && kb + 1 < KB;
            uint32_t s1 = s + 1, ph1 = ph;
            if (s1 == (uint32_t)S) {
              s1 = 0;
              ph1 ^= 1;
            }
            const int q0 = it * KB + kb, q1 = q0 + 1;
            const int sl0 = q0 % NS, sl1 = q1 % NS;
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
            ptx::mma_commit_pair_mc(a_empty0 + 8 * s, both);
            if (two) ptx::mma_commit_pair_mc(a_empty0 + 8 * s1, both);
            if (c == Cp - 1) {
              ptx::mma_commit_pair_mc(phi_free0 + 8 * sl0, both);
              if (two) ptx::mma_commit_pair_mc(phi_free0 + 8 * sl1, both);
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
          ptx::mma_commit_pair_mc(acc_full0 + 8 * buf, both);
          ++acc_it;
        }
      }
      // every MMA issued above has completed once this arrives
      ptx::mma_commit_pair(ptx::smem_addr(drain));
      wait_bar_drain(ptx::smem_addr(drain), 0, a.status);
    }
  } else if (warp == 2) {
    // ---------------- feature producer (staged features only) ----------------
    if (lane == 0 && a.xstage) {
      int issued = 0;
      const uint32_t bytes = (uint32_t)(N * kRows * 4);
      for (int it = 0; it < my_tiles; ++it) {
        const int64_t t = (int64_t)cl + (int64_t)it * ncl;
        if (!wait_bar(ptx::smem_addr(x_empty), (it & 1) ^ 1, abort_flag, a.status)) break;
        ptx::mbar_arrive_expect_tx(ptx::smem_addr(x_full), bytes);
        const int64_t blk = t * 2 + rank;   // this CTA's 128-pattern block
        ptx::bulk_g2s(ptx::smem_addr(xs), a.Xt + blk * N * kPatBlock, bytes,
                      ptx::smem_addr(x_full));
        if (it + 1 < my_tiles)
          ptx::bulk_prefetch_l2(a.Xt + ((t + ncl) * 2 + rank) * N * kPatBlock, bytes);
        ++issued;
      }
      if (issued > 0) wait_bar_drain(ptx::smem_addr(x_full), (issued - 1) & 1, a.status);
    }
  } else if (warp == 3) {
    // ---------------- odd CTA: relay of gene-copy completions ----------------
    if (lane == 0 && !lead) {
      const int total = my_tiles * Cp * KB;
      uint32_t s = 0, ph = 0;
      int done = 0;
      for (; done < total; ++done) {
        if (!wait_bar(ptx::smem_addr(&a_full[s]), ph, abort_flag, a.status)) break;
        ptx::mbar_arrive_cluster(ptx::mapa(ptx::smem_addr(&a_full[s]), 0));
        if (++s == (uint32_t)S) {
          s = 0;
          ph ^= 1;
        }
      }
    }
  } else if (warp >= kEpiWarp0 && warp < kBasisWarp0) {
    // ---------------- epilogue (both CTAs) ----------------
    const int qw = warp & 3;
    const int half = (warp - kEpiWarp0) >> 2;
    const int row = qw * 32 + lane;
    const int col_lo = half * kRows;
    const uint32_t lane_addr = (uint32_t)(qw * 32) << 16;
    double* part_row = a.part + (size_t)(2 * cl + half) * a.Ppad;
    const uint32_t acc_empty_lead0 = ptx::mapa(ptx::smem_addr(acc_empty), 0);
    uint32_t acc_it = 0;
    bool ok = true;
    for (int it = 0; it < my_tiles && ok; ++it) {
      const int64_t m0 = ((int64_t)cl + (int64_t)it * ncl) * kBN;
      const int64_t rem = a.M - m0 - col_lo;
      const int valid = rem <= 0 ? 0 : (rem >= kRows ? kRows : (int)rem);
      const float* yt = a.y + m0 + col_lo;
      for (int c = 0; c < Cp; ++c) {
        const uint32_t buf = acc_it & 1, u = acc_it >> 1;
        ok = wait_bar(ptx::smem_addr(&acc_full[buf]), u & 1, abort_flag, a.status);
        if (!ok) break;
        ptx::tc_fence_after();
        const int chrom = c * 2 * kRows + (int)rank * kRows + row;
        const float bias = a.a0[chrom];
        const uint64_t bias2 = ptx::f2_pack(bias, bias);
        const uint64_t negu2 = ptx::f2_pack(-1.f, -1.f);
        uint64_t s2 = 0;
        float s_tail = 0.f;
        const uint32_t tbase = tmem + lane_addr + buf * (uint32_t)kBN + (uint32_t)col_lo;
        const int nfull = valid / 32;
        if (nfull > 0) {
          uint32_t va[32], vb[32];
          ptx::tmem_ld32_issue(tbase, va);
          ptx::tmem_ld32_wait(va);
          for (int k = 0; k < nfull; k += 2) {
            const bool has_b = k + 1 < nfull;
            if (has_b) ptx::tmem_ld32_issue(tbase + (uint32_t)(k + 1) * 32, vb);
            epi_chunk<false, ABS>(va, yt + k * 32, bias2, negu2, s2);
            if (has_b) {
              ptx::tmem_ld32_wait(vb);
              const bool has_a = k + 2 < nfull;
              if (has_a) ptx::tmem_ld32_issue(tbase + (uint32_t)(k + 2) * 32, va);
              epi_chunk<false, ABS>(vb, yt + (k + 1) * 32, bias2, negu2, s2);
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
              const float r = (yt[nfull * 32 + e] - bias) - __uint_as_float(v[e]);
              s_tail = ABS ? s_tail + fabsf(r) : fmaf(r, r, s_tail);
            }
          }
        }
        ptx::tc_fence_before();
        __syncwarp();
        if (lane == 0) ptx::mbar_arrive_cluster(acc_empty_lead0 + 8 * buf);
        const float2 sp2 = ptx::f2_unpack(s2);
        const double tile_sse = (double)sp2.x + (double)sp2.y + (double)s_tail;
        part_row[chrom] = (it == 0) ? tile_sse : part_row[chrom] + tile_sse;
        ++acc_it;
      }
    }
  } else {
    // ---------------- expansion (both CTAs) ----------------
    const int r0 = threadIdx.x - kBasisWarp0 * 32;   // this thread's pattern row
    for (int cid = r0; cid < KB * 8; cid += kBasisThreads)
      tab[cid] = chunk_desc(cid, a.basis, a.d, a.Kp);
    ptx::named_bar(1, kBasisThreads);
    const uint32_t phi_full_lead0 = ptx::mapa(ptx::smem_addr(phi_full), 0);
    auto slot_free = [&](int q) -> bool {
      const int use = q / NS;
      return use == 0 ||
             wait_bar(ptx::smem_addr(&phi_free[q % NS]), (use - 1) & 1, abort_flag, a.status);
    };
    auto publish = [&](int q) {
      ptx::fence_proxy_async_smem();
      __syncwarp();
      if (lane == 0) ptx::mbar_arrive_cluster(phi_full_lead0 + 8 * (q % NS));
    };
    bool ok = true;
    if (!a.xstage) {
      // Chebyshev runs of 8 degrees, features read from global memory (L2):
      // the x of a K-block's 8 chunks are loaded one K-block ahead; thread 0
      // prefetches this CTA's feature block of the tile after next into L2
      auto xptr = [&](int itn) -> const float* {
        const int64_t blk = ((int64_t)cl + (int64_t)itn * ncl) * 2 + rank;
        return a.Xt + blk * (int64_t)N * kPatBlock + r0;
      };
      auto prefetch_tile = [&](int itn) {
        const int64_t blk = ((int64_t)cl + (int64_t)itn * ncl) * 2 + rank;
        ptx::bulk_prefetch_l2(a.Xt + blk * N * kPatBlock, (uint32_t)(N * kPatBlock * 4));
      };
      float nx[8];
      auto load_kb = [&](int itn, int kbn) {
        const float* p = xptr(itn);
#pragma unroll
        for (int q = 0; q < 8; ++q) nx[q] = __ldg(p + (int)(tab[kbn * 8 + q] & 0xFFFFu) * kPatBlock);
      };
      if (r0 == 0) {
        if (my_tiles > 0) prefetch_tile(0);
        if (my_tiles > 1) prefetch_tile(1);
      }
      if (my_tiles > 0) load_kb(0, 0);
      for (int it = 0; it < my_tiles && ok; ++it) {
        if (r0 == 0 && it + 2 < my_tiles) prefetch_tile(it + 2);
        for (int kb = 0; kb < KB; ++kb) {
          float x[8];
#pragma unroll
          for (int q = 0; q < 8; ++q) x[q] = nx[q];
          if (kb + 1 < KB) load_kb(it, kb + 1);
          else if (it + 1 < my_tiles) load_kb(it + 1, 0);
          const int q = it * KB + kb;
          ok = slot_free(q);
          if (!ok) break;
          uint8_t* phik = phi + (size_t)(q % NS) * kRows * 128;
#pragma unroll
          for (int qd = 0; qd < 8; qd += 2) {
            const uint32_t da = tab[kb * 8 + qd], db = tab[kb * 8 + qd + 1];
            float va[8], vb[8];
            cheb_run_pair(x[qd], (int)((da >> 16) & 31u), x[qd + 1], (int)((db >> 16) & 31u),
                          va, vb);
            if (da & kChunkZero) {
#pragma unroll
              for (int e = 0; e < 8; ++e) va[e] = 0.f;
            }
            if (db & kChunkZero) {
#pragma unroll
              for (int e = 0; e < 8; ++e) vb[e] = 0.f;
            }
            store_bf16x8(phik, r0, qd, va);
            store_bf16x8(phik, r0, qd + 1, vb);
          }
          publish(q);
        }
      }
    } else {
      const float* xrow = xs + r0;   // block layout [N][128]
      for (int it = 0; it < my_tiles && ok; ++it) {
        ok = wait_bar(ptx::smem_addr(x_full), it & 1, abort_flag, a.status);
        if (!ok) break;
        for (int kb = 0; kb < KB; ++kb) {
          const int q = it * KB + kb;
          ok = slot_free(q);
          if (!ok) break;
          uint8_t* phik = phi + (size_t)(q % NS) * kRows * 128;
#pragma unroll 1
          for (int qd = 0; qd < 8; qd += 2) {
            float va[8], vb[8];
            gen8(tab[kb * 8 + qd], a.basis, a.d, N, xrow, kRows, va);
            gen8(tab[kb * 8 + qd + 1], a.basis, a.d, N, xrow, kRows, vb);
            store_bf16x8(phik, r0, qd, va);
            store_bf16x8(phik, r0, qd + 1, vb);
          }
          publish(q);
        }
        if (!ok) break;
        ptx::mbar_arrive(ptx::smem_addr(x_empty));
      }
    }
  }

  ptx::tc_fence_before();
  __syncthreads();
  ptx::cluster_sync();   // the pair's MMAs, loads and remote arrivals are over
  if (warp == 1) {
    ptx::tc_fence_after();
    ptx::tmem_dealloc2(tmem, 512u);
  }
}

}  // namespace

TcPlan plan_tc_pair(const Shape& s, int P, int num_sms) {
  TcPlan pl{};
  pl.form = kFormBF16;
  pl.pair = 1;
  pl.KB = ceil_div(s.Kp, 64);
  pl.C = 2 * ceil_div(P, kBN);
  pl.BN = kBN;
  pl.ok = false;
  if (num_sms < 2) return pl;
  // features from L2 for Chebyshev runs of 8 degrees (the x of a chunk is one
  // load), else staged
  const int xstage = (s.basis == GAME_BASIS_CHEB && s.d % 8 == 0) ? 0 : 1;
  for (int stages = 4; stages >= 3 && !pl.ok; --stages)
    for (int NS = 2 * pl.KB; NS >= pl.KB && !pl.ok; --NS) {
      const int sm = smem_plan2(pl.KB, NS, s.N, stages, xstage).total;
      if (sm <= kMaxSmem) {
        pl.NS = NS;
        pl.stages = stages;
        pl.xstage = xstage;
        pl.smem_bytes = sm < kMinSmem ? kMinSmem : sm;
        pl.ok = true;
      }
    }
  if (!pl.ok) return pl;
  const int ntiles = ceil_div(s.M, kBN);
  const int clusters = ntiles < num_sms / 2 ? ntiles : num_sms / 2;
  pl.grid = 2 * clusters;
  pl.tmem_cols = 512;
  pl.rows = 2 * clusters;   // one partial row per (cluster, column half)
  return pl;
}

cudaError_t launch_fitness_tc_pair(const TcPlan& pl, const Shape& s, const float* Xt,
                                   const float* y, const uint8_t* popA, const float* a0, int Ppad,
                                   double* part, int* status, int err, cudaStream_t st) {
  if (!pl.ok || !pl.pair || pl.form != kFormBF16) return cudaErrorInvalidValue;
  if (pl.NS < pl.KB || pl.NS > 2 * pl.KB || pl.grid % 2 != 0 || Ppad < pl.C * 128)
    return cudaErrorInvalidValue;
  Tc2Args a;
  a.M = s.M;
  a.N = s.N;
  a.d = s.d;
  a.basis = s.basis;
  a.Kp = s.Kp;
  a.KB = pl.KB;
  a.Cp = pl.C / 2;
  a.NS = pl.NS;
  a.stages = pl.stages;
  a.xstage = pl.xstage;
  const int last_cols = s.Kp - 64 * (pl.KB - 1);
  a.nmma_last = (last_cols + 15) / 16;
  a.ntiles = ceil_div(s.M, kBN);
  a.Ppad = Ppad;
  a.Xt = Xt;
  a.y = y;
  a.popA = popA;
  a.a0 = a0;
  a.part = part;
  a.status = status;
  a.stall_ns = hook_take_stall_ns();
  void (*kern)(const Tc2Args) =
      err == GAME_ERR_MAE ? fitness_tc2_kernel<true> : fitness_tc2_kernel<false>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       pl.smem_bytes);
  if (e != cudaSuccess) return e;
  kern<<<pl.grid, kThreads, pl.smem_bytes, st>>>(a);
  return cudaGetLastError();
}

}  // namespace game
