// surrogate.cu -- a small MLP that predicts a chromosome's fitness, trained
// online on the (chromosome, exact fitness) pairs the GA produces, and used to
// screen oversampled offspring so that only the most promising get the exact
// fitness of paper Section 3 (Eq. 2, Eq. 3).
//
// Network: x in R^K (the genes) -> 256 -> 256 -> 1. Layers 1 and 2 take BF16
// operands (inputs, weights and the layer-1 activations rounded to BF16) with
// FP32 accumulation; the output layer is FP32. Activation: GELU in its tanh
// form, g(z) = z/2 (1 + tanh(c (z + 0.044715 z^3))), c = sqrt(2/pi). Target:
// the log-fitness l = log(max(fit, 1e-30)) standardised over the training
// batch, t = (l - mean l) / sd l (FP64 statistics; sd 0 counts as 1): the
// MSE spans orders of magnitude and only the ranking of the prediction is
// used. Loss: mean of (out - t)^2 over the batch. Optimiser: Adam (lr 1e-3, beta1 0.9, beta2 0.999, eps 1e-8) on FP32
// master weights. Initial weights uniform in +-1/sqrt(fan_in) from
// Philox4x32-10 (key = seed, counter = (layer, index, 0, tag 9)), biases 0.
//
// Parameter vector (FP32, this order): W1 [256][K], b1 [256], W2 [256][256],
// b2 [256], w3 [256], b3 [1].
//
// Kernels: one tensor-core GEMM with strides (C = A B with any transposition,
// BF16 operands -- FP32 ones split into BF16 hi + lo -- with FP32
// accumulation in tensor memory, an optional bias + GELU epilogue), column sums in a fixed order, the GELU
// derivative, the output layer, and Adam. Screening: a one-CTA bitonic sort
// of (prediction, slot) keys, a flag per kept slot and a prefix-sum
// compaction that assembles the next population in slot order. The exact
// fitness checks the surrogate: after each screened generation the Pearson
// correlation r of the kept children's predictions with their exact
// log-fitness is measured, and the next screening trusts the surrogate only
// if r > 0.25; otherwise it keeps the first P - E children, i.e. exactly the
// children of the unscreened generation.
#include <cuda_bf16.h>

#include "game_internal.cuh"
#include "philox.cuh"

namespace game {

namespace {

constexpr int kH = kSurrogateHidden;
constexpr float kGeluC = 0.7978845608028654f;   // sqrt(2 / pi)
constexpr float kGeluA = 0.044715f;

__device__ __forceinline__ float round_bf16(float x) {
  return __bfloat162float(__float2bfloat16_rn(x));
}

__device__ __forceinline__ float gelu(float z) {
  const float u = kGeluC * (z + kGeluA * z * z * z);
  return 0.5f * z * (1.f + tanhf(u));
}

__device__ __forceinline__ float gelu_grad(float z) {
  const float u = kGeluC * (z + kGeluA * z * z * z);
  const float t = tanhf(u);
  return 0.5f * (1.f + t) + 0.5f * z * (1.f - t * t) * kGeluC * (1.f + 3.f * kGeluA * z * z);
}

// C[m][n] = sum_k A(m, k) B(k, n), A(m, k) = A[m * am + k * ak], B(k, n) =
// B[k * bk + n * bn], on the tensor cores (tcgen05, FP32 accumulation in tensor
// memory). Operands flagged for rounding enter as their BF16 values; the
// others (FP32 gradients) as hi = bf16(v) plus lo = bf16(v - hi), with the
// MMAs hi*hi + hi*lo + lo*hi, so products lose at most ~2^-16 of their
// value. CTA tile: 128 rows of C (MMA-M, tensor-memory lanes) x TN columns
// (MMA-N); K in blocks of 64 through a double-buffered shared-memory ring in
// the K-major SWIZZLE_128B layout, filled by all 256 threads (g_load),
// consumed by MMAs issued by thread 0;
// the epilogue reads the accumulator rows back (thread = row of C). Split-K:
// blockIdx.z takes k-range [z * kz, (z + 1) * kz) and, with splits > 1, writes
// its partial product to C + z * M * ldc (reduced in order by splitk_reduce).
// Epilogue modes (splits == 1): 0 store C; 1 store Z = C + bias[n] to C and
// g(Z) (BF16-rounded when round_out) to out2; 2 store C + bias[n].
// Waits are bounded (1 s): an expired wait abandons the tile and raises
// *status.
constexpr int kGTK = 64;                  // K per block (128 bytes of BF16 per row)
constexpr uint32_t kGemmWaitNs = 1000000000ull;

__device__ __forceinline__ uint32_t g_smem(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ bool g_wait(uint32_t bar, uint32_t parity, int* status) {
  uint32_t ok = 0;
  uint64_t t0 = 0;
  for (int it = 0;; ++it) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    if (ok) return true;
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    if (it == 0) t0 = t;
    else if (t - t0 > kGemmWaitNs) {
      atomicExch(status, 1);
      return false;
    }
  }
}

__device__ __forceinline__ uint64_t g_desc(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
  d |= (uint64_t)1 << 16;
  d |= (uint64_t)(1024u >> 4) << 32;
  d |= (uint64_t)1 << 46;
  d |= (uint64_t)2 << 61;
  return d;
}

__device__ __forceinline__ void g_mma(uint32_t d_tmem, uint64_t ad, uint64_t bd, uint32_t idesc,
                                      uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
      "l"(ad), "l"(bd), "r"(idesc), "r"(acc)
      : "memory");
}

__device__ __forceinline__ uint32_t bf16pair(float lo, float hi) {
  const __nv_bfloat162 b = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<const uint32_t*>(&b);
}

// 8 consecutive k of one row into the swizzled image (hi, and lo when split)
__device__ __forceinline__ void g_store8(uint8_t* img, uint8_t* img_lo, int r, int qd,
                                         const float (&v)[8], bool split) {
  const int off = r * 128 + ((qd ^ (r & 7)) << 4);
  uint32_t h[4], l[4];
#pragma unroll
  for (int e = 0; e < 4; ++e) {
    h[e] = bf16pair(v[2 * e], v[2 * e + 1]);
    if (split) {
      const __nv_bfloat162 hb = *reinterpret_cast<const __nv_bfloat162*>(&h[e]);
      const float2 hf = __bfloat1622float2(hb);
      l[e] = bf16pair(v[2 * e] - hf.x, v[2 * e + 1] - hf.y);
    }
  }
  *reinterpret_cast<uint4*>(img + off) = make_uint4(h[0], h[1], h[2], h[3]);
  if (split) *reinterpret_cast<uint4*>(img_lo + off) = make_uint4(l[0], l[1], l[2], l[3]);
}

// Rows [0, R) x k in [k0, k0 + 64) of an operand X(r, k) = X[(r0 + r) rs + k ks]
// (zero where r0 + r >= rlim or k >= kend) into the swizzled image, by the
// CTA's kGThreads threads. Every thread issues all of its loads before it
// converts and stores anything, so each waits one memory latency per
// K-block. With k contiguous (ks == 1) eight threads share a row, each
// converting one 16-byte unit, so a warp reads four rows' 256 contiguous
// bytes; otherwise consecutive threads take consecutive rows (a warp's loads
// span 32 rows) and the row's eight units are split among kGThreads / R
// threads.
constexpr int kGThreads = 256;
template <int R>
__device__ __forceinline__ void g_load(uint8_t* img, uint8_t* img_lo, const float* __restrict__ X,
                                       int64_t rs, int64_t ks, int r0, int rlim, int k0,
                                       int kend, bool split) {
  const int tid = threadIdx.x;
  if (ks == 1) {
    constexpr int RPP = kGThreads / 8;              // rows per pass
    constexpr int NP = (R + RPP - 1) / RPP;
    const int unit = tid & 7, rr = tid >> 3;
    float v[NP][8];
#pragma unroll
    for (int p = 0; p < NP; ++p) {
      const int r = rr + p * RPP, row = r0 + r;
      const float* src = X + (int64_t)row * rs;
#pragma unroll
      for (int e = 0; e < 8; ++e) {
        const int k = k0 + unit * 8 + e;
        v[p][e] = (r < R && row < rlim && k < kend) ? src[k] : 0.f;
      }
    }
#pragma unroll
    for (int p = 0; p < NP; ++p)
      if (rr + p * RPP < R) g_store8(img, img_lo, rr + p * RPP, unit, v[p], split);
  } else {
    constexpr int TPR = kGThreads / R;              // threads per row
    constexpr int UPT = 8 / TPR;                    // units per thread
    const int r = tid % R, ug = tid / R, row = r0 + r;
    float v[UPT][8];
#pragma unroll
    for (int u = 0; u < UPT; ++u)
#pragma unroll
      for (int e = 0; e < 8; ++e) {
        const int k = k0 + (ug * UPT + u) * 8 + e;
        v[u][e] = (row < rlim && k < kend) ? X[(int64_t)row * rs + (int64_t)k * ks] : 0.f;
      }
#pragma unroll
    for (int u = 0; u < UPT; ++u) g_store8(img, img_lo, r, ug * UPT + u, v[u], split);
  }
}

template <int TN>
__global__ void __launch_bounds__(kGThreads, 1)
gemm_tc_kernel(int M, int N, int Kd, const float* __restrict__ A, int64_t am, int64_t ak,
               const float* __restrict__ B, int64_t bk, int64_t bn, int round_a, int round_b,
               float* __restrict__ C, int64_t ldc, int mode, const float* __restrict__ bias,
               float* __restrict__ out2, int round_out, int kz, int* status) {
  constexpr uint32_t kAImg = 128 * 128, kBImg = TN * 128;
  constexpr uint32_t kStage = 2 * kAImg + 2 * kBImg;   // hi and lo images of both operands
  extern __shared__ uint8_t smem_raw[];
  uint8_t* base = reinterpret_cast<uint8_t*>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~static_cast<uintptr_t>(1023));
  uint64_t* bars = reinterpret_cast<uint64_t*>(base + 2 * kStage);   // [2] stage free, [1] done
  uint32_t* holder = reinterpret_cast<uint32_t*>(bars + 3);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  static_assert(TN % 64 == 0, "two column halves of whole 32-column loads");
  const int m0 = blockIdx.y * 128, n0 = blockIdx.x * TN;
  const int kbeg = blockIdx.z * kz;
  const int kend = min(Kd, kbeg + kz);
  const int nkb = kend > kbeg ? (kend - kbeg + kGTK - 1) / kGTK : 0;
  const bool split_a = !round_a, split_b = !round_b;
  if (tid == 0) {
    for (int b = 0; b < 3; ++b)
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(g_smem(&bars[b])), "r"(1)
                   : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     g_smem(holder)),
                 "r"(TN < 32 ? 32 : TN)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *holder;
  const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(TN >> 3) << 17) |
                         ((uint32_t)(128 >> 4) << 24);
  bool ok = true;
  for (int kb = 0; kb < nkb && ok; ++kb) {
    const int st = kb & 1;
    uint8_t* a_img = base + st * kStage;
    uint8_t* a_lo = a_img + kAImg;
    uint8_t* b_img = a_img + 2 * kAImg;
    uint8_t* b_lo = b_img + kBImg;
    // the MMAs that read this stage two blocks ago are done
    if (kb >= 2) ok = g_wait(g_smem(&bars[st]), ((kb - 2) >> 1) & 1, status);
    if (!ok) break;
    const int k0 = kbeg + kb * kGTK;
    g_load<128>(a_img, a_lo, A, am, ak, m0, M, k0, kend, split_a);
    g_load<TN>(b_img, b_lo, B, bn, bk, n0, N, k0, kend, split_b);
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    if (tid == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint64_t ad = g_desc(g_smem(a_img)), adl = g_desc(g_smem(a_lo));
      const uint64_t bd = g_desc(g_smem(b_img)), bdl = g_desc(g_smem(b_lo));
#pragma unroll
      for (int ks = 0; ks < 4; ++ks) {
        const uint32_t o = 2u * ks;
        g_mma(tmem, ad + o, bd + o, idesc, (kb | ks) != 0);
        if (split_b) g_mma(tmem, ad + o, bdl + o, idesc, 1u);
        if (split_a) g_mma(tmem, adl + o, bd + o, idesc, 1u);
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                       g_smem(&bars[st]))
                   : "memory");
    }
  }
  // all MMAs done
  if (tid == 0)
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                     g_smem(&bars[2]))
                 : "memory");
  const bool done = g_wait(g_smem(&bars[2]), 0, status);
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (done && ok) {
    // each warp's 32 accumulator rows go through a 32 x 33 scratch tile (in
    // the operand ring, idle now) so that the stores run along rows of C
    // warp w reads tensor-memory lanes 32 (w % 4) .. (its quadrant), columns
    // of half w / 4
    float* stage = reinterpret_cast<float*>(base) + warp * (32 * 33);
    float* Cz = C + (int64_t)blockIdx.z * M * ldc;
    const int quad = warp & 3, half = warp >> 2;
#pragma unroll 1
    for (int c0 = half * (TN / 2); c0 < (half + 1) * (TN / 2); c0 += 32) {
      uint32_t v[32];
      const uint32_t ta = tmem + ((uint32_t)(quad * 32) << 16) + (uint32_t)c0;
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
          "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
          "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];\n\t"
          "tcgen05.wait::ld.sync.aligned;"
          : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
            "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]),
            "=r"(v[13]), "=r"(v[14]), "=r"(v[15]), "=r"(v[16]), "=r"(v[17]), "=r"(v[18]),
            "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]), "=r"(v[24]),
            "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]),
            "=r"(v[31])
          : "r"(ta)
          : "memory");
#pragma unroll
      for (int e = 0; e < 32; ++e) stage[lane * 33 + e] = nkb > 0 ? __uint_as_float(v[e]) : 0.f;
      __syncwarp();
      const int n = n0 + c0 + lane;
#pragma unroll 4
      for (int r = 0; r < 32; ++r) {
        const int m = m0 + quad * 32 + r;
        if (m < M && n < N) {
          float x = stage[r * 33 + lane];
          if (mode >= 1) x += bias[n];
          Cz[(int64_t)m * ldc + n] = x;
          if (mode == 1) {
            const float gv = gelu(x);
            out2[(int64_t)m * ldc + n] = round_out ? round_bf16(gv) : gv;
          }
        }
      }
      __syncwarp();
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(TN < 32 ? 32 : TN)
                 : "memory");
  }
}

// C[m][n] = sum over the splits, in order, of the partial products.
__global__ void splitk_reduce_kernel(int64_t MN, int splits, const float* __restrict__ parts,
                                     float* __restrict__ C) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < MN;
       e += (int64_t)gridDim.x * blockDim.x) {
    float s = 0.f;
    for (int z = 0; z < splits; ++z) s += parts[z * MN + e];
    C[e] = s;
  }
}

// out[b] = sum_j H2[b][j] w3[j] + b3 (one warp per row, fixed lane order)
__global__ void output_kernel(int B, const float* __restrict__ H2, const float* __restrict__ w3,
                              const float* __restrict__ b3, float* __restrict__ out) {
  const int w = (int)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5);
  const int lane = threadIdx.x & 31;
  if (w >= B) return;
  float s = 0.f;
  for (int j = lane; j < kH; j += 32) s = fmaf(H2[(int64_t)w * kH + j], w3[j], s);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (lane == 0) out[w] = s + b3[0];
}

// Mean and standard deviation of l = log(max(fit, 1e-30)) over the batch
// (FP64, fixed order: thread-strided sums then a sequential sum of the 256
// partials).
// Mean and sd of the batch's log-fitness (FP64): 1024 threads, each
// thread's rows summed in order, then a fixed pairwise tree over the
// threads (the same order every run).
__device__ __forceinline__ double tree_sum_1024(double v, double* sh) {
  sh[threadIdx.x] = v;
  __syncthreads();
  for (int w = 512; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
    __syncthreads();
  }
  const double t = sh[0];
  __syncthreads();
  return t;
}

// l[b] = log(max(fit[b], 1e-30)) in FP64, over the whole GPU (FP64 is slow
// on one SM)
__global__ void log_fit_kernel(int B, const double* __restrict__ fit, double* __restrict__ l) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= B) return;
  const double f = fit[b];
  l[b] = log(f > 1e-30 ? f : 1e-30);
}

__global__ void __launch_bounds__(1024)
target_stats_kernel(int B, const double* __restrict__ l, double* __restrict__ stats) {
  __shared__ double sh[1024];
  double a = 0.0;
  for (int b = threadIdx.x; b < B; b += 1024) a += l[b];
  const double mu = tree_sum_1024(a, sh) / B;
  double q = 0.0;
  for (int b = threadIdx.x; b < B; b += 1024) {
    const double d = l[b] - mu;
    q += d * d;
  }
  const double t = tree_sum_1024(q, sh);
  if (threadIdx.x == 0) {
    const double sd = sqrt(t / B);
    stats[0] = mu;
    stats[1] = sd > 0.0 ? sd : 1.0;
  }
}

// d_out[b] = 2 (out[b] - t[b]) / B with the standardised target t; also the
// loss terms (out - t)^2 / B for reporting.
__global__ void dout_kernel(int B, const float* __restrict__ out, const double* __restrict__ l,
                            const double* __restrict__ stats, float* __restrict__ dout,
                            float* __restrict__ loss_terms) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= B) return;
  const float t = (float)((l[b] - stats[0]) / stats[1]);
  const float r = out[b] - t;
  dout[b] = 2.f * r / (float)B;
  loss_terms[b] = r * r / (float)B;
}

// dH2[b][j] = dout[b] w3[j], dZ2 = dH2 * g'(Z2) (in place into dZ)
__global__ void dz2_kernel(int B, const float* __restrict__ dout, const float* __restrict__ w3,
                           const float* __restrict__ Z2, float* __restrict__ dZ) {
  const int64_t n = (int64_t)B * kH;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int b = (int)(e / kH), j = (int)(e % kH);
    dZ[e] = dout[b] * w3[j] * gelu_grad(Z2[e]);
  }
}

// dZ[e] *= g'(Z[e])
__global__ void gelu_bwd_kernel(int64_t n, const float* __restrict__ Z, float* __restrict__ dZ) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n;
       e += (int64_t)gridDim.x * blockDim.x)
    dZ[e] *= gelu_grad(Z[e]);
}

// s[j] = sum_b X[b][j] y[b] (y = NULL: plain column sum). CTA = 32 columns x
// 32 row slices (1024 threads): thread (slice, column) adds its slice's rows
// in order, then the 32 slice sums of a column are added in slice order --
// a fixed order, so the result is the same run to run.
constexpr int kColSlices = 32;
__global__ void __launch_bounds__(1024)
colsum_kernel(int B, int N, const float* __restrict__ X, const float* __restrict__ y,
              float* __restrict__ s) {
  __shared__ float part[kColSlices][33];
  const int c = threadIdx.x & 31, sl = threadIdx.x >> 5;
  const int j = blockIdx.x * 32 + c;
  const int per = (B + kColSlices - 1) / kColSlices;
  const int b0 = sl * per, b1 = min(B, b0 + per);
  float acc = 0.f;
  if (j < N)
    for (int b = b0; b < b1; ++b) acc = fmaf(X[(int64_t)b * N + j], y ? y[b] : 1.f, acc);
  part[sl][c] = acc;
  __syncthreads();
  if (sl == 0 && j < N) {
    float t = 0.f;
    for (int k = 0; k < kColSlices; ++k) t += part[k][c];
    s[j] = t;
  }
}

__global__ void sum_kernel(int B, const float* __restrict__ v, float* __restrict__ s) {
  if (blockIdx.x != 0) return;
  __shared__ float part[256];
  float acc = 0.f;
  for (int b = threadIdx.x; b < B; b += 256) acc += v[b];
  part[threadIdx.x] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    float t = 0.f;
    for (int i = 0; i < 256; ++i) t += part[i];
    s[0] = t;
  }
}

__global__ void adam_kernel(int64_t n, float* __restrict__ w, const float* __restrict__ g,
                            float* __restrict__ m, float* __restrict__ v, float lr, float b1,
                            float b2, float eps, float c1, float c2) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n;
       e += (int64_t)gridDim.x * blockDim.x) {
    const float gi = g[e];
    const float mi = b1 * m[e] + (1.f - b1) * gi;
    const float vi = b2 * v[e] + (1.f - b2) * gi * gi;
    m[e] = mi;
    v[e] = vi;
    const float mh = mi / c1, vh = vi / c2;
    w[e] -= lr * mh / (sqrtf(vh) + eps);
  }
}

__global__ void init_params_kernel(uint64_t seed, int K, float* __restrict__ w) {
  const int64_t n1 = (int64_t)kH * K, n2 = (int64_t)kH * kH;
  const int64_t total = n1 + kH + n2 + kH + kH + 1;
  const float a1 = 1.f / sqrtf((float)K), a2 = 1.f / sqrtf((float)kH);
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    int layer;
    int64_t idx;
    float a;
    if (e < n1) {
      layer = 1, idx = e, a = a1;
    } else if (e < n1 + kH) {
      w[e] = 0.f;
      continue;
    } else if (e < n1 + kH + n2) {
      layer = 2, idx = e - n1 - kH, a = a2;
    } else if (e < n1 + kH + n2 + kH) {
      w[e] = 0.f;
      continue;
    } else if (e < n1 + kH + n2 + 2 * kH) {
      layer = 3, idx = e - n1 - 2 * kH - n2, a = a2;
    } else {
      w[e] = 0.f;
      continue;
    }
    const uint32_t r =
        philox4x32_10(seed, (uint32_t)layer, (uint32_t)idx, 0u, kTagSurrogate).x;
    // u in [-1, 1): (r >> 8) 2^-23 - 1, exact in FP32
    const float u = (float)(r >> 8) * (1.0f / 8388608.0f) - 1.0f;
    w[e] = u * a;
  }
}

// ---- screening: keep the n_keep smallest predictions of n ----
constexpr int kSortMax = 16384;

__global__ void __launch_bounds__(1024)
select_kernel(int n, int n_keep, const float* __restrict__ pred, int* __restrict__ keep_flag,
              const int* __restrict__ trusted, int* __restrict__ used_trust) {
  extern __shared__ uint64_t keys[];   // (order-preserving float bits << 32) | slot
  const int trust = *trusted;
  if (threadIdx.x == 0) *used_trust = trust;
  if (!trust) {   // the exact evaluator stands in: the unscreened generation's children
    for (int i = threadIdx.x; i < n; i += blockDim.x) keep_flag[i] = i < n_keep ? 1 : 0;
    return;
  }
  int npow = 1;
  while (npow < n) npow <<= 1;
  for (int i = threadIdx.x; i < npow; i += blockDim.x) {
    uint64_t k = ~0ull;
    if (i < n) {
      float p = pred[i];
      if (isnan(p)) p = __int_as_float(0x7f800000);   // NaN ranks last (+inf)
      uint32_t u = __float_as_uint(p);
      u = (u & 0x80000000u) ? ~u : (u | 0x80000000u);   // float order as unsigned
      k = ((uint64_t)u << 32) | (uint32_t)i;
    }
    keys[i] = k;
  }
  __syncthreads();
  for (int size = 2; size <= npow; size <<= 1) {
    for (int stride = size >> 1; stride > 0; stride >>= 1) {
      for (int i = threadIdx.x; i < npow; i += blockDim.x) {
        const int j = i ^ stride;
        if (j > i) {
          const bool up = (i & size) == 0;
          const uint64_t a = keys[i], b = keys[j];
          if ((a > b) == up) {
            keys[i] = b;
            keys[j] = a;
          }
        }
      }
      __syncthreads();
    }
  }
  for (int i = threadIdx.x; i < n; i += blockDim.x) keep_flag[i] = 0;
  __syncthreads();
  for (int i = threadIdx.x; i < n_keep; i += blockDim.x)
    keep_flag[(int)(keys[i] & 0xffffffffu)] = 1;
}

// pos[i] = number of kept children before child i (or -1 if child i is not
// kept): one CTA, an exclusive prefix sum of the flags in slot order.
__global__ void __launch_bounds__(1024)
assemble_kernel(int n, const int* __restrict__ keep_flag, int* __restrict__ pos) {
  __shared__ int warp_tot[32];
  __shared__ int carry;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (int base = 0; base < n; base += blockDim.x) {
    const int i = base + threadIdx.x;
    const int f = i < n ? keep_flag[i] : 0;
    int x = f;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    if (lane == 31) warp_tot[wid] = x;
    __syncthreads();
    if (wid == 0) {
      int t = warp_tot[lane];
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, t, o);
        if (lane >= o) t += y;
      }
      warp_tot[lane] = t;
    }
    __syncthreads();
    const int excl = carry + (wid ? warp_tot[wid - 1] : 0) + x - f;
    if (i < n) pos[i] = f ? excl : -1;
    __syncthreads();
    if (threadIdx.x == blockDim.x - 1) carry = excl + f;
    __syncthreads();
  }
}

__global__ void gather_kernel(int n, int E, int K, const int* __restrict__ pos,
                              const float* __restrict__ off, float* __restrict__ next) {
  // rows 0..E-1: elites; row E + pos[i] <- offspring slot E + i
  const int64_t total = (int64_t)(E + n) * K;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int s = (int)(e / K), k = (int)(e % K);
    if (s < E) {
      next[e] = off[e];
    } else {
      const int p = pos[s - E];
      if (p >= 0) next[(int64_t)(E + p) * K + k] = off[e];
    }
  }
}

// Pearson correlation of the kept children's predictions with their exact
// log-fitness (fit_kept[pos[i]] for kept child i), FP64 sums in a fixed
// order; trusted = r > 0.25.
__global__ void trust_kernel(int n, const float* __restrict__ pred, const int* __restrict__ flag,
                             const int* __restrict__ pos, const double* __restrict__ lfit_kept,
                             float* __restrict__ r_out, int* __restrict__ trusted) {
  __shared__ double sh[6][256];
  double a[6] = {0, 0, 0, 0, 0, 0};
  for (int i = threadIdx.x; i < n; i += 256) {
    if (!flag[i]) continue;
    const double x = pred[i];
    const double y = lfit_kept[pos[i]];
    a[0] += 1.0;
    a[1] += x;
    a[2] += y;
    a[3] += x * y;
    a[4] += x * x;
    a[5] += y * y;
  }
  for (int k = 0; k < 6; ++k) sh[k][threadIdx.x] = a[k];
  __syncthreads();
  if (threadIdx.x == 0) {
    double t[6] = {0, 0, 0, 0, 0, 0};
    for (int i = 0; i < 256; ++i)
      for (int k = 0; k < 6; ++k) t[k] += sh[k][i];
    const double c = t[0];
    double r = 0.0;
    if (c > 1.0) {
      const double cov = t[3] / c - (t[1] / c) * (t[2] / c);
      const double vx = t[4] / c - (t[1] / c) * (t[1] / c);
      const double vy = t[5] / c - (t[2] / c) * (t[2] / c);
      r = (vx > 0.0 && vy > 0.0) ? cov / sqrt(vx * vy) : 0.0;
    }
    *r_out = (float)r;
    *trusted = r > 0.25 ? 1 : 0;
  }
}

// Split-K factor of the weight-gradient GEMMs (reduction over the batch):
// about 64 rows per split, at most kMaxSplits.
int kGradSplits(int B) {
  int sp = (B + 63) / 64;
  return sp < 1 ? 1 : (sp > kMaxSplits ? kMaxSplits : sp);
}

int grid1d(int64_t n) {
  int64_t b = (n + 255) / 256;
  if (b < 1) b = 1;
  if (b > 8192) b = 8192;
  return (int)b;
}

constexpr int kGTN = 64;   // columns of C per CTA of the tensor-core GEMM

cudaError_t gemm(int M, int N, int Kd, const float* A, int64_t am, int64_t ak, const float* B,
                 int64_t bk, int64_t bn, int ra, int rb, float* C, int64_t ldc, int mode,
                 const float* bias, float* out2, int round_out, int* status, cudaStream_t st,
                 float* split_ws = nullptr, int splits = 1) {
  dim3 grid((N + kGTN - 1) / kGTN, (M + 127) / 128, splits);
  int kz = (Kd + splits - 1) / splits;
  kz = (kz + kGTK - 1) / kGTK * kGTK;
  const int smem = 2 * (2 * 128 * 128 + 2 * kGTN * 128) + 1024 + 64;
  cudaError_t e = cudaFuncSetAttribute(gemm_tc_kernel<kGTN>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  if (splits > 1) {
    // partial products into the workspace, then their sum in split order
    gemm_tc_kernel<kGTN><<<grid, kGThreads, smem, st>>>(M, N, Kd, A, am, ak, B, bk, bn, ra, rb,
                                                  split_ws, N, 0, nullptr, nullptr, 0, kz, status);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    splitk_reduce_kernel<<<grid1d((int64_t)M * N), 256, 0, st>>>((int64_t)M * N, splits,
                                                                  split_ws, C);
    return cudaGetLastError();
  }
  gemm_tc_kernel<kGTN><<<grid, kGThreads, smem, st>>>(M, N, Kd, A, am, ak, B, bk, bn, ra, rb, C, ldc,
                                                mode, bias, out2, round_out, kz, status);
  return cudaGetLastError();
}

}  // namespace

int64_t surrogate_param_count(int K) {
  return (int64_t)kH * K + kH + (int64_t)kH * kH + kH + kH + 1;
}

cudaError_t surrogate_init(const SurrogateDev& s, uint64_t seed, cudaStream_t st) {
  const int64_t n = surrogate_param_count(s.K);
  init_params_kernel<<<grid1d(n), 256, 0, st>>>(seed, s.K, s.w);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  e = cudaMemsetAsync(s.m, 0, n * sizeof(float), st);
  if (e == cudaSuccess) e = cudaMemsetAsync(s.v, 0, n * sizeof(float), st);
  return e;
}

// Forward pass of B rows X [B][K] (FP32 genes) into out [B]; keeps Z1, H1,
// Z2, H2 [B][256] in the workspace for a backward pass.
cudaError_t surrogate_forward(const SurrogateDev& s, const float* X, int B, float* out,
                              cudaStream_t st) {
  if (B > s.Bmax) return cudaErrorInvalidValue;
  const int K = s.K;
  const float* W1 = s.w;
  const float* b1 = W1 + (int64_t)kH * K;
  const float* W2 = b1 + kH;
  const float* b2 = W2 + (int64_t)kH * kH;
  const float* w3 = b2 + kH;
  const float* b3 = w3 + kH;
  // Z1 = bf(X) bf(W1)^T + b1, H1 = bf(g(Z1))
  cudaError_t e = gemm(B, kH, K, X, K, 1, W1, 1, K, 1, 1, s.Z1, kH, 1, b1, s.H1, 1, s.status, st);
  if (e != cudaSuccess) return e;
  // Z2 = H1 bf(W2)^T + b2, H2 = g(Z2)
  e = gemm(B, kH, kH, s.H1, kH, 1, W2, 1, kH, 1, 1, s.Z2, kH, 1, b2, s.H2, 0, s.status, st);
  if (e != cudaSuccess) return e;
  output_kernel<<<(int)(((int64_t)B * 32 + 255) / 256), 256, 0, st>>>(B, s.H2, w3, b3, out);
  return cudaGetLastError();
}

// Gradient of the mean squared error of log-fitness over B pairs into s.g
// (after a forward pass of the same X); loss into s.loss[0].
cudaError_t surrogate_backward(const SurrogateDev& s, const float* X, const double* fit, int B,
                               cudaStream_t st) {
  const int K = s.K;
  const float* W1 = s.w;
  const float* W2 = W1 + (int64_t)kH * K + kH;
  const float* w3 = W2 + (int64_t)kH * kH + kH;
  float* gW1 = s.g;
  float* gb1 = gW1 + (int64_t)kH * K;
  float* gW2 = gb1 + kH;
  float* gb2 = gW2 + (int64_t)kH * kH;
  float* gw3 = gb2 + kH;
  float* gb3 = gw3 + kH;
  log_fit_kernel<<<(B + 255) / 256, 256, 0, st>>>(B, fit, s.lfit);
  target_stats_kernel<<<1, 1024, 0, st>>>(B, s.lfit, s.tstat);
  dout_kernel<<<(B + 255) / 256, 256, 0, st>>>(B, s.out, s.lfit, s.tstat, s.dout, s.lterm);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  sum_kernel<<<1, 256, 0, st>>>(B, s.lterm, s.loss);
  // output layer
  colsum_kernel<<<kH / 32, 1024, 0, st>>>(B, kH, s.H2, s.dout, gw3);
  sum_kernel<<<1, 256, 0, st>>>(B, s.dout, gb3);
  // dZ2 = dout w3 g'(Z2)
  dz2_kernel<<<grid1d((int64_t)B * kH), 256, 0, st>>>(B, s.dout, w3, s.Z2, s.dZ2);
  // gW2 = dZ2^T H1, gb2 = colsum(dZ2)
  const int splits = kGradSplits(B);
  e = gemm(kH, kH, B, s.dZ2, 1, kH, s.H1, kH, 1, 0, 1, gW2, kH, 0, nullptr, nullptr, 0, s.status,
           st, s.split_ws, splits);
  if (e != cudaSuccess) return e;
  colsum_kernel<<<kH / 32, 1024, 0, st>>>(B, kH, s.dZ2, nullptr, gb2);
  // dZ1 = (dZ2 bf(W2)) g'(Z1)
  e = gemm(B, kH, kH, s.dZ2, kH, 1, W2, kH, 1, 0, 1, s.dZ1, kH, 0, nullptr, nullptr, 0, s.status,
           st);
  if (e != cudaSuccess) return e;
  gelu_bwd_kernel<<<grid1d((int64_t)B * kH), 256, 0, st>>>((int64_t)B * kH, s.Z1, s.dZ1);
  // gW1 = dZ1^T bf(X), gb1 = colsum(dZ1)
  e = gemm(kH, K, B, s.dZ1, 1, kH, X, K, 1, 0, 1, gW1, K, 0, nullptr, nullptr, 0, s.status, st,
           s.split_ws, splits);
  if (e != cudaSuccess) return e;
  colsum_kernel<<<kH / 32, 1024, 0, st>>>(B, kH, s.dZ1, nullptr, gb1);
  return cudaGetLastError();
}

cudaError_t surrogate_adam(SurrogateDev& s, cudaStream_t st) {
  s.step += 1;
  const float c1 = 1.f - powf(kAdamB1, (float)s.step);
  const float c2 = 1.f - powf(kAdamB2, (float)s.step);
  const int64_t n = surrogate_param_count(s.K);
  adam_kernel<<<grid1d(n), 256, 0, st>>>(n, s.w, s.g, s.m, s.v, kAdamLr, kAdamB1, kAdamB2,
                                         kAdamEps, c1, c2);
  return cudaGetLastError();
}

cudaError_t surrogate_trust_check(const SurrogateDev& s, int n, int n_kept, const float* pred,
                                  const int* flag, const int* pos, const double* fit_kept,
                                  float* r_out, int* trusted, cudaStream_t st) {
  if (n_kept > s.Bmax) return cudaErrorInvalidValue;
  // the kept children's log-fitness over the whole GPU first (FP64)
  log_fit_kernel<<<(n_kept + 255) / 256, 256, 0, st>>>(n_kept, fit_kept, s.lfit);
  trust_kernel<<<1, 256, 0, st>>>(n, pred, flag, pos, s.lfit, r_out, trusted);
  return cudaGetLastError();
}

cudaError_t surrogate_screen(int n, int n_keep, int E, int K, const float* pred, int* flag,
                             int* pos, const float* off, float* next, const int* trusted,
                             int* used_trust, cudaStream_t st) {
  if (n > kSortMax || n_keep > n) return cudaErrorInvalidValue;
  int npow = 1;
  while (npow < n) npow <<= 1;
  const size_t smem = (size_t)npow * sizeof(uint64_t);
  cudaError_t e = cudaFuncSetAttribute(select_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)(kSortMax * sizeof(uint64_t)));
  if (e != cudaSuccess) return e;
  select_kernel<<<1, 1024, smem, st>>>(n, n_keep, pred, flag, trusted, used_trust);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  assemble_kernel<<<1, 1024, 0, st>>>(n, flag, pos);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  gather_kernel<<<grid1d((int64_t)(E + n) * K), 256, 0, st>>>(n, E, K, pos, off, next);
  return cudaGetLastError();
}

}  // namespace game
