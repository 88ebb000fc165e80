// fitness_static.cu -- FP32 fitness evaluation that allocates no memory.
//
// Some callers cannot call cudaMalloc: plug-ins that live inside a host
// application which owns the whole device-memory budget and hands out only
// what it pre-allocated, runtimes that forbid allocation after start-up (an
// allocation can fail, and cudaMalloc / cudaFree may synchronise the device,
// which stalls every other stream of the process), and code that must not
// change the device's memory footprint while other work runs.
// game_eval_fitness_static serves them: the caller passes device pointers to
// its own inputs and output, the kernel reads the inputs in their natural
// layout (X row-major, pop [P][K]), and the one intermediate buffer -- the
// per-CTA FP64 partial sums of squared residuals -- is the file-scope array
// g_static_part below, of fixed size (4 MiB). Every GPU that loads the
// library holds that array until the process exits.
//
// Its first call on a device looks the array's device address up
// (cudaGetSymbolAddress, with that device current) and caches it; make that
// first call before any stream capture. The cached address belongs to the
// device's primary context: after cudaDeviceReset the module is loaded
// anew and the address may change, so no call may follow a reset of that
// device in the same process. All calls share the array: calls that
// overlap on the GPU (different streams, or different host threads on one
// device) race on it and must be serialised by the caller. Each call
// overwrites every entry it later reads, so nothing needs clearing between
// calls.
#include <stdio.h>

#include <mutex>

#include "basis.cuh"
#include "game_internal.cuh"

namespace game {

namespace {

constexpr int64_t kStaticPartDoubles = (int64_t)1 << 19;   // 4 MiB of FP64 partials
constexpr int kMaxDevices = 64;

static __device__ __align__(256) double g_static_part[kStaticPartDoubles];

constexpr int BP = 128;   // chromosomes per CTA
constexpr int BM = 128;   // patterns per tile
constexpr int KC = 16;    // contraction columns per chunk
constexpr int kThreads = 256;

// The CUDA-core FP32 contraction of fitness_fp32.cu, reading raw inputs:
// genes from pop [P][K] (guarded scalar loads instead of the transposed
// pack), features from X [M][N] (row clamped to M-1, masked later), targets
// from y [M] (guarded).
__global__ void __launch_bounds__(kThreads, 2)
fitness_static_kernel(int64_t M, int N, int d, int basis, int K, int Kc,
                      const float* __restrict__ X, const float* __restrict__ y,
                      const float* __restrict__ pop, int P, int Ppad, int ntiles,
                      double* __restrict__ part) {
  __shared__ __align__(16) float As[2][KC][BP];
  __shared__ __align__(16) float Bs[2][KC][BM];
  __shared__ double sse_s[BP];

  const int Kp = K - 1;
  const int tid = threadIdx.x;
  const int tx = tid & 15;
  const int ty = tid >> 4;
  const int cb = blockIdx.x * BP;
  const int nch = Kc / KC;
  const int la_row0 = tid >> 5, la_col = (tid & 31) * 4;
  const int gp = tid & (BM - 1);
  const int ghalf = tid >> 7;

  auto load_genes = [&](int k, float4& out) {
    float v[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int p = cb + la_col + j;
      v[j] = (p < P && k < Kp) ? pop[(int64_t)p * K + 1 + k] : 0.f;
    }
    out = make_float4(v[0], v[1], v[2], v[3]);
  };

  for (int i = tid; i < BP; i += kThreads) sse_s[i] = 0.0;

  for (int t = blockIdx.y; t < ntiles; t += gridDim.y) {
    int64_t m = (int64_t)t * BM + gp;
    if (m > M - 1) m = M - 1;
    const float* xs = X + m * N;

    float acc[8][8];
#pragma unroll
    for (int u = 0; u < 8; ++u)
#pragma unroll
      for (int v = 0; v < 8; ++v) acc[u][v] = 0.f;

    float4 ra[2];
    float rb[8];
#pragma unroll
    for (int h = 0; h < 2; ++h) load_genes(la_row0 + 8 * h, ra[h]);
    basis_run<8>(basis, d, Kp, xs, 1, ghalf * 8, rb);
    __syncthreads();
#pragma unroll
    for (int h = 0; h < 2; ++h)
      *reinterpret_cast<float4*>(&As[0][la_row0 + 8 * h][la_col]) = ra[h];
#pragma unroll
    for (int v = 0; v < 8; ++v) Bs[0][ghalf * 8 + v][gp] = rb[v];
    __syncthreads();

    for (int kc = 0; kc < nch; ++kc) {
      const int buf = kc & 1;
      const bool more = kc + 1 < nch;
      if (more) {
#pragma unroll
        for (int h = 0; h < 2; ++h) load_genes((kc + 1) * KC + la_row0 + 8 * h, ra[h]);
        basis_run<8>(basis, d, Kp, xs, 1, (kc + 1) * KC + ghalf * 8, rb);
      }
#pragma unroll
      for (int k = 0; k < KC; ++k) {
        const float4 a_lo = *reinterpret_cast<const float4*>(&As[buf][k][ty * 4]);
        const float4 a_hi = *reinterpret_cast<const float4*>(&As[buf][k][64 + ty * 4]);
        const float4 b_lo = *reinterpret_cast<const float4*>(&Bs[buf][k][tx * 4]);
        const float4 b_hi = *reinterpret_cast<const float4*>(&Bs[buf][k][64 + tx * 4]);
        const float a[8] = {a_lo.x, a_lo.y, a_lo.z, a_lo.w, a_hi.x, a_hi.y, a_hi.z, a_hi.w};
        const float b[8] = {b_lo.x, b_lo.y, b_lo.z, b_lo.w, b_hi.x, b_hi.y, b_hi.z, b_hi.w};
#pragma unroll
        for (int u = 0; u < 8; ++u)
#pragma unroll
          for (int v = 0; v < 8; ++v) acc[u][v] = fmaf(a[u], b[v], acc[u][v]);
      }
      if (more) {
#pragma unroll
        for (int h = 0; h < 2; ++h)
          *reinterpret_cast<float4*>(&As[buf ^ 1][la_row0 + 8 * h][la_col]) = ra[h];
#pragma unroll
        for (int v = 0; v < 8; ++v) Bs[buf ^ 1][ghalf * 8 + v][gp] = rb[v];
      }
      __syncthreads();
    }

    const int64_t mbase = (int64_t)t * BM;
    float yv[8];
    bool ok[8];
#pragma unroll
    for (int v = 0; v < 8; ++v) {
      const int64_t mm = mbase + (v < 4 ? tx * 4 + v : 60 + tx * 4 + v);
      ok[v] = mm < M;
      yv[v] = ok[v] ? y[mm] : 0.f;
    }
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int cl = u < 4 ? ty * 4 + u : 60 + ty * 4 + u;
      const int p = cb + cl;
      const float bias = p < P ? pop[(int64_t)p * K] : 0.f;
      float s = 0.f;
#pragma unroll
      for (int v = 0; v < 8; ++v) {
        const float r = (yv[v] - bias) - acc[u][v];
        s = ok[v] ? fmaf(r, r, s) : s;
      }
      s += __shfl_xor_sync(0xffffffffu, s, 1);
      s += __shfl_xor_sync(0xffffffffu, s, 2);
      s += __shfl_xor_sync(0xffffffffu, s, 4);
      s += __shfl_xor_sync(0xffffffffu, s, 8);
      if (tx == 0) sse_s[cl] += (double)s;
    }
  }
  __syncthreads();
  for (int i = tid; i < BP; i += kThreads)
    part[(int64_t)blockIdx.y * Ppad + cb + i] = sse_s[i];
}

std::mutex g_setup_mu;
double* g_part_ptr[kMaxDevices] = {};
int g_num_sms[kMaxDevices] = {};

thread_local char g_static_err[256];

}  // namespace

// Host side of game_eval_fitness_static (declared in include/game.h). Error
// text goes to *err (static thread-local storage, no allocation).
int eval_fitness_static(const float* X, const float* y, int64_t M, int32_t N, int32_t degree,
                        int32_t basis, const float* pop, int32_t P, double* fit_out,
                        void* cuda_stream, const char** err) {
  *err = g_static_err;
  g_static_err[0] = '\0';
  auto fail = [&](int code, const char* msg) {
    snprintf(g_static_err, sizeof(g_static_err), "%s", msg);
    return code;
  };
  if (!X || !y || !pop || !fit_out) return fail(GAME_EINVAL, "NULL argument");
  if (M < 1 || N < 1 || degree < 1) return fail(GAME_EINVAL, "M, N and degree must be >= 1");
  if (basis != GAME_BASIS_CHEB && basis != GAME_BASIS_TRIG)
    return fail(GAME_EINVAL, "unknown basis");
  const int B = basis == GAME_BASIS_TRIG ? 2 : 1;
  const int64_t K = (int64_t)B * N * degree + 1;
  if (K > kMaxK) return fail(GAME_EINVAL, "K = B*N*d + 1 exceeds 4097 genes");
  if (P < 1) return fail(GAME_EINVAL, "P must be >= 1");
  const int64_t Ppad = ((int64_t)P + BP - 1) / BP * BP;
  if (Ppad > kStaticPartDoubles)
    return fail(GAME_EINVAL,
                "P exceeds the static scratch: at most 524288 chromosomes (4 MiB of partials)");
  if (M > ((int64_t)1 << 40)) return fail(GAME_EINVAL, "M too large");
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return fail(GAME_ECUDA, cudaGetErrorString(e));
  if (dev < 0 || dev >= kMaxDevices) return fail(GAME_EINVAL, "device ordinal beyond 63");
  // every array must be device memory of the current device (managed memory
  // is reachable from any device): a pointer into another GPU would make the
  // kernel read or write that GPU's memory
  const void* ptrs[4] = {X, y, pop, fit_out};
  const char* names[4] = {"X", "y", "pop", "fit_out"};
  for (int i = 0; i < 4; ++i) {
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, ptrs[i]) != cudaSuccess ||
        (at.type != cudaMemoryTypeDevice && at.type != cudaMemoryTypeManaged)) {
      cudaGetLastError();
      return fail(GAME_EINVAL, "X, y, pop and fit_out must be device pointers");
    }
    if (at.type == cudaMemoryTypeDevice && at.device != dev) {
      snprintf(g_static_err, sizeof(g_static_err),
               "%s is memory of device %d, not of the current device %d", names[i], at.device,
               dev);
      return GAME_EINVAL;
    }
  }
  double* part = nullptr;
  int sms = 0;
  {
    std::lock_guard<std::mutex> lk(g_setup_mu);
    if (!g_part_ptr[dev]) {
      void* p = nullptr;
      e = cudaGetSymbolAddress(&p, g_static_part);
      if (e != cudaSuccess) return fail(GAME_ECUDA, cudaGetErrorString(e));
      e = cudaDeviceGetAttribute(&g_num_sms[dev], cudaDevAttrMultiProcessorCount, dev);
      if (e != cudaSuccess) return fail(GAME_ECUDA, cudaGetErrorString(e));
      g_part_ptr[dev] = static_cast<double*>(p);
    }
    part = g_part_ptr[dev];
    sms = g_num_sms[dev];
  }
  const int Kc = (int)((K - 1 + KC - 1) / KC * KC);
  const int grid_x = (int)(Ppad / BP);
  const int64_t ntiles64 = (M + BM - 1) / BM;
  if (ntiles64 > INT32_MAX) return fail(GAME_EINVAL, "M too large");
  const int ntiles = (int)ntiles64;
  int64_t rows = (2 * (int64_t)sms + grid_x - 1) / grid_x;
  if (rows < 1) rows = 1;
  if (rows > ntiles) rows = ntiles;
  if (rows > kStaticPartDoubles / Ppad) rows = kStaticPartDoubles / Ppad;
  if (rows > 65535) rows = 65535;
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  dim3 grid(grid_x, (unsigned)rows);
  fitness_static_kernel<<<grid, kThreads, 0, st>>>(M, N, degree, basis, (int)K, Kc, X, y, pop,
                                                   P, (int)Ppad, ntiles, part);
  e = cudaGetLastError();
  if (e != cudaSuccess) return fail(GAME_ECUDA, cudaGetErrorString(e));
  e = launch_reduce(part, (int)rows, P, (int)Ppad, M, GAME_ERR_MSE, fit_out, st);
  if (e != cudaSuccess) return fail(GAME_ECUDA, cudaGetErrorString(e));
  return GAME_OK;
}

}  // namespace game

extern "C" int game_eval_fitness_static(const float* X, const float* y, int64_t M, int32_t N,
                                        int32_t degree, int32_t basis, const float* pop,
                                        int32_t P, double* fit_out, void* cuda_stream) {
  const char* err = nullptr;
  const int rc = game::eval_fitness_static(X, y, M, N, degree, basis, pop, P, fit_out,
                                           cuda_stream, &err);
  game::record_error(rc == GAME_OK ? "" : err);
  return rc;
}
