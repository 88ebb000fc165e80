"""The host planners that size every fitness launch keep the invariants the
kernels rely on, over a sweep of shapes (no GPU: the planners are host code
of libgame.so, called from a small host program built against the library's
internal header).

Tensor-core plan: shared memory within the 227 KB opt-in limit; a tile width
that divides the 768-pattern padding (192 for BF16 only); the K-block count
of the form's column width; an expansion ring of KB to 2 KB slots; features
read from L2 only for the BF16 Chebyshev runs of 8 degrees at 128 or 256
patterns; a power-of-two TMEM allocation of at most 512 columns that holds
two accumulators; a grid of at most one CTA per SM and per pattern tile; one
partial row per CTA and column half (per 2-CTA cluster and column half for
the paired-SM plans of the BF16 form, whose chromosome tiles come in pairs);
refusal monotone in the contraction length and independent of P. CUDA-core plan: a contraction padded to whole
chunks, at least one and at most ceil(M / 128) pattern blocks."""
import os
import shutil
import subprocess

import pytest

from paper_1211_5481_gb300 import build as gbuild

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1211_5481_gb300", "csrc")

HARNESS = r"""
#include <cstdio>
#include "game_internal.cuh"
using namespace game;
static int bad = 0;
#define CHECK(c, ...) do { if (!(c)) { ++bad; if (bad < 20) { printf("violation: %s ", #c); \
  printf(__VA_ARGS__); printf("\n"); } } } while (0)
static Shape shape(long long M, int N, int d, int basis) {
  Shape s{}; s.M = M; s.Mpad = (M + 767) / 768 * 768; s.N = N; s.d = d; s.basis = basis;
  s.B = basis ? 2 : 1; s.K = s.B * N * d + 1; s.Kp = s.K - 1; return s;
}
int main() {
  const int sms = 152;
  const int Ns[] = {1, 2, 3, 5, 8, 16, 32, 48, 64, 128, 256};
  const long long Ms[] = {1, 777, 1000000};
  const int Ps[] = {1, 64, 129, 1024, 16384};
  long long plans = 0;
  // 1024: the slack kept before any probe; 0: a probe found the dynamic
  // shared memory already 1024-aligned (then the targets can be staged too)
  for (int pad : {1024, 0}) {
  set_smem_base_pad(pad);
  for (int form = 0; form < 3; ++form)
    for (int basis = 0; basis < 2; ++basis)
      for (int N : Ns)
        for (long long M : Ms) {
          bool refused = false;
          for (int d = 1; ; d += d < 64 ? 1 : d / 16) {
            Shape s = shape(M, N, d, basis);
            if (s.K > 4097) break;
            bool ok0 = false;
            for (int pi = 0; pi < 5; ++pi) {
              const int P = Ps[pi];
              TcPlan pl = plan_tc(s, P, sms, form);
              ++plans;
              if (pi == 0) ok0 = pl.ok;
              CHECK(pl.ok == ok0, "form %d N %d d %d: refusal depends on P", form, N, d);
              if (!pl.ok) continue;
              CHECK(pl.pair == 0 || pl.pair == 1, "pair");
              CHECK(!pl.pair || (form == kFormBF16 && P > 128), "pair plan for form %d P %d", form, P);
              if (pl.pair) CHECK(pl.C == 2 * ((P + 255) / 256), "pair C");
              else CHECK(pl.C == (P + 127) / 128, "C");
              CHECK(!refused, "form %d basis %d N %d d %d: accepted after a shorter K' was refused",
                    form, basis, N, d);
              CHECK(pl.smem_bytes <= 232448 && pl.smem_bytes >= 120 * 1024, "smem %d", pl.smem_bytes);
              CHECK(pl.BN == 256 || pl.BN == 192 || pl.BN == 128 || pl.BN == 64 || pl.BN == 32,
                    "BN %d", pl.BN);
              CHECK(!pl.pair || pl.BN == 256, "pair tile %d", pl.BN);
              CHECK(768 % pl.BN == 0, "BN %d", pl.BN);
              CHECK(pl.BN != 192 || form == kFormBF16, "192 for form %d", form);
              CHECK(pl.KB == (s.Kp + form_cols(form) - 1) / form_cols(form), "KB %d", pl.KB);
              CHECK(pl.NS >= pl.KB && pl.NS <= 2 * pl.KB, "NS %d KB %d", pl.NS, pl.KB);
              CHECK(pl.xstage == 0 || pl.xstage == 1, "xstage");
              CHECK(pl.ystage == 0 || (pl.ystage == 1 && pl.xstage == 0 && !pl.pair), "ystage");
              CHECK(pl.pair || pl.slack == pad, "slack %d pad %d", pl.slack, pad);
              CHECK(pl.xstage == 1 || (form == kFormBF16 && basis == 0 && d % 8 == 0 &&
                                       pl.BN % 128 == 0), "unstaged features, form %d d %d BN %d",
                    form, d, pl.BN);
              CHECK(pl.stages <= 4 && pl.stages >= (form == kFormBF16x3 ? 2 : 3), "stages %d",
                    pl.stages);
              const int c = pl.tmem_cols;
              CHECK(c >= 32 && c <= 512 && (c & (c - 1)) == 0 && c >= 2 * pl.BN, "tmem %d", c);
              const long long ntiles = (M + pl.BN - 1) / pl.BN;
              if (pl.pair) {
                // 2-CTA clusters, each at least one tile; one partial row per
                // (cluster, column half)
                CHECK(pl.grid >= 2 && pl.grid % 2 == 0 && pl.grid <= sms && pl.grid / 2 <= ntiles,
                      "pair grid %d", pl.grid);
                CHECK(pl.rows == pl.grid, "pair rows");
                CHECK(pl.tmem_cols == 512, "pair tmem");
              } else {
                CHECK(pl.grid >= 1 && pl.grid <= sms && pl.grid <= ntiles, "grid %d", pl.grid);
                CHECK(pl.rows == 2 * pl.grid, "rows");
              }
              CHECK((long long)ntiles * pl.BN <= s.Mpad, "padding");
            }
            if (!ok0) refused = true;
            Fp32Plan fp = plan_fp32(s, 1000, sms);
            CHECK(fp.Kc % 16 == 0 && fp.Kc >= s.Kp && fp.Kc < s.Kp + 16, "Kc %d", fp.Kc);
            CHECK(fp.grid_x == (1000 + 127) / 128, "grid_x");
            CHECK(fp.grid_y >= 1 && fp.grid_y <= (M + 127) / 128, "grid_y %d", fp.grid_y);
          }
        }
  }
  // the large classification shape stages its targets once the base is aligned
  set_smem_base_pad(0);
  TcPlan big = plan_tc(shape(1000000, 32, 8, 0), 1024, sms, kFormBF16);
  CHECK(big.ok && big.BN == 256 && big.xstage == 0 && big.ystage == 1 && big.NS == 5 &&
        big.stages == 4, "classification plan BN %d ystage %d NS %d stages %d", big.BN,
        big.ystage, big.NS, big.stages);
  set_smem_base_pad(1024);
  big = plan_tc(shape(1000000, 32, 8, 0), 1024, sms, kFormBF16);
  CHECK(big.ok && big.BN == 256 && big.ystage == 0 && big.NS == 5 && big.stages == 4,
        "classification plan without alignment BN %d ystage %d", big.BN, big.ystage);
  printf("plans %lld violations %d\n", plans, bad);
  return bad != 0;
}
"""


@pytest.mark.skipif(shutil.which("nvcc") is None, reason="needs nvcc to build the host program")
def test_planners_keep_kernel_invariants(tmp_path):
    lib = gbuild.build()
    src = tmp_path / "plan.cu"
    src.write_text(HARNESS)
    exe = tmp_path / "plan"
    libdir = os.path.dirname(lib)
    subprocess.run(["nvcc", "-std=c++17", "-I", CSRC, str(src), "-o", str(exe), "-L", libdir,
                    "-lgame", "-Xlinker", "-rpath=" + libdir], check=True)
    res = subprocess.run([str(exe)], capture_output=True, text=True, timeout=300)
    assert res.returncode == 0, res.stdout
    assert "violations 0" in res.stdout
