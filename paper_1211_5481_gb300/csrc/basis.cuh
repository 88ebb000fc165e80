// basis.cuh -- in-register polynomial expansion of one pattern's features.
//
// Contraction column c (0-based) carries gene c+1. With Bd = B*d columns per
// feature, column c belongs to feature i = c / Bd, group b = (c % Bd) / d and
// degree j = c % d + 1, and holds phi_{b,j}(x_i) (paper Section 3, Eq. 1 and
// Eq. 6):
//   Chebyshev:      T_j(x) by T_{j+1} = 2x T_j - T_{j-1}, T_0 = 1, T_1 = x;
//   trigonometric:  cos(jx) (b = 0) and sin(jx) (b = 1), from one sincosf(x)
//                   and the recurrences f_{j+1} = 2 cos(x) f_j - f_{j-1}.
// basis_run<NV> produces NV consecutive columns for one pattern, stepping the
// recurrence from column to column, so a run inside one feature costs one FMA
// per value. Columns >= Kp are zero (padding of the contraction length).
#pragma once
#include <cuda_runtime.h>

#include "../../include/game.h"

namespace game {

template <int NV>
__device__ __forceinline__ void basis_run_cheb(int d, int Kp, const float* xs, int xstride,
                                               int c0, float (&out)[NV]) {
  int i = c0 / d;
  int j = c0 - i * d + 1;
  float x = (c0 < Kp) ? xs[i * xstride] : 0.f;
  float x2 = x + x;
  float tm1 = 1.f, t = x;
  for (int s = 1; s < j; ++s) {
    const float tn = fmaf(x2, t, -tm1);
    tm1 = t;
    t = tn;
  }
#pragma unroll
  for (int v = 0; v < NV; ++v) {
    const int col = c0 + v;
    out[v] = (col < Kp) ? t : 0.f;
    if (j == d) {
      ++i;
      j = 1;
      x = (col + 1 < Kp) ? xs[i * xstride] : 0.f;
      x2 = x + x;
      tm1 = 1.f;
      t = x;
    } else {
      ++j;
      const float tn = fmaf(x2, t, -tm1);
      tm1 = t;
      t = tn;
    }
  }
}

template <int NV>
__device__ __forceinline__ void basis_run_trig(int d, int Kp, const float* xs, int xstride,
                                               int c0, float (&out)[NV]) {
  const int Bd = 2 * d;
  int i = c0 / Bd;
  const int rem = c0 - i * Bd;
  int b = rem >= d ? 1 : 0;
  int j = rem - b * d + 1;
  float x = (c0 < Kp) ? xs[i * xstride] : 0.f;
  float s1, c1;
  sincosf(x, &s1, &c1);
  float c2x = c1 + c1;
  float fm = b ? 0.f : 1.f;   // f_{j-1}: cos(0) = 1, sin(0) = 0
  float f = b ? s1 : c1;      // f_j
  for (int s = 1; s < j; ++s) {
    const float fn = fmaf(c2x, f, -fm);
    fm = f;
    f = fn;
  }
#pragma unroll
  for (int v = 0; v < NV; ++v) {
    const int col = c0 + v;
    out[v] = (col < Kp) ? f : 0.f;
    if (j == d) {
      j = 1;
      if (b == 0) {
        b = 1;
        fm = 0.f;
        f = s1;
      } else {
        ++i;
        b = 0;
        x = (col + 1 < Kp) ? xs[i * xstride] : 0.f;
        sincosf(x, &s1, &c1);
        c2x = c1 + c1;
        fm = 1.f;
        f = c1;
      }
    } else {
      ++j;
      const float fn = fmaf(c2x, f, -fm);
      fm = f;
      f = fn;
    }
  }
}

template <int NV>
__device__ __forceinline__ void basis_run(int basis, int d, int Kp, const float* xs,
                                          int xstride, int c0, float (&out)[NV]) {
  if (basis == GAME_BASIS_CHEB)
    basis_run_cheb<NV>(d, Kp, xs, xstride, c0, out);
  else
    basis_run_trig<NV>(d, Kp, xs, xstride, c0, out);
}

}  // namespace game
