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
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

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

namespace game {

// ---- chunk descriptors for the tensor-core operand generator ----
// A chunk is 8 consecutive contraction columns [8*cid, 8*cid + 8). Its
// descriptor records where the chunk starts in the feature / group / degree
// sequence, so the generator needs no division in its inner loop:
//   bits  0-15  feature i of the first column
//   bits 16-20  degree j of the first column (1..d)
//   bit  21     group b of the first column (trigonometric: 0 cos, 1 sin)
//   bit  22     all 8 columns lie in one (feature, group) run of degrees
//   bits 24-27  number of columns below Kp (8 except in the last chunk)
//   bit  31     no column below Kp (all-zero chunk)
constexpr uint32_t kChunkZero = 1u << 31;
constexpr uint32_t kChunkRun = 1u << 22;

__host__ __device__ inline uint32_t chunk_desc(int cid, int basis, int d, int Kp) {
  const int c0 = 8 * cid;
  if (c0 >= Kp) return kChunkZero;
  const int W = (basis == GAME_BASIS_TRIG ? 2 : 1) * d;
  const int i = c0 / W, off = c0 % W;
  const int b = off / d, j = off % d + 1;
  const int nvalid = (Kp - c0) < 8 ? (Kp - c0) : 8;
  uint32_t desc = (uint32_t)i | ((uint32_t)j << 16) | ((uint32_t)b << 21) |
                  ((uint32_t)nvalid << 24);
  if (j + 7 <= d) desc |= kChunkRun;
  return desc;
}

// Chebyshev chunk crossing feature runs, degree d >= 4 (so the chunk's 8
// columns touch at most three features), for two patterns at once (va for
// xrow0; vb for xrow1 when hasB): the same values, bit for bit, as gen_chunk,
// with the three features' x loaded up front and both recurrences
// interleaved. Columns from nvalid on are zero.
__device__ __forceinline__ void cheb_cross2(uint32_t desc, int d, int N, const float* xrow0,
                                            const float* xrow1, int xstride, bool hasB,
                                            float (&va)[8], float (&vb)[8]) {
  const int i = (int)(desc & 0xFFFFu);
  const int j0 = (int)((desc >> 16) & 31u);
  const int nvalid = (int)((desc >> 24) & 15u);
  const int i1 = i + 1 < N ? i + 1 : N - 1, i2 = i + 2 < N ? i + 2 : N - 1;
  const float xa0 = xrow0[i * xstride], xa1 = xrow0[i1 * xstride], xa2 = xrow0[i2 * xstride];
  const float xb0 = hasB ? xrow1[i * xstride] : 0.f;
  const float xb1 = hasB ? xrow1[i1 * xstride] : 0.f;
  const float xb2 = hasB ? xrow1[i2 * xstride] : 0.f;
  float a2 = xa0 + xa0, ta = xa0, tam = 1.f;
  float b2 = xb0 + xb0, tb = xb0, tbm = 1.f;
  for (int st = 1; st < j0; ++st) {
    const float na = fmaf(a2, ta, -tam), nb = fmaf(b2, tb, -tbm);
    tam = ta;
    ta = na;
    tbm = tb;
    tb = nb;
  }
  int j = j0;
  bool second = false;   // the next restart takes the third feature
#pragma unroll
  for (int e = 0; e < 8; ++e) {
    va[e] = ta;
    vb[e] = tb;
    if (j == d) {
      j = 1;
      const float xa = second ? xa2 : xa1, xb = second ? xb2 : xb1;
      second = true;
      a2 = xa + xa;
      ta = xa;
      tam = 1.f;
      b2 = xb + xb;
      tb = xb;
      tbm = 1.f;
    } else {
      ++j;
      const float na = fmaf(a2, ta, -tam), nb = fmaf(b2, tb, -tbm);
      tam = ta;
      ta = na;
      tbm = tb;
      tb = nb;
    }
  }
  if (nvalid < 8) {
#pragma unroll
    for (int e = 0; e < 8; ++e)
      if (e >= nvalid) {
        va[e] = 0.f;
        vb[e] = 0.f;
      }
  }
}

// One-pattern form of cheb_cross2 (same values as gen_chunk).
__device__ __forceinline__ void cheb_cross1(uint32_t desc, int d, int N, const float* xrow,
                                            int xstride, float (&v)[8]) {
  const int i = (int)(desc & 0xFFFFu);
  const int j0 = (int)((desc >> 16) & 31u);
  const int nvalid = (int)((desc >> 24) & 15u);
  const int i1 = i + 1 < N ? i + 1 : N - 1, i2 = i + 2 < N ? i + 2 : N - 1;
  const float x0 = xrow[i * xstride], x1 = xrow[i1 * xstride], x2 = xrow[i2 * xstride];
  float a2 = x0 + x0, t = x0, tm = 1.f;
  for (int st = 1; st < j0; ++st) {
    const float n = fmaf(a2, t, -tm);
    tm = t;
    t = n;
  }
  int j = j0;
  bool second = false;
#pragma unroll
  for (int e = 0; e < 8; ++e) {
    v[e] = t;
    if (j == d) {
      j = 1;
      const float x = second ? x2 : x1;
      second = true;
      a2 = x + x;
      t = x;
      tm = 1.f;
    } else {
      ++j;
      const float n = fmaf(a2, t, -tm);
      tm = t;
      t = n;
    }
  }
  if (nvalid < 8) {
#pragma unroll
    for (int e = 0; e < 8; ++e)
      if (e >= nvalid) v[e] = 0.f;
  }
}

// ---- whole-feature groups (the batched generator) ----
// With W = B d columns per feature, a group is the shortest run of whole
// features that fills whole 8-column chunks: F = 8 / gcd(W, 8) features, G =
// F W columns, G / 8 chunks, and group g starts at column g G. With the basis
// and the degree known at compile time, a group's values are straight-line
// code: one FMA per value after each feature's start (T_1 = x, or one
// sincosf), the F features' recurrences independent of one another, no
// branch and no restart. The values are those of gen_chunk bit for bit (the
// same operations from the same start values).
constexpr int const_gcd(int a, int b) { return b == 0 ? a : const_gcd(b, a % b); }

template <int BASIS, int D>
struct FeatureGroup {
  static constexpr int W = (BASIS == GAME_BASIS_TRIG ? 2 : 1) * D;
  static constexpr int F = 8 / const_gcd(W, 8);
  static constexpr int G = F * W;
  static constexpr int CH = G / 8;
  // groups generated together before their chunks are stored (several
  // groups at once, for more independent recurrences, measured slower)
  static constexpr int U = 1;
};

// The values of NF consecutive whole features x[0..NF) (NF a multiple of the
// group's F), rounded to BF16 and packed in column pairs: pk[k] holds columns
// 2k and 2k + 1, the lower column in the low half. Features f >= nf (past the
// problem's last feature) give zeros. The NF recurrences are independent, so
// the compiler can interleave them.
template <int BASIS, int D, int NF>
__device__ __forceinline__ void features_bf16(const float (&x)[NF], int nf,
                                              uint32_t (&pk)[NF * (BASIS == GAME_BASIS_TRIG ? 2 : 1) * D / 2]) {
  constexpr int W = (BASIS == GAME_BASIS_TRIG ? 2 : 1) * D;
  float lo = 0.f;   // the pending even column
#pragma unroll
  for (int f = 0; f < NF; ++f) {
    const bool on = f < nf;
    float fm, fv, c2;
    float s1 = 0.f;
    if (BASIS == GAME_BASIS_CHEB) {
      c2 = x[f] + x[f];
      fm = 1.f;
      fv = x[f];
    } else {
      float c1;
      sincosf(x[f], &s1, &c1);
      c2 = c1 + c1;
      fm = 1.f;   // cos(0 x)
      fv = c1;    // cos(1 x)
    }
#pragma unroll
    for (int e = 0; e < W; ++e) {
      if (e > 0) {
        if (BASIS == GAME_BASIS_TRIG && e == D) {
          fm = 0.f;   // sin(0 x)
          fv = s1;    // sin(1 x)
        } else {
          const float fn = fmaf(c2, fv, -fm);
          fm = fv;
          fv = fn;
        }
      }
      const int c = f * W + e;
      const float val = on ? fv : 0.f;
      if (c & 1) {
        const __nv_bfloat162 b2 = __floats2bfloat162_rn(lo, val);
        pk[c >> 1] = *reinterpret_cast<const uint32_t*>(&b2);
      } else {
        lo = val;
      }
    }
  }
}

// The 8 expansion values of one chunk for one pattern whose features are
// x_i = xrow[i * xstride] (shared or global memory).
__device__ __forceinline__ void gen_chunk(uint32_t desc, int basis, int d, int N,
                                          const float* xrow, int xstride, float (&v)[8]) {
  if (desc & kChunkZero) {
#pragma unroll
    for (int e = 0; e < 8; ++e) v[e] = 0.f;
    return;
  }
  int i = (int)(desc & 0xFFFFu);
  int j = (int)((desc >> 16) & 31u);
  int b = (int)((desc >> 21) & 1u);
  const int nvalid = (int)((desc >> 24) & 15u);
  float x = xrow[i * xstride];
  if (basis == GAME_BASIS_CHEB) {
    float x2 = x + x, tm1 = 1.f, t = x;
    for (int s = 1; s < j; ++s) {
      const float tn = fmaf(x2, t, -tm1);
      tm1 = t;
      t = tn;
    }
    if (desc & kChunkRun) {
      v[0] = t;
#pragma unroll
      for (int e = 1; e < 8; ++e) {
        const float tn = fmaf(x2, t, -tm1);
        tm1 = t;
        t = tn;
        v[e] = t;
      }
    } else {
#pragma unroll
      for (int e = 0; e < 8; ++e) {
        v[e] = t;
        if (j == d) {
          ++i;
          j = 1;
          x = (i < N) ? xrow[i * xstride] : 0.f;
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
  } else {
    float s1, c1;
    sincosf(x, &s1, &c1);
    float c2x = c1 + c1;
    float fm = b ? 0.f : 1.f;
    float f = b ? s1 : c1;
    for (int s = 1; s < j; ++s) {
      const float fn = fmaf(c2x, f, -fm);
      fm = f;
      f = fn;
    }
#pragma unroll
    for (int e = 0; e < 8; ++e) {
      v[e] = f;
      if (j == d) {
        j = 1;
        if (b == 0) {
          b = 1;
          fm = 0.f;
          f = s1;
        } else {
          ++i;
          b = 0;
          x = (i < N) ? xrow[i * xstride] : 0.f;
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
  if (nvalid < 8) {
#pragma unroll
    for (int e = 0; e < 8; ++e)
      if (e >= nvalid) v[e] = 0.f;
  }
}

}  // namespace game
