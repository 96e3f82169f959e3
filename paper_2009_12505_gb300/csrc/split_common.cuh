// Device helpers shared by the split-precision kernels: digit slicing,
// integer recombination and fixed-point accumulation, double-float (f32
// pair) arithmetic.
#pragma once

#include <cuda_bf16.h>

#include "umma.cuh"

namespace split {

constexpr int TM = 128, TK = 32, NT = 64, NSTAGE = 2;
constexpr int KT_CHUNK = 20;  // K tiles per job: exact group sums need K <= 640

__host__ __device__ __forceinline__ int tile_off(int r, int c) {
  return ((r >> 3) * 4 + (c >> 3)) * 64 + (r & 7) * 8 + (c & 7);
}

// Row exponent e (|x| < 2^(e-1)) from the largest magnitude's bit pattern.
__device__ __forceinline__ int row_exponent(long long mbits) {
  if (mbits == 0) return -1000;
  const int ef = (int)(mbits >> 52);
  return (ef == 0 ? -1022 : ef - 1023) + 2;
}

// k balanced base-128 digits of x 2^(-e): x = 2^e sum_s d_s 2^(-7 s).
template <int KS>
__device__ __forceinline__ void to_digits(double x, int e, int (&d)[KS]) {
  long long X = (e > -1000) ? __double2ll_rn(ldexp(x, 7 * KS - e)) : 0ll;
#pragma unroll
  for (int s = KS - 1; s > 0; --s) {
    const int dd = (int)(((X + 64) & 127) - 64);
    d[s] = dd;
    X = (X - dd) >> 7;
  }
  d[0] = (int)X;
}

// k balanced base-128 digits of an integer X with |X| <= 2^(7 KS - 1):
// X = sum_s d_s 2^(7 (KS - 1 - s)), |d_s| <= 64.
template <int KS>
__device__ __forceinline__ void to_digits_i64(long long X, int (&d)[KS]) {
#pragma unroll
  for (int s = KS - 1; s > 0; --s) {
    const int dd = (int)(((X + 64) & 127) - 64);
    d[s] = dd;
    X = (X - dd) >> 7;
  }
  d[0] = (int)X;
}

// Add W * 2^e to a fixed-point Sigma element (hi: 2^-32 units, lo: 2^-64
// units) with integer arithmetic; |W 2^e| < 2^31, else nothing is added and
// HFX_DEV_ERR_BOUNDS is recorded in *err.
__device__ __forceinline__ void fx_add_scaled(unsigned long long *hi_lo, long long W, int e,
                                              unsigned *err) {
  if (W == 0) return;
  const unsigned long long mag = W < 0 ? 0ull - (unsigned long long)W : (unsigned long long)W;
  if (64 - __clzll((long long)mag) + e > 31) {  // |W| 2^e >= 2^31 possible
    atomicOr(err, 8u);
    return;
  }
  const int t = e + 64;  // W * 2^t in units of 2^-64
  __int128 V;
  if (t >= 0) {
    V = (__int128)W << t;
  } else if (t > -64) {
    V = (__int128)(W >> (-t));
  } else {
    V = W < 0 ? -1 : 0;
  }
  const long long hi = (long long)(V >> 32);
  const long long lo = (long long)(V & (__int128)0xFFFFFFFFll);
  if (hi) atomicAdd(hi_lo, (unsigned long long)hi);
  if (lo) atomicAdd(hi_lo + 1, (unsigned long long)lo);
}

// Index of the neighbour entry of [base, base + n) whose column range holds col.
__device__ __forceinline__ int entry_of(const NbrEntry *nbr, int64_t base, int n, int col) {
  int lo = 0, hi = n - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (nbr[base + mid].aopre <= col) lo = mid; else hi = mid - 1;
  }
  return lo;
}

}  // namespace split


namespace split {

// (sh, sl) += (bh, bl): error-free sum of the high parts, low parts added.
__device__ __forceinline__ void df_add(float &sh, float &sl, float2 b) {
  const float s = __fadd_rn(sh, b.x);
  const float bb = __fsub_rn(s, sh);
  const float err = __fadd_rn(__fsub_rn(sh, __fsub_rn(s, bb)), __fsub_rn(b.x, bb));
  sh = s;
  sl = __fadd_rn(sl, __fadd_rn(err, b.y));
}

// f in units of 2^-64 as a 128-bit integer (bits below 2^-64 dropped), with
// integer operations only; |f| < 2^60.
__device__ __forceinline__ __int128 fx128_f32(float f) {
  const unsigned u = __float_as_uint(f);
  const int ex = (int)((u >> 23) & 255u);
  if (ex == 0) return 0;  // zero or below 2^-126
  const long long m = (long long)((u & 0x7FFFFFu) | 0x800000u);
  const int sh = ex - 150 + 64;  // f = m 2^(ex - 150)
  __int128 v;
  if (sh >= 0) v = (__int128)m << sh;
  else v = sh > -24 ? (__int128)(m >> (-sh)) : (__int128)0;
  return (u >> 31) ? -v : v;
}

// Add -(v.x + v.y) (neg) or v.x + v.y to a fixed-point Sigma element
// (hi: 2^-32 units, lo: 2^-64 units) with integer arithmetic only.  Requires
// |v| < 2^31: the caller checks (fx_df_in_range) and records an error instead.
__device__ __forceinline__ void fx_add_df(unsigned long long *hi_lo, float2 v, bool neg) {
  __int128 V = fx128_f32(v.x) + fx128_f32(v.y);
  if (neg) V = -V;
  const long long hi = (long long)(V >> 32);
  const long long lo = (long long)(V & (__int128)0xFFFFFFFFll);
  if (hi) atomicAdd(hi_lo, (unsigned long long)hi);
  if (lo) atomicAdd(hi_lo + 1, (unsigned long long)lo);
}

// fx_add_df's range: |h| < 2^31 (false for NaN).
__device__ __forceinline__ bool fx_df_in_range(float h) { return fabsf(h) < 2147483648.f; }

// (sh, sl) += (ah, al) * (bh, bl), error-free products and sums (no
// contraction: every operation is an explicit round-to-nearest intrinsic).
__device__ __forceinline__ void df_mac(float &sh, float &sl, float2 a, float2 b) {
  const float p = __fmul_rn(a.x, b.x);
  float e = __fmaf_rn(a.x, b.x, -p);
  e = __fmaf_rn(a.x, b.y, e);
  e = __fmaf_rn(a.y, b.x, e);
  const float s = __fadd_rn(sh, p);
  const float bb = __fsub_rn(s, sh);
  const float err = __fadd_rn(__fsub_rn(sh, __fsub_rn(s, bb)), __fsub_rn(p, bb));
  sh = s;
  sl = __fadd_rn(sl, __fadd_rn(err, e));
}

// Two f32 lanes in one 64-bit register pair, with the packed f32x2
// arithmetic of sm_100 and later: each lane is rounded to nearest exactly as
// the scalar operation, so error-free transformations carry over lane-wise.
__device__ __forceinline__ uint64_t f2_pk(float x, float y) {
  uint64_t d;
  asm("mov.b64 %0, {%1, %2};" : "=l"(d) : "f"(x), "f"(y));
  return d;
}
__device__ __forceinline__ float2 f2_un(uint64_t v) {
  float2 r;
  asm("mov.b64 {%0, %1}, %2;" : "=f"(r.x), "=f"(r.y) : "l"(v));
  return r;
}
__device__ __forceinline__ uint64_t f2_add(uint64_t a, uint64_t b) {
  uint64_t d;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ uint64_t f2_sub(uint64_t a, uint64_t b) {
  uint64_t d;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ uint64_t f2_mul(uint64_t a, uint64_t b) {
  uint64_t d;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ uint64_t f2_fma(uint64_t a, uint64_t b, uint64_t c) {
  uint64_t d;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
  return d;
}

// df_mac in both lanes: (sh, sl) += (ah, al) (bh, bl), given na = -ah and
// nl = -al.  The product's error term is carried negated
// (ne = p - ah bh - ah bl - al bh), which gives the same roundings as df_mac.
__device__ __forceinline__ void df_mac2(uint64_t &sh, uint64_t &sl, uint64_t ah, uint64_t na,
                                        uint64_t nl, uint64_t bh, uint64_t bl) {
  const uint64_t p = f2_mul(ah, bh);
  uint64_t ne = f2_fma(na, bh, p);
  ne = f2_fma(na, bl, ne);
  ne = f2_fma(nl, bh, ne);
  const uint64_t s = f2_add(sh, p);
  const uint64_t bb = f2_sub(s, sh);
  const uint64_t err = f2_add(f2_sub(sh, f2_sub(s, bb)), f2_sub(p, bb));
  sh = s;
  sl = f2_add(sl, f2_sub(err, ne));
}

// Lane-wise double-float accumulation (s, r) += t: the sum s + t is split
// exactly (TwoSum), its error added to r.
__device__ __forceinline__ void df_acc2(uint64_t &s, uint64_t &r, uint64_t t) {
  const uint64_t s1 = f2_add(s, t);
  const uint64_t bb = f2_sub(s1, s);
  const uint64_t err = f2_add(f2_sub(s, f2_sub(s1, bb)), f2_sub(t, bb));
  s = s1;
  r = f2_add(r, err);
}

// (s, r) of lanes 0 and 1 renormalised (TwoSum) and scaled by 2^e0, 2^e1 in
// two exact steps each; exponents below -250 are taken as -250 (|s| < 2^64,
// so those values fall below the f32 range anyway).  Requires e <= 100.
__device__ __forceinline__ void df_fin2(uint64_t s, uint64_t r, int e0, int e1, float2 &o0,
                                        float2 &o1) {
  uint64_t h = 0, l = 0;
  df_acc2(h, l, s);
  df_acc2(h, l, r);
  e0 = max(e0, -250);
  e1 = max(e1, -250);
  const int a0 = e0 / 2, a1 = e1 / 2;
  const uint64_t f1 = f2_pk(__int_as_float((a0 + 127) << 23), __int_as_float((a1 + 127) << 23));
  const uint64_t f2 =
      f2_pk(__int_as_float((e0 - a0 + 127) << 23), __int_as_float((e1 - a1 + 127) << 23));
  const float2 H = f2_un(f2_mul(f2_mul(h, f1), f2)), L = f2_un(f2_mul(f2_mul(l, f1), f2));
  o0 = make_float2(H.x, L.x);
  o1 = make_float2(H.y, L.y);
}

}  // namespace split
