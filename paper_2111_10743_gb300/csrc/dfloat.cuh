// Double-float arithmetic (a value carried as the unevaluated sum hi + lo of
// two floats) and warp reductions shared by the far-field and correction
// kernels.
//
// Error-free transformations: TwoSum (Knuth), FastTwoSum (Dekker) and the
// fused-multiply-add TwoProduct; the reciprocal square root takes one Newton
// step y <- y + y (1 - x y^2) / 2 on the float32 seed.  Pairs are left
// unnormalised between operations: hi + lo stays an accurate unevaluated sum
// with |lo| within a few ulp of hi, and products drop only the lo * lo term.
#pragma once

#include <cuda_runtime.h>

struct F2 {
  float h, l;
};

__device__ __forceinline__ F2 two_sum(float a, float b) {
  const float s = a + b;
  const float bb = s - a;
  return {s, (a - (s - bb)) + (b - bb)};
}
__device__ __forceinline__ F2 fast_two_sum(float a, float b) {
  const float s = a + b;
  return {s, b - (s - a)};
}
__device__ __forceinline__ F2 df_add(F2 a, F2 b) {
  const F2 s = two_sum(a.h, b.h);
  return {s.h, s.l + (a.l + b.l)};
}
__device__ __forceinline__ F2 df_sub(F2 a, F2 b) { return df_add(a, {-b.h, -b.l}); }
__device__ __forceinline__ F2 df_mul(F2 a, F2 b) {
  const float p = a.h * b.h;
  return {p, fmaf(a.h, b.l, fmaf(a.l, b.h, fmaf(a.h, b.h, -p)))};
}
__device__ __forceinline__ F2 df_sqr(F2 a) {
  const float p = a.h * a.h;
  return {p, fmaf(a.h + a.h, a.l, fmaf(a.h, a.h, -p))};
}
__device__ __forceinline__ F2 df_scale(F2 a, float s) {  // s a power of two or small integer
  const float p = a.h * s;
  return {p, fmaf(a.h, s, -p) + a.l * s};
}
__device__ __forceinline__ float rsqrt_approx(float x) {  // one MUFU instruction
  float y;
  asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ F2 df_rsqrt(F2 x) {
  const float y = rsqrt_approx(x.h);
  const float yy = y * y;
  const F2 xy2 = df_mul(x, {yy, fmaf(y, y, -yy)});
  const float e = (1.f - xy2.h) - xy2.l;
  return fast_two_sum(y, 0.5f * y * e);
}
__device__ __forceinline__ void df_acc(F2& acc, F2 t) {
  const F2 s = two_sum(acc.h, t.h);
  acc.h = s.h;
  acc.l += s.l + t.l;
}
__device__ __forceinline__ F2 df_dot3(F2 a0, F2 a1, F2 a2, F2 b0, F2 b1, F2 b2) {
  return df_add(df_add(df_mul(a0, b0), df_mul(a1, b1)), df_mul(a2, b2));
}
__device__ __forceinline__ double df_to_double(F2 a) { return (double)a.h + (double)a.l; }

// ---- packed float32 pairs ---------------------------------------------------
// sm_100-family f32x2 instructions: one instruction on two floats held in a
// 64-bit register (the first operand of pk2 in the low half)
typedef unsigned long long u64;
__device__ __forceinline__ u64 pk2(float a, float b) {
  u64 r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
  return r;
}
__device__ __forceinline__ void upk2(u64 v, float& a, float& b) { asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(v)); }
__device__ __forceinline__ u64 add2(u64 a, u64 b) { u64 r; asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b)); return r; }
__device__ __forceinline__ u64 sub2(u64 a, u64 b) { u64 r; asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b)); return r; }
__device__ __forceinline__ u64 mul2(u64 a, u64 b) { u64 r; asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b)); return r; }
__device__ __forceinline__ u64 fma2(u64 a, u64 b, u64 c) {
  u64 r;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(a), "l"(b), "l"(c));
  return r;
}

// float64 addition to global memory without a returned value (the symmetric
// pair kernels' sums; the order of additions is not fixed)
__device__ __forceinline__ void red_add_f64(double* p, double v) {
  asm volatile("red.global.add.f64 [%0], %1;" ::"l"(p), "d"(v) : "memory");
}

// block pair (I, J), I <= J, of the linear index lin = J (J + 1) / 2 + I
__device__ __forceinline__ void tri_pair(int64_t lin, int64_t& I, int64_t& J) {
  J = (int64_t)((sqrt(8.0 * (double)lin + 1.0) - 1.0) * 0.5);
  while (J * (J + 1) / 2 > lin) --J;
  while ((J + 1) * (J + 2) / 2 <= lin) ++J;
  I = lin - J * (J + 1) / 2;
}

// ---- warp reductions --------------------------------------------------------
__device__ __forceinline__ float shfl_xor_v(float v, int off) { return __shfl_xor_sync(0xffffffffu, v, off); }
__device__ __forceinline__ double shfl_xor_v(double v, int off) { return __shfl_xor_sync(0xffffffffu, v, off); }
__device__ __forceinline__ F2 shfl_xor_v(F2 v, int off) {
  return {__shfl_xor_sync(0xffffffffu, v.h, off), __shfl_xor_sync(0xffffffffu, v.l, off)};
}
__device__ __forceinline__ F2 shfl_idx_v(F2 v, int src) {
  return {__shfl_sync(0xffffffffu, v.h, src), __shfl_sync(0xffffffffu, v.l, src)};
}
__device__ __forceinline__ float add_v(float a, float b) { return a + b; }
__device__ __forceinline__ double add_v(double a, double b) { return a + b; }
__device__ __forceinline__ F2 add_v(F2 a, F2 b) { return df_add(a, b); }

// Reduce-scatter over a warp of V values per lane (V a power of two, at most
// 32): at each of the five butterfly stages a lane keeps half of the values
// it still holds and adds its partner's copy of that half, so that 31
// shuffles (rather than 5 V) leave in v[0] of lane L the warp total of value
// index L >> (5 - log2 V); value idx ends in lanes idx << (5 - log2 V) and up.
template <int V, typename T>
__device__ __forceinline__ void warp_reduce_scatter(T (&v)[V], int lane) {
#pragma unroll
  for (int s = 0; s < 5; ++s) {
    const int off = 16 >> s;
    const int half = V >> (s + 1);  // values kept after this stage
    if (half >= 1) {
      const bool up = (lane & off) != 0;
#pragma unroll
      for (int j = 0; j < half; ++j) {
        const T lo = v[j], hi = v[j + half];
        const T send = up ? lo : hi;
        const T keep = up ? hi : lo;
        v[j] = add_v(keep, shfl_xor_v(send, off));
      }
    } else {
      v[0] = add_v(v[0], shfl_xor_v(v[0], off));
    }
  }
}

// log2 of a power of two known at compile time
template <int V> struct Log2 { static const int value = 1 + Log2<V / 2>::value; };
template <> struct Log2<1> { static const int value = 0; };
