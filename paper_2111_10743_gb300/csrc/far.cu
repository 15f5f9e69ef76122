// Far-field pair sums, near-field correction SpMV and the A2 / A3 applies.
//
// A discretised potential at node i (Section 4, the corrected Nystrom form)
// is the smooth-rule sum over all sources outside Near(i) plus the sum of
// precomputed correction blocks over the patches in Near(i):
//   K[sigma]_i = sum_{j : patch(j) not in Near(i)} w_j K(x_i, x_j) sigma_j
//              + sum_{P in Near(i)} sum_q W^K_{i,P}[q] sigma_{P,q}.
// Kernels (Section 3), d = x - y, r = |d|, G = 1/(4 pi r):
//   S = 1/(4 pi r),  D = n_y.d/(4 pi r^3),  S' = -n_x.d/(4 pi r^3),
//   S''+D' = [3 (n_x.d)((n_x - n_y).d)/r^2 - |n_x - n_y|^2/2]/(4 pi r^3)
// (for unit normals |n_x - n_y|^2/2 = 1 - n_x.n_y; the difference form avoids
// cancellation in float32).
//
// Pair kernels (the FMM calls of Section 4.2 / 4.3, Table 1, done as exact
// direct sums): each thread owns NT targets in registers, the CTA stages TS
// sources at a time in shared memory (one float4/double4_32a of position and
// charge, one of normal and second charge), and the source range is split
// over gridDim.y so that every SM holds several CTAs; split partials are
// reduced in a fixed order by the epilogue (deterministic).  Near pairs are
// skipped exactly: a per-(target block, source tile) flag selects a masked
// inner loop only where some target of the block has some patch of the tile
// in its near list.  float32 sums accumulate per tile in float32 and are
// folded into a float-float (TwoSum) running total after every tile.
//
// Operator applies (Sections 4.2, 4.3), W[f] = sum w f / sum w:
//   A3: pass 1 (charge tau) -> mu1 = S' tau, mu2 = S tau;
//       pass 2 (charges mu1, mu2; dipole for S''+D') ->
//       A3 tau = -tau/4 + S'[mu1] - (S''+D')[mu2] - 2 H S'[mu2] + W S[mu2].
//   A2: pass 1 (charge tau) -> S, D, S', S''+D' of tau;
//       mu1 = D tau, mu2 = -(S''+D') tau - 2 H S' tau + W S tau;
//       pass 2 -> A2 tau = -tau/4 + D[mu1] + S[mu2]
//       (the printed "- D[mu1]" is read as + D[mu1]: A2 contains +D^2).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <map>
#include <mutex>
#include <tuple>
#include <type_traits>

#include "dfloat.cuh"
#include "internal.cuh"

template <typename R> struct V4T;
template <> struct V4T<float> { typedef float4 type; };
template <> struct V4T<double> { typedef double4_32a type; };

// one MUFU instruction (approximate, flushes subnormals: pair distances here
// are far from the subnormal range)
__device__ __forceinline__ float lb_rsqrt(float x) {
  float y;
  asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ double lb_rsqrt(double x) { return rsqrt(x); }

// float-float running total: hi + lo, updated with TwoSum (Knuth)
struct FF {
  float hi, lo;
  __device__ __forceinline__ void add(float p) {
    float s = hi + p;
    float bp = s - hi;
    float e = (hi - (s - bp)) + (p - bp);
    hi = s;
    lo += e;
  }
};

template <int KIND> struct FarOut { static const int n = 4; };
template <> struct FarOut<FAR_K4> { static const int n = 2; };

template <typename R, int KIND>
__device__ __forceinline__ void far_pair(const R tx, const R ty, const R tz, const R nx, const R ny, const R nz,
                                         const typename V4T<R>::type& a, const typename V4T<R>::type& b,
                                         bool masked, R* acc) {
  const R dx = tx - a.x, dy = ty - a.y, dz = tz - a.z;
  const R r2 = dx * dx + dy * dy + dz * dz;
  R rinv = lb_rsqrt(r2);
  if (masked) rinv = R(0);
  if (KIND == FAR_K1) {
    const R qr = a.w * rinv;
    acc[0] += qr;
    const R t = qr * rinv * rinv;
    acc[1] += t * dx;
    acc[2] += t * dy;
    acc[3] += t * dz;
  } else if (KIND == FAR_KALL) {
    const R rinv2 = rinv * rinv;
    const R rinv3 = rinv2 * rinv;
    const R nxd = nx * dx + ny * dy + nz * dz;
    const R nyd = b.x * dx + b.y * dy + b.z * dz;
    const R ex = nx - b.x, ey = ny - b.y, ez = nz - b.z;
    const R dnd = ex * dx + ey * dy + ez * dz;
    const R dn2 = ex * ex + ey * ey + ez * ez;
    const R qr3 = a.w * rinv3;
    acc[0] += a.w * rinv;
    acc[1] += qr3 * nyd;
    acc[2] += qr3 * nxd;
    acc[3] += qr3 * (R(3) * nxd * dnd * rinv2 - R(0.5) * dn2);
  } else if (KIND == FAR_K2) {
    const R rinv2 = rinv * rinv;
    const R rinv3 = rinv2 * rinv;
    const R nxd = nx * dx + ny * dy + nz * dz;
    const R t = nxd * rinv3;
    acc[0] += a.w * t;
    acc[1] += b.w * rinv;
    acc[2] += b.w * t;
    const R ex = nx - b.x, ey = ny - b.y, ez = nz - b.z;
    const R dnd = ex * dx + ey * dy + ez * dz;
    const R dn2 = ex * ex + ey * ey + ez * ez;
    acc[3] += b.w * rinv3 * ((nxd * dnd) * (R(3) * rinv2) - R(0.5) * dn2);
  } else {  // FAR_K4
    const R rinv3 = rinv * rinv * rinv;
    const R nyd = b.x * dx + b.y * dy + b.z * dz;
    acc[0] += a.w * nyd * rinv3;
    acc[1] += b.w * rinv;
  }
}

template <typename R, int KIND, int NT, int NTH, int TS>
__global__ void __launch_bounds__(NTH) k_far(int64_t N, int np, const typename V4T<R>::type* __restrict__ tpos,
                                             const typename V4T<R>::type* __restrict__ tnrm,
                                             const typename V4T<R>::type* __restrict__ srcA,
                                             const typename V4T<R>::type* __restrict__ srcB,
                                             const uint8_t* __restrict__ flags, int64_t ntiles,
                                             const int64_t* __restrict__ row_ptr,
                                             const int32_t* __restrict__ near_patch, int tiles_per_split,
                                             double* __restrict__ part) {
  typedef typename V4T<R>::type V4;
  constexpr int NO = FarOut<KIND>::n;
  constexpr bool kUseB = KIND != FAR_K1;
  __shared__ V4 sA[TS];
  __shared__ V4 sB[kUseB ? TS : 1];
  __shared__ int sLp[TS];

  const int64_t t0 = (int64_t)blockIdx.x * (NTH * NT);
  R tx[NT], ty[NT], tz[NT], nx[NT], ny[NT], nz[NT];
#pragma unroll
  for (int j = 0; j < NT; ++j) {
    const int64_t t = t0 + threadIdx.x + j * NTH;
    const V4 p = tpos[t];
    tx[j] = p.x; ty[j] = p.y; tz[j] = p.z;
    if (KIND != FAR_K1 && KIND != FAR_K4) {
      const V4 q = tnrm[t];
      nx[j] = q.x; ny[j] = q.y; nz[j] = q.z;
    } else {
      nx[j] = ny[j] = nz[j] = R(0);
    }
  }
  R acc[NT][NO];
  FF tot[NT][NO];
#pragma unroll
  for (int j = 0; j < NT; ++j)
#pragma unroll
    for (int o = 0; o < NO; ++o) {
      acc[j][o] = R(0);
      tot[j][o].hi = 0.f;
      tot[j][o].lo = 0.f;
    }

  const int64_t tile_b = (int64_t)blockIdx.y * tiles_per_split;
  const int64_t tile_e = min(ntiles, tile_b + tiles_per_split);
  for (int64_t tile = tile_b; tile < tile_e; ++tile) {
    const int64_t s0 = tile * TS;
    const int64_t P0 = s0 / np;
    for (int s = threadIdx.x; s < TS; s += NTH) {
      sA[s] = srcA[s0 + s];
      if (kUseB) sB[s] = srcB[s0 + s];
      sLp[s] = (int)((s0 + s) / np - P0);
    }
    __syncthreads();
    const bool any_near = flags[(int64_t)blockIdx.x * ntiles + tile] != 0;
    if (!any_near) {
#pragma unroll 8
      for (int s = 0; s < TS; ++s) {
        const V4 a = sA[s];
        const V4 b = kUseB ? sB[s] : a;
#pragma unroll
        for (int j = 0; j < NT; ++j)
          far_pair<R, KIND>(tx[j], ty[j], tz[j], nx[j], ny[j], nz[j], a, b, false, acc[j]);
      }
    } else {
      unsigned long long m[NT];
#pragma unroll
      for (int j = 0; j < NT; ++j) {
        const int64_t t = t0 + threadIdx.x + j * NTH;
        m[j] = 0ull;
        if (t < N)
          for (int64_t bb = row_ptr[t]; bb < row_ptr[t + 1]; ++bb) {
            const int64_t d = (int64_t)near_patch[bb] - P0;
            if (d >= 0 && d < 64) m[j] |= 1ull << d;
          }
      }
      for (int s = 0; s < TS; ++s) {
        const V4 a = sA[s];
        const V4 b = kUseB ? sB[s] : a;
        const int lp = sLp[s];
#pragma unroll
        for (int j = 0; j < NT; ++j)
          far_pair<R, KIND>(tx[j], ty[j], tz[j], nx[j], ny[j], nz[j], a, b, (m[j] >> lp) & 1ull, acc[j]);
      }
    }
    if (sizeof(R) == 4) {
#pragma unroll
      for (int j = 0; j < NT; ++j)
#pragma unroll
        for (int o = 0; o < NO; ++o) {
          tot[j][o].add((float)acc[j][o]);
          acc[j][o] = R(0);
        }
    }
    __syncthreads();
  }
#pragma unroll
  for (int j = 0; j < NT; ++j) {
    const int64_t t = t0 + threadIdx.x + j * NTH;
    if (t >= N) continue;
#pragma unroll
    for (int o = 0; o < NO; ++o) {
      const int64_t k = ((int64_t)blockIdx.y * NO + o) * N + t;
      if (sizeof(R) == 4)  // float32 partials as (hi, lo) pairs
        reinterpret_cast<float2*>(part)[k] = make_float2(tot[j][o].hi, tot[j][o].lo);
      else
        part[k] = (double)acc[j][o];
    }
  }
}

// ---------------------------------------------------------------------------
// float32 pair kernels with packed two-lane arithmetic (sm_100 family
// f32x2 add/sub/mul/fma): each target is held splatted in both halves of a
// 64-bit register and every instruction evaluates the target against two
// consecutive sources, halving the issued instructions per pair (used for
// the longer kernels K2, KALL, K4; the short K1 measured faster scalar).  Sources
// are staged as structure-of-arrays so that consecutive pairs load directly
// as packed operands.  Tiles with near pairs fall back to the scalar loop.
__device__ __forceinline__ u64 rsqrt2(u64 x) {
  float a, b;
  upk2(x, a, b);
  return pk2(lb_rsqrt(a), lb_rsqrt(b));
}

// two pairs (one target, sources s and s+1); T: target x, y, z, nx, ny, nz
// splatted; S: packed source components x, y, z, q1, nx, ny, nz, q2
template <int KIND>
__device__ __forceinline__ void pair2(const u64* T, const u64* S, u64* acc, const u64 three, const u64 mhalf) {
  const u64 dx = sub2(T[0], S[0]), dy = sub2(T[1], S[1]), dz = sub2(T[2], S[2]);
  const u64 r2 = fma2(dz, dz, fma2(dy, dy, mul2(dx, dx)));
  const u64 rinv = rsqrt2(r2);
  if (KIND == FAR_K1) {
    const u64 qr = mul2(S[3], rinv);
    acc[0] = add2(acc[0], qr);
    const u64 t = mul2(qr, mul2(rinv, rinv));
    acc[1] = fma2(t, dx, acc[1]);
    acc[2] = fma2(t, dy, acc[2]);
    acc[3] = fma2(t, dz, acc[3]);
    return;
  }
  const u64 rinv2 = mul2(rinv, rinv);
  const u64 rinv3 = mul2(rinv2, rinv);
  if (KIND == FAR_K4) {
    const u64 nyd = fma2(S[6], dz, fma2(S[5], dy, mul2(S[4], dx)));
    acc[0] = fma2(mul2(S[3], rinv3), nyd, acc[0]);
    acc[1] = fma2(S[7], rinv, acc[1]);
    return;
  }
  const u64 nxd = fma2(T[5], dz, fma2(T[4], dy, mul2(T[3], dx)));
  const u64 ex = sub2(T[3], S[4]), ey = sub2(T[4], S[5]), ez = sub2(T[5], S[6]);
  const u64 dnd = fma2(ez, dz, fma2(ey, dy, mul2(ex, dx)));
  const u64 dn2 = fma2(ez, ez, fma2(ey, ey, mul2(ex, ex)));
  const u64 kk = fma2(mul2(nxd, dnd), mul2(three, rinv2), mul2(mhalf, dn2));
  if (KIND == FAR_KALL) {
    const u64 qr3 = mul2(S[3], rinv3);
    const u64 nyd = sub2(nxd, dnd);
    acc[0] = fma2(S[3], rinv, acc[0]);
    acc[1] = fma2(qr3, nyd, acc[1]);
    acc[2] = fma2(qr3, nxd, acc[2]);
    acc[3] = fma2(qr3, kk, acc[3]);
  } else {  // FAR_K2
    const u64 t = mul2(nxd, rinv3);
    acc[0] = fma2(S[3], t, acc[0]);
    acc[1] = fma2(S[7], rinv, acc[1]);
    acc[2] = fma2(S[7], t, acc[2]);
    acc[3] = fma2(mul2(S[7], rinv3), kk, acc[3]);
  }
}

template <int KIND, int NT, int NTH, int TS, int MINB = 1>
__global__ void __launch_bounds__(NTH, MINB) k_far32x2(int64_t N, int np, const float4* __restrict__ tpos,
                                                 const float4* __restrict__ tnrm, const float4* __restrict__ srcA,
                                                 const float4* __restrict__ srcB, const uint8_t* __restrict__ flags,
                                                 int64_t ntiles, const int64_t* __restrict__ row_ptr,
                                                 const int32_t* __restrict__ near_patch, int tiles_per_split,
                                                 double* __restrict__ part) {
  constexpr int NO = FarOut<KIND>::n;
  constexpr bool kUseB = KIND != FAR_K1;
  constexpr int NC = kUseB ? 8 : 4;                   // staged source components
  constexpr bool kTN = KIND == FAR_K2 || KIND == FAR_KALL;  // target normals needed
  __shared__ __align__(16) float sS[NC][TS];
  __shared__ int sLp[TS];
  const int64_t t0 = (int64_t)blockIdx.x * (NTH * NT);
  u64 T[NT][6];
  float tf[NT][6];
#pragma unroll
  for (int j = 0; j < NT; ++j) {
    const int64_t t = t0 + threadIdx.x + j * NTH;
    const float4 p = tpos[t];
    tf[j][0] = p.x; tf[j][1] = p.y; tf[j][2] = p.z;
    tf[j][3] = tf[j][4] = tf[j][5] = 0.f;
    if (kTN) {
      const float4 q = tnrm[t];
      tf[j][3] = q.x; tf[j][4] = q.y; tf[j][5] = q.z;
    }
#pragma unroll
    for (int k = 0; k < 6; ++k) T[j][k] = pk2(tf[j][k], tf[j][k]);
  }
  const u64 three = pk2(3.f, 3.f), mhalf = pk2(-0.5f, -0.5f);
  u64 acc[NT][NO];
  FF tot[NT][NO];
#pragma unroll
  for (int j = 0; j < NT; ++j)
#pragma unroll
    for (int o = 0; o < NO; ++o) {
      acc[j][o] = 0ull;
      tot[j][o].hi = 0.f;
      tot[j][o].lo = 0.f;
    }
  const int64_t tile_b = (int64_t)blockIdx.y * tiles_per_split;
  const int64_t tile_e = min(ntiles, tile_b + tiles_per_split);
  for (int64_t tile = tile_b; tile < tile_e; ++tile) {
    const int64_t s0 = tile * TS;
    const int64_t P0 = s0 / np;
    for (int s = threadIdx.x; s < TS; s += NTH) {
      const float4 a = srcA[s0 + s];
      sS[0][s] = a.x; sS[1][s] = a.y; sS[2][s] = a.z; sS[3][s] = a.w;
      if (kUseB) {
        const float4 b = srcB[s0 + s];
        sS[4][s] = b.x; sS[5][s] = b.y; sS[6][s] = b.z; sS[7][s] = b.w;
      }
      sLp[s] = (int)((s0 + s) / np - P0);
    }
    __syncthreads();
    const bool any_near = flags[(int64_t)blockIdx.x * ntiles + tile] != 0;
    if (!any_near) {
#pragma unroll 2
      for (int s = 0; s < TS; s += 4) {
        u64 S0[8], S1[8];
#pragma unroll
        for (int c = 0; c < NC; ++c) {
          const float4 v = *reinterpret_cast<const float4*>(&sS[c][s]);
          S0[c] = pk2(v.x, v.y);
          S1[c] = pk2(v.z, v.w);
        }
#pragma unroll
        for (int j = 0; j < NT; ++j) {
          pair2<KIND>(T[j], S0, acc[j], three, mhalf);
          pair2<KIND>(T[j], S1, acc[j], three, mhalf);
        }
      }
    } else {
      // scalar loop with the per-target near-patch mask
      unsigned long long m[NT];
#pragma unroll
      for (int j = 0; j < NT; ++j) {
        const int64_t t = t0 + threadIdx.x + j * NTH;
        m[j] = 0ull;
        if (t < N)
          for (int64_t bb = row_ptr[t]; bb < row_ptr[t + 1]; ++bb) {
            const int64_t d = (int64_t)near_patch[bb] - P0;
            if (d >= 0 && d < 64) m[j] |= 1ull << d;
          }
      }
      for (int s = 0; s < TS; ++s) {
        const float4 a = make_float4(sS[0][s], sS[1][s], sS[2][s], sS[3][s]);
        const float4 b = kUseB ? make_float4(sS[4][s], sS[5][s], sS[6][s], sS[7][s]) : a;
        const int lp = sLp[s];
#pragma unroll
        for (int j = 0; j < NT; ++j) {
          float sa[4] = {0.f, 0.f, 0.f, 0.f};
          far_pair<float, KIND>(tf[j][0], tf[j][1], tf[j][2], tf[j][3], tf[j][4], tf[j][5], a, b,
                                (m[j] >> lp) & 1ull, sa);
#pragma unroll
          for (int o = 0; o < NO; ++o) acc[j][o] = add2(acc[j][o], pk2(sa[o], 0.f));
        }
      }
    }
#pragma unroll
    for (int j = 0; j < NT; ++j)
#pragma unroll
      for (int o = 0; o < NO; ++o) {
        float lo, hi;
        upk2(acc[j][o], lo, hi);
        tot[j][o].add(lo + hi);
        acc[j][o] = 0ull;
      }
    __syncthreads();
  }
#pragma unroll
  for (int j = 0; j < NT; ++j) {
    const int64_t t = t0 + threadIdx.x + j * NTH;
    if (t >= N) continue;
#pragma unroll
    for (int o = 0; o < NO; ++o)
      reinterpret_cast<float2*>(part)[((int64_t)blockIdx.y * NO + o) * N + t] =
          make_float2(tot[j][o].hi, tot[j][o].lo);
  }
}

// ---------------------------------------------------------------------------
// Symmetric float32 pair sums (A3 passes K1 and K2, node sources): each
// unordered pair {i, j} evaluated once for both directions, in the layout of
// the double-float kernel k_far_df_sym (far_df.cu): CTAs over block pairs
// I <= J of 128 nodes, target sums in registers, source sums circulating one
// lane per step through 32 x 32 warp tiles, float64 red.add of each CTA's
// sums.  d, r, 1/r, 1/r^3, n_i.d, n_j.d and |n_i - n_j|^2 are shared; for
// target j, d -> -d.  Block pairs without a near pair in either direction
// take a loop without masks.
template <int KIND, bool MASKED>
__device__ __forceinline__ void f32_pair_sym(const float4& ta, const float4& tb, const float4& a, const float4& b,
                                             bool mi, bool mj, float* acci, float* accj) {
  // ta = (x_i, q1_i), tb = (n_i, q2_i); a = (y_j, q1_j), b = (n_j, q2_j)
  const float dx = ta.x - a.x, dy = ta.y - a.y, dz = ta.z - a.z;
  const float r2 = fmaf(dz, dz, fmaf(dy, dy, dx * dx));
  float rinv = lb_rsqrt(r2);
  float q1j = a.w, q1i = ta.w;
  if (MASKED) {
    if (mi && mj) rinv = 0.f;
    if (mi) q1j = 0.f;
    if (mj) q1i = 0.f;
  }
  const float rinv2 = rinv * rinv, rinv3 = rinv2 * rinv;
  if (KIND == FAR_K1) {
    acci[0] = fmaf(q1j, rinv, acci[0]);
    accj[0] = fmaf(q1i, rinv, accj[0]);
    const float tj = q1j * rinv3, ti = q1i * rinv3;
    acci[1] = fmaf(tj, dx, acci[1]);
    acci[2] = fmaf(tj, dy, acci[2]);
    acci[3] = fmaf(tj, dz, acci[3]);
    accj[1] = fmaf(-ti, dx, accj[1]);
    accj[2] = fmaf(-ti, dy, accj[2]);
    accj[3] = fmaf(-ti, dz, accj[3]);
    return;
  }
  float q2j = b.w, q2i = tb.w;
  if (MASKED) {
    if (mi) q2j = 0.f;
    if (mj) q2i = 0.f;
  }
  const float an = fmaf(tb.z, dz, fmaf(tb.y, dy, tb.x * dx));  // n_i.d
  const float ex = tb.x - b.x, ey = tb.y - b.y, ez = tb.z - b.z;
  const float cn = fmaf(ez, dz, fmaf(ey, dy, ex * dx));          // (n_i - n_j).d
  const float bn = an - cn;                                      // n_j.d
  const float hd = 0.5f * fmaf(ez, ez, fmaf(ey, ey, ex * ex));  // 1 - n_i.n_j
  const float c3 = cn * (3.f * rinv2);
  // target i: 3 a c / r^2 - hd; target j: -(3 b c / r^2 + hd)
  const float kki = fmaf(an, c3, -hd), kkj = fmaf(bn, c3, hd);
  const float tti = an * rinv3, ttj = bn * rinv3;
  acci[0] = fmaf(q1j, tti, acci[0]);
  acci[1] = fmaf(q2j, rinv, acci[1]);
  acci[2] = fmaf(q2j, tti, acci[2]);
  acci[3] = fmaf(q2j * rinv3, kki, acci[3]);
  accj[0] = fmaf(-q1i, ttj, accj[0]);
  accj[1] = fmaf(q2i, rinv, accj[1]);
  accj[2] = fmaf(-q2i, ttj, accj[2]);
  accj[3] = fmaf(-q2i * rinv3, kkj, accj[3]);
}

// Two unordered pairs at once in packed f32x2 arithmetic: one target
// (components splatted in both halves) against two consecutive sources (one
// per half).  T: target x, y, z, n_x, n_y, n_z; QI1, QI2 its charges and
// QI1N = -QI1; S: packed source x, y, z, q1, n_x, n_y, n_z, q2.  acci: the
// target's sums per source half; accj: the two sources' sums.
template <int KIND>
__device__ __forceinline__ void pair2_sym(const u64* T, u64 QI1, u64 QI1N, u64 QI2, const u64* S, u64* acci,
                                          u64* accj, const u64 three, const u64 mhalf) {
  const u64 dx = sub2(T[0], S[0]), dy = sub2(T[1], S[1]), dz = sub2(T[2], S[2]);
  const u64 r2 = fma2(dz, dz, fma2(dy, dy, mul2(dx, dx)));
  const u64 rinv = rsqrt2(r2);
  const u64 rinv2 = mul2(rinv, rinv), rinv3 = mul2(rinv2, rinv);
  if (KIND == FAR_K1) {
    acci[0] = fma2(S[3], rinv, acci[0]);
    accj[0] = fma2(QI1, rinv, accj[0]);
    const u64 tj = mul2(S[3], rinv3), tin = mul2(QI1N, rinv3);
    acci[1] = fma2(tj, dx, acci[1]);
    acci[2] = fma2(tj, dy, acci[2]);
    acci[3] = fma2(tj, dz, acci[3]);
    accj[1] = fma2(tin, dx, accj[1]);
    accj[2] = fma2(tin, dy, accj[2]);
    accj[3] = fma2(tin, dz, accj[3]);
    return;
  }
  const u64 an = fma2(T[5], dz, fma2(T[4], dy, mul2(T[3], dx)));       // n_i.d
  const u64 ex = sub2(T[3], S[4]), ey = sub2(T[4], S[5]), ez = sub2(T[5], S[6]);
  const u64 cn = fma2(ez, dz, fma2(ey, dy, mul2(ex, dx)));             // (n_i - n_j).d
  const u64 bneg = sub2(cn, an);                                       // -n_j.d
  const u64 hdn = mul2(mhalf, fma2(ez, ez, fma2(ey, ey, mul2(ex, ex))));  // -(1 - n_i.n_j)
  const u64 c3 = mul2(cn, mul2(three, rinv2));
  const u64 kki = fma2(an, c3, hdn);     // 3 a c / r^2 - (1 - n_i.n_j)
  const u64 kkjn = fma2(bneg, c3, hdn);  // -(3 b c / r^2 + 1 - n_i.n_j)
  const u64 tti = mul2(an, rinv3), ttjn = mul2(bneg, rinv3);
  acci[0] = fma2(S[3], tti, acci[0]);
  acci[1] = fma2(S[7], rinv, acci[1]);
  acci[2] = fma2(S[7], tti, acci[2]);
  acci[3] = fma2(mul2(S[7], rinv3), kki, acci[3]);
  accj[0] = fma2(QI1, ttjn, accj[0]);
  accj[1] = fma2(QI2, rinv, accj[1]);
  accj[2] = fma2(QI2, ttjn, accj[2]);
  accj[3] = fma2(mul2(QI2, rinv3), kkjn, accj[3]);
}

__device__ __forceinline__ u64 shfl_u64(u64 v, int src) {
  float a, b;
  upk2(v, a, b);
  return pk2(__shfl_sync(0xffffffffu, a, src), __shfl_sync(0xffffffffu, b, src));
}

// NT: targets per lane (the CTA has 128 / NT threads for a 128-node block),
// so that each source load and each rotation step serves NT pairs; MINB:
// resident blocks per SM asked of ptxas (0: unspecified)
template <int KIND, bool PACKED, int NT, int MINB = 0>
__global__ void __launch_bounds__(128 / NT, MINB) k_far32_sym(int64_t N, int np, const float4* __restrict__ srcA,
                                                        const float4* __restrict__ srcB,
                                                        const uint8_t* __restrict__ flags, int64_t ntiles,
                                                        const int64_t* __restrict__ row_ptr,
                                                        const int32_t* __restrict__ near_patch,
                                                        double* __restrict__ out) {
  constexpr int NO = 4, B = 128, NTH = B / NT, NW = NTH / 32;
  constexpr bool kB = KIND != FAR_K1;
  // scalar loop: each 32-source tile stored twice over (64 entries), so that
  // lane t reads source (t + k) mod 32 of tile r at entry 64 r + t + k: a
  // per-lane base address plus the step as an immediate offset.  The packed
  // forms read these tiles only in the masked and diagonal loops and keep
  // one copy (entry 32 r + (t + k) mod 32), which saves the shared memory
  // that bounds their resident blocks.
  constexpr int DUP = PACKED ? 1 : 2;
  __shared__ float4 sA[DUP * B], sB[kB ? DUP * B : 1];
  // packed loop: the same tiles pair-interleaved, entry e of tile r holding
  // (c_e, c_(e+1 mod 32)) for two components c per plane (planes: x y, z q1,
  // n_x n_y, n_z q2), so that one 16-byte load gives two packed operands
  constexpr int NPL = PACKED ? (kB ? 4 : 2) : 1;
  __shared__ float4 sP[NPL][PACKED ? B : 1];
  __shared__ unsigned long long sMask[B];
  __shared__ int sLp[B];
  __shared__ float sRed[NW][B][NO];
  int64_t I, J;
  tri_pair(blockIdx.x, I, J);
  const bool diag = I == J;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int64_t P0I = (I * B) / np, P0J = (J * B) / np;
  const bool any = flags[I * ntiles + J] != 0 || flags[J * ntiles + I] != 0;
#pragma unroll
  for (int u = 0; u < NT; ++u) {  // stage block J: this thread's sources ls = tid + u NTH
    const int ls = tid + u * NTH, rt = ls >> 5;
    const int64_t j = J * B + ls;
    const int e = 32 * DUP * rt + lane;
    const float4 va = srcA[j];
    const float4 vb = kB ? srcB[j] : va;
    sA[e] = va;
    if (!PACKED) sA[e + 32] = va;
    if (kB) {
      sB[e] = vb;
      if (!PACKED) sB[e + 32] = vb;
    }
    if (PACKED) {
      // this source is the first element of entry lane and the second of
      // entry lane - 1 (mod 32) of its tile
      const float c[8] = {va.x, va.y, va.z, va.w, vb.x, vb.y, vb.z, vb.w};
      const int f0 = 32 * rt + lane, g0 = 32 * rt + ((lane + 31) & 31);
#pragma unroll
      for (int p = 0; p < NPL; ++p) {
        float* a0 = reinterpret_cast<float*>(&sP[p][f0]);
        float* b0 = reinterpret_cast<float*>(&sP[p][g0]);
        a0[0] = c[2 * p];
        a0[2] = c[2 * p + 1];
        b0[1] = c[2 * p];
        b0[3] = c[2 * p + 1];
      }
    }
    sLp[ls] = (int)(j / np - P0J);
    unsigned long long mj = 0ull;
    if (any && !diag && j < N)
      for (int64_t bb = row_ptr[j]; bb < row_ptr[j + 1]; ++bb) {
        const int64_t d = (int64_t)near_patch[bb] - P0I;
        if (d >= 0 && d < 64) mj |= 1ull << d;
      }
    sMask[ls] = mj;
  }
  // the targets i = I B + tid + t NTH: data, i-side masks, patch offsets
  float4 ta[NT], tb[NT];
  unsigned long long mi[NT];
  int lpi[NT];
  bool pad[NT];
  float acci[NT][NO];
#pragma unroll
  for (int t = 0; t < NT; ++t) {
    const int64_t i = I * B + tid + t * NTH;
    ta[t] = srcA[i];
    tb[t] = kB ? srcB[i] : ta[t];
    mi[t] = 0ull;
    if (any && i < N)
      for (int64_t bb = row_ptr[i]; bb < row_ptr[i + 1]; ++bb) {
        const int64_t d = (int64_t)near_patch[bb] - P0J;
        if (d >= 0 && d < 64) mi[t] |= 1ull << d;
      }
    lpi[t] = (int)(i / np - P0I);
    pad[t] = i >= N;
#pragma unroll
    for (int o = 0; o < NO; ++o) acci[t][o] = 0.f;
  }
  __syncthreads();
  const int up = (lane + 1) & 31;
  if (diag) {  // the target side only (padded targets lie in this block only)
    float none[NO] = {0.f, 0.f, 0.f, 0.f};
    for (int s = 0; s < B; ++s) {
      const int e = 32 * DUP * (s >> 5) + (s & 31);
#pragma unroll
      for (int t = 0; t < NT; ++t) {
        const bool msk_i = pad[t] || ((mi[t] >> sLp[s]) & 1ull);
        f32_pair_sym<KIND, true>(ta[t], tb[t], sA[e], kB ? sB[e] : sA[e], msk_i, true, acci[t], none);
      }
    }
  } else {
    // 32 x 32 warp tiles: lane t takes source (t + k) mod 32 at step k; the
    // source sums move one lane down after each step
    for (int r = 0; r < B / 32; ++r) {
      float accj[NO] = {0.f, 0.f, 0.f, 0.f};
      const float4* pa = sA + 32 * DUP * r;
      const float4* pb = kB ? sB + 32 * DUP * r : pa;
      if (!any && PACKED) {
        // lane t takes sources t + 2k and t + 2k + 1 at step k; its two
        // source-sum slots move two lanes down after each step, so that lane
        // t ends with source t in the low slot and source t + 1 in the high
        u64 T[NT][6], QI1[NT], QI1N[NT], QI2[NT];
#pragma unroll
        for (int t = 0; t < NT; ++t) {
          T[t][0] = pk2(ta[t].x, ta[t].x); T[t][1] = pk2(ta[t].y, ta[t].y); T[t][2] = pk2(ta[t].z, ta[t].z);
          T[t][3] = pk2(tb[t].x, tb[t].x); T[t][4] = pk2(tb[t].y, tb[t].y); T[t][5] = pk2(tb[t].z, tb[t].z);
          QI1[t] = pk2(ta[t].w, ta[t].w);
          QI1N[t] = pk2(-ta[t].w, -ta[t].w);
          QI2[t] = pk2(tb[t].w, tb[t].w);
        }
        const u64 three = pk2(3.f, 3.f), mhalf = pk2(-0.5f, -0.5f);
        const int up2 = (lane + 2) & 31;
        u64 ai[NT][NO], aj[NO] = {0ull, 0ull, 0ull, 0ull};
#pragma unroll
        for (int t = 0; t < NT; ++t)
#pragma unroll
          for (int o = 0; o < NO; ++o) ai[t][o] = 0ull;
        const float4* q = &sP[0][32 * r];
#pragma unroll 4
        for (int k = 0; k < 16; ++k) {
          const int e = (lane + 2 * k) & 31;
          u64 S[8];
#pragma unroll
          for (int p = 0; p < NPL; ++p) {
            const float4 v = q[p * B + e];
            S[2 * p] = pk2(v.x, v.y);
            S[2 * p + 1] = pk2(v.z, v.w);
          }
#pragma unroll
          for (int t = 0; t < NT; ++t) pair2_sym<KIND>(T[t], QI1[t], QI1N[t], QI2[t], S, ai[t], aj, three, mhalf);
#pragma unroll
          for (int o = 0; o < NO; ++o) aj[o] = shfl_u64(aj[o], up2);
        }
        const int dn = (lane + 31) & 31;
#pragma unroll
        for (int o = 0; o < NO; ++o) {
          float lo, hi;
#pragma unroll
          for (int t = 0; t < NT; ++t) {
            upk2(ai[t][o], lo, hi);
            acci[t][o] += lo + hi;
          }
          upk2(aj[o], lo, hi);
          accj[o] = lo + __shfl_sync(0xffffffffu, hi, dn);  // source t: low slot here, high slot of lane t - 1
        }
      } else if (!PACKED && !any) {
#pragma unroll 8
        for (int k = 0; k < 32; ++k) {
          const float4 a = pa[lane + k], b = pb[lane + k];  // (scalar form: DUP = 2)
#pragma unroll
          for (int t = 0; t < NT; ++t) f32_pair_sym<KIND, false>(ta[t], tb[t], a, b, false, false, acci[t], accj);
#pragma unroll
          for (int o = 0; o < NO; ++o) accj[o] = __shfl_sync(0xffffffffu, accj[o], up);
        }
      } else {
        for (int k = 0; k < 32; ++k) {
          const int s = 32 * r + ((lane + k) & 31);
          const int e = PACKED ? ((lane + k) & 31) : lane + k;
          const float4 a = pa[e], b = pb[e];
          const int lp = sLp[s];
          const unsigned long long ms = sMask[s];
#pragma unroll
          for (int t = 0; t < NT; ++t) {
            const bool msk_i = (mi[t] >> lp) & 1ull;
            const bool msk_j = (ms >> lpi[t]) & 1ull;
            f32_pair_sym<KIND, true>(ta[t], tb[t], a, b, msk_i, msk_j, acci[t], accj);
          }
#pragma unroll
          for (int o = 0; o < NO; ++o) accj[o] = __shfl_sync(0xffffffffu, accj[o], up);
        }
      }
#pragma unroll
      for (int o = 0; o < NO; ++o) sRed[warp][32 * r + lane][o] = accj[o];
    }
  }
#pragma unroll
  for (int t = 0; t < NT; ++t) {
    const int64_t i = I * B + tid + t * NTH;
    if (!pad[t])
#pragma unroll
      for (int o = 0; o < NO; ++o) red_add_f64(out + o * N + i, (double)acci[t][o]);
  }
  if (diag) return;
  __syncthreads();
#pragma unroll
  for (int u = 0; u < NT; ++u) {
    const int ls = tid + u * NTH;
    const int64_t j = J * B + ls;
    if (j >= N) continue;
#pragma unroll
    for (int o = 0; o < NO; ++o) {
      double v = 0.0;
#pragma unroll
      for (int w = 0; w < NW; ++w) v += (double)sRed[w][ls][o];
      red_add_f64(out + o * N + j, v);
    }
  }
}

// flag (target block, source tile) pairs that contain a near pair
__global__ void k_mask_flags(int64_t N, int np, int tb, int ts, int64_t ntiles, const int64_t* __restrict__ row_ptr,
                             const int32_t* __restrict__ near_patch, uint8_t* __restrict__ flags) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= N) return;
  const int64_t blk = i / tb;
  for (int64_t b = row_ptr[i]; b < row_ptr[i + 1]; ++b) {
    const int64_t P = near_patch[b];
    const int64_t f = (P * np) / ts, l = ((P + 1) * np - 1) / ts;
    for (int64_t t = f; t <= l; ++t) flags[blk * ntiles + t] = 1;
  }
}

int lb_get_mask_src(lb_ctx* c, int tb, int ts, int snp, int64_t nsrc_pad, MaskTable** out) {
  const int64_t ntiles = nsrc_pad / ts;
  for (auto& m : c->masks)
    if (m.tb == tb && m.ts == ts && m.snp == snp && m.ntiles == ntiles) {
      *out = &m;
      return LB_OK;
    }
  MaskTable m;
  m.tb = tb;
  m.ts = ts;
  m.snp = snp;
  m.ntb = (c->N + tb - 1) / tb;
  m.ntiles = ntiles;
  LB_CHECK(lb_alloc(c, &m.flags, (size_t)(m.ntb * m.ntiles)));
  LB_CUDA(c, cudaMemsetAsync(m.flags, 0, (size_t)(m.ntb * m.ntiles), c->stream));
  k_mask_flags<<<lb_div_up(c->N, 256), 256, 0, c->stream>>>(c->N, snp, tb, ts, m.ntiles, c->row_ptr,
                                                              c->near_patch, m.flags);
  LB_LAUNCH(c);
  c->masks.push_back(m);
  *out = &c->masks.back();
  return LB_OK;
}

int lb_get_mask(lb_ctx* c, int tb, int ts, MaskTable** out) { return lb_get_mask_src(c, tb, ts, c->np, c->Npad, out); }

// Sources of a pass: the nodes themselves, or the oversampled far rule's
// points (Ns of them, nps per patch) when one is set.
static inline int64_t src_pad(const lb_ctx* c) { return c->far_order ? c->Nspad : c->Npad; }
static inline int src_np(const lb_ctx* c) { return c->far_order ? c->nps : c->np; }
static inline int64_t src_count(const lb_ctx* c) { return c->far_order ? c->Ns : c->N; }

template <typename R, int KIND, int NT, int NTH, int TS>
static int launch_far_t(lb_ctx* c, const void* srcA, const void* srcB, double* part, int* nsplit_out) {
  typedef typename V4T<R>::type V4;
  const int tb = NT * NTH;
  const int snp = src_np(c);
  if (snp * 62 < TS) return lb_fail(c, LB_EINVAL, "patch too small for the source tile");
  MaskTable* m = nullptr;
  LB_CHECK(lb_get_mask_src(c, tb, TS, snp, src_pad(c), &m));
  const int64_t ntb = m->ntb, ntiles = m->ntiles;
  // split the source range so that the grid fills whole waves
  int nsplit = 1;
  LB_CHECK(lb_pick_nsplit(c, k_far<R, KIND, NT, NTH, TS>, NTH, ntb, ntiles, &nsplit));
  const int tps = (int)((ntiles + nsplit - 1) / nsplit);
  const V4* tp = sizeof(R) == 4 ? (const V4*)c->pos32 : (const V4*)c->pos64;
  const V4* tn = sizeof(R) == 4 ? (const V4*)c->nrm32 : (const V4*)c->nrm64;
  dim3 grid((unsigned)ntb, (unsigned)nsplit);
  const int64_t pairs = c->N * src_count(c);
  ProfScope prof(c, (sizeof(R) == 4 ? LB_PROF_FAR32_K1 : LB_PROF_FAR64_K1) + KIND, pairs);
  k_far<R, KIND, NT, NTH, TS><<<grid, NTH, 0, c->stream>>>(c->N, snp, tp, tn, (const V4*)srcA, (const V4*)srcB,
                                                          m->flags, ntiles, c->row_ptr, c->near_patch, tps, part);
  LB_LAUNCH(c);
  lb_pair_counter += pairs;
  *nsplit_out = (int)nsplit;
  return LB_OK;
}

template <int KIND, int NT, int NTH, int TS, int MINB = 1>
static int launch_far32x2(lb_ctx* c, const void* srcA, const void* srcB, double* part, int* nsplit_out) {
  const int tb = NT * NTH;
  if (c->np * 62 < TS) return lb_fail(c, LB_EINVAL, "patch too small for the source tile");
  MaskTable* m = nullptr;
  LB_CHECK(lb_get_mask(c, tb, TS, &m));
  const int64_t ntb = m->ntb, ntiles = m->ntiles;
  int nsplit = 1;
  LB_CHECK(lb_pick_nsplit(c, k_far32x2<KIND, NT, NTH, TS, MINB>, NTH, ntb, ntiles, &nsplit));
  const int tps = (int)((ntiles + nsplit - 1) / nsplit);
  dim3 grid((unsigned)ntb, (unsigned)nsplit);
  ProfScope prof(c, LB_PROF_FAR32_K1 + KIND, c->N * c->N);
  k_far32x2<KIND, NT, NTH, TS, MINB><<<grid, NTH, 0, c->stream>>>(c->N, c->np, c->pos32, c->nrm32, (const float4*)srcA,
                                                            (const float4*)srcB, m->flags, ntiles, c->row_ptr,
                                                            c->near_patch, tps, part);
  LB_LAUNCH(c);
  lb_pair_counter += c->N * c->N;
  *nsplit_out = (int)nsplit;
  return LB_OK;
}

// Single-density float32 passes: three launch variants per kind, chosen by
// timing.  K1: the scalar kernel with 4 targets per thread (variant 0), the
// packed two-source kernel capped for three resident blocks per SM (1), the
// scalar kernel with 8 targets per thread
// (2); the longer kinds: the packed kernel with 4 targets per thread at its
// natural register count (0), capped for three resident blocks per SM (1),
// with 2 targets per thread (2).
// the symmetric kernels (one float64 sum per accumulator: *ns = -1)
template <int KIND, bool PACKED, int NT, int MINB = 0>
static int launch_far32_sym(lb_ctx* c, const void* A, const void* B, double* part, int* ns) {
  constexpr int NTH = 128;  // nodes per block; the CTA has NTH / NT threads
  if (c->np * 62 < NTH) return lb_fail(c, LB_EINVAL, "patch too small for the source tile");
  if (c->Npad % NTH) return lb_fail(c, LB_EINVAL, "node padding is not a multiple of the block");
  MaskTable* m = nullptr;
  LB_CHECK(lb_get_mask(c, NTH, NTH, &m));
  const int64_t nb = m->ntb;
  const int64_t nblk = nb * (nb + 1) / 2;
  if (nblk > 0x7fffffffLL) return lb_fail(c, LB_EINVAL, "too many node blocks for one launch");
  LB_CUDA(c, cudaMemsetAsync(part, 0, 4 * c->N * sizeof(double), c->stream));
  ProfScope prof(c, LB_PROF_FAR32_K1 + KIND, c->N * c->N);
  k_far32_sym<KIND, PACKED, NT, MINB><<<(unsigned)nblk, NTH / NT, 0, c->stream>>>(c->N, c->np, (const float4*)A, (const float4*)B,
                                                               m->flags, m->ntiles, c->row_ptr, c->near_patch, part);
  LB_LAUNCH(c);
  lb_pair_counter += c->N * c->N;
  *ns = -1;
  return LB_OK;
}

// launch variants of the single-density float32 passes (chosen by timing):
// 0-2 the tiled kernels below; K1 and K2 also 3, the symmetric kernel, 4,
// the same with the packed two-source loop, and 5 and 6, those two with two
// targets per lane
#define LB_FP32_VARIANTS 3
static int fp32_nvariants(int kind) { return (kind == FAR_K1 || kind == FAR_K2) ? 7 : LB_FP32_VARIANTS; }
static int launch_fp32(lb_ctx* c, int kind, int variant, const void* A, const void* B, double* part, int* ns) {
  if (kind == FAR_K1 || kind == FAR_K2) {
    const bool k1 = kind == FAR_K1;
    switch (variant) {
      case 3: return k1 ? launch_far32_sym<FAR_K1, false, 1>(c, A, B, part, ns)
                        : launch_far32_sym<FAR_K2, false, 1>(c, A, B, part, ns);
      case 4: return k1 ? launch_far32_sym<FAR_K1, true, 1>(c, A, B, part, ns)
                        : launch_far32_sym<FAR_K2, true, 1>(c, A, B, part, ns);
      case 5: return k1 ? launch_far32_sym<FAR_K1, false, 2>(c, A, B, part, ns)
                        : launch_far32_sym<FAR_K2, false, 2>(c, A, B, part, ns);
      case 6: return k1 ? launch_far32_sym<FAR_K1, true, 2>(c, A, B, part, ns)
                        : launch_far32_sym<FAR_K2, true, 2>(c, A, B, part, ns);
      default: break;
    }
  }
  switch (kind) {
    case FAR_K1:
      if (variant == 1) return launch_far32x2<FAR_K1, 4, 128, 128, 3>(c, A, B, part, ns);
      if (variant == 2) return launch_far_t<float, FAR_K1, 8, 128, 128>(c, A, B, part, ns);
      return launch_far_t<float, FAR_K1, 4, 128, 128>(c, A, B, part, ns);
    case FAR_KALL:
      if (variant == 1) return launch_far32x2<FAR_KALL, 4, 128, 128, 3>(c, A, B, part, ns);
      if (variant == 2) return launch_far32x2<FAR_KALL, 2, 128, 128>(c, A, B, part, ns);
      return launch_far32x2<FAR_KALL, 4, 128, 128>(c, A, B, part, ns);
    case FAR_K2:
      if (variant == 1) return launch_far32x2<FAR_K2, 4, 128, 128, 3>(c, A, B, part, ns);
      if (variant == 2) return launch_far32x2<FAR_K2, 2, 128, 128>(c, A, B, part, ns);
      return launch_far32x2<FAR_K2, 4, 128, 128>(c, A, B, part, ns);
    default:
      if (variant == 1) return launch_far32x2<FAR_K4, 4, 128, 128, 3>(c, A, B, part, ns);
      if (variant == 2) return launch_far32x2<FAR_K4, 2, 128, 128>(c, A, B, part, ns);
      return launch_far32x2<FAR_K4, 4, 128, 128>(c, A, B, part, ns);
  }
}

namespace {
struct SingleKey {
  int device;
  int64_t N;
  int np, kind;
  bool operator<(const SingleKey& o) const {
    return std::tie(device, N, np, kind) < std::tie(o.device, o.N, o.np, o.kind);
  }
};
std::mutex g_single_mu;
std::map<SingleKey, int> g_single;
}  // namespace

// The variant for this pass: tuned earlier in the process, or timed now on
// the caller's data (each variant launched twice, the second timed; nothing
// is counted or profiled), or variant 0 inside a stream capture.
int lb_tune_choice(lb_ctx* c, int key_kind, int nvar, int (*launch)(lb_ctx*, int, void*), void* arg, int* choice) {
  const SingleKey key{c->device, c->N, c->np, key_kind};
  {
    std::lock_guard<std::mutex> lk(g_single_mu);
    auto it = g_single.find(key);
    if (it != g_single.end()) { *choice = it->second; return LB_OK; }
  }
  *choice = 0;
  if (c->capturing) return LB_OK;
  const int prof = c->prof_on;
  const int64_t pairs = lb_pair_counter, launches = c->launches;
  c->prof_on = 0;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  int rc = LB_OK;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
    rc = lb_fail(c, LB_ECUDA, "cudaEventCreate failed");
  float best_ms = 1e30f;
  int best = 0;
  for (int v = 0; v < nvar && rc == LB_OK; ++v) {
    rc = launch(c, v, arg);  // warm-up (module load, occupancy query)
    if (rc == LB_OK && cudaEventRecord(e0, c->stream) != cudaSuccess) rc = lb_fail(c, LB_ECUDA, "event record");
    if (rc == LB_OK) rc = launch(c, v, arg);
    if (rc == LB_OK && cudaEventRecord(e1, c->stream) != cudaSuccess) rc = lb_fail(c, LB_ECUDA, "event record");
    float ms = 0.f;
    if (rc == LB_OK && (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess))
      rc = lb_fail(c, LB_ECUDA, "timing a far-field launch variant failed");
    if (rc == LB_OK && ms < best_ms) { best_ms = ms; best = v; }
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  c->prof_on = prof;
  lb_pair_counter = pairs;
  c->launches = launches;
  if (rc != LB_OK) return rc;
  {
    std::lock_guard<std::mutex> lk(g_single_mu);
    g_single[key] = best;
  }
  *choice = best;
  return LB_OK;
}

int lb_tuned_choice(lb_ctx* c, int key_kind) {
  std::lock_guard<std::mutex> lk(g_single_mu);
  auto it = g_single.find(SingleKey{c->device, c->N, c->np, key_kind});
  return it == g_single.end() ? -1 : it->second;
}

struct Fp32Launch {
  int kind;
  const void *A, *B;
  double* part;
};
static int fp32_launch_cb(lb_ctx* c, int v, void* arg) {
  const Fp32Launch* a = (const Fp32Launch*)arg;
  int ns = 0;
  return launch_fp32(c, a->kind, v, a->A, a->B, a->part, &ns);
}

static int fp32_variant(lb_ctx* c, int kind, const void* A, const void* B, double* part, int* variant) {
  if (c->far_order) { *variant = 0; return LB_OK; }  // oversampled sources: the scalar float32 kernels
  Fp32Launch a{kind, A, B, part};
  return lb_tune_choice(c, kind, fp32_nvariants(kind), fp32_launch_cb, &a, variant);
}

int lb_far_tuned_variant(lb_ctx* c, int kind) { return lb_tuned_choice(c, kind); }

extern "C" int lb_debug_set_variant(lb_ctx* c, int kind, int variant) {
  if (!c) return lb_fail(nullptr, LB_EINVAL, "null context");
  if (!c->have_geom) return lb_fail(c, LB_ESTATE, "no geometry uploaded");
  // kinds 0..3: float32 passes; 4, 5: the symmetric double-float K1, K2
  const int nvar = kind >= 0 && kind <= 3 ? fp32_nvariants(kind) : (kind == 4 || kind == 5 ? 2 : 0);
  if (variant < 0 || variant >= nvar)
    return lb_fail(c, LB_EINVAL, "no launch variant %d for pass kind %d", variant, kind);
  const int key = kind <= 3 ? kind : LB_TUNE_DFSYM + (kind == 4 ? FAR_K1 : FAR_K2);
  std::lock_guard<std::mutex> lk(g_single_mu);
  g_single[SingleKey{c->device, c->N, c->np, key}] = variant;
  return LB_OK;
}

int lb_far_launch(lb_ctx* c, int kind, int prec, const void* srcA, const void* srcB, double* part, int* nsplit) {
  if (prec == LB_DF64) return lb_far_launch_df(c, kind, srcA, part, nsplit);
  if (c->far_order && prec != LB_FP64) {  // oversampled sources: the scalar float32 kernels
    switch (kind) {
      case FAR_K1: return launch_far_t<float, FAR_K1, 4, 128, 128>(c, srcA, srcB, part, nsplit);
      case FAR_KALL: return launch_far_t<float, FAR_KALL, 4, 128, 128>(c, srcA, srcB, part, nsplit);
      case FAR_K2: return launch_far_t<float, FAR_K2, 4, 128, 128>(c, srcA, srcB, part, nsplit);
      default: return launch_far_t<float, FAR_K4, 4, 128, 128>(c, srcA, srcB, part, nsplit);
    }
  }
  if (prec == LB_FP64) {
    switch (kind) {
      case FAR_K1: return launch_far_t<double, FAR_K1, 2, 128, 64>(c, srcA, srcB, part, nsplit);
      case FAR_KALL: return launch_far_t<double, FAR_KALL, 2, 128, 64>(c, srcA, srcB, part, nsplit);
      case FAR_K2: return launch_far_t<double, FAR_K2, 2, 128, 64>(c, srcA, srcB, part, nsplit);
      default: return launch_far_t<double, FAR_K4, 2, 128, 64>(c, srcA, srcB, part, nsplit);
    }
  }
  int variant = 0;
  LB_CHECK(fp32_variant(c, kind, srcA, srcB, part, &variant));
  return launch_fp32(c, kind, variant, srcA, srcB, part, nsplit);
}

// ---------------------------------------------------------------------------
// sources for a pass: A = (x, y, z, w * d1), B = (n, w * d2)
template <typename R>
__global__ void k_pack(int64_t N, int64_t Npad, const typename V4T<R>::type* __restrict__ pos,
                       const typename V4T<R>::type* __restrict__ nrm, const double* __restrict__ w,
                       const double* __restrict__ d1, const double* __restrict__ d2,
                       typename V4T<R>::type* __restrict__ A, typename V4T<R>::type* __restrict__ B) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= Npad) return;
  typename V4T<R>::type p = pos[i], n = nrm[i];
  if (i < N) {
    p.w = (R)(w[i] * d1[i]);
    n.w = d2 ? (R)(w[i] * d2[i]) : R(0);
  } else {
    p.w = R(0);
    n.w = R(0);
  }
  A[i] = p;
  B[i] = n;
}

static int pack_sources(lb_ctx* c, int prec, const double* d1, const double* d2, void** A, void** B) {
  if (c->far_order) return lb_far_rule_pack(c, prec, d1, d2, A, B);
  if (prec == LB_DF64) {  // four float4 planes
    LB_CHECK(lb_ensure(c, c->ws_src, 4 * c->Npad * sizeof(float4)));
    *A = c->ws_src.p;
    *B = nullptr;
    return lb_pack_df(c, d1, d2, *A);
  }
  const size_t v4 = prec == LB_FP64 ? sizeof(double4_32a) : sizeof(float4);
  LB_CHECK(lb_ensure(c, c->ws_src, 2 * c->Npad * v4));
  *A = c->ws_src.p;
  *B = (char*)c->ws_src.p + c->Npad * v4;
  if (prec == LB_FP64)
    k_pack<double><<<lb_div_up(c->Npad, 256), 256, 0, c->stream>>>(c->N, c->Npad, c->pos64, c->nrm64, c->w, d1, d2,
                                                                    (double4_32a*)*A, (double4_32a*)*B);
  else
    k_pack<float><<<lb_div_up(c->Npad, 256), 256, 0, c->stream>>>(c->N, c->Npad, c->pos32, c->nrm32, c->w, d1, d2,
                                                                   (float4*)*A, (float4*)*B);
  LB_LAUNCH(c);
  return LB_OK;
}

// ---------------------------------------------------------------------------
// epilogue: reduce split partials, add correction SpMV, one warp per row.
struct EpiSpec {
  int nout;
  int acc[4];            // accumulator index, or -1 for -(n_x . (a1, a2, a3)) (K1's S')
  double scale[4];       // multiplies the far accumulator
  int kern[4];           // correction kernel (LB_K_*), or -1 for none
  const double* dens[4]; // density of the correction sum (float64)
  int64_t kplane;        // float4 vectors per kernel plane of the float weight copies (nnzb * npv)
  const float* dh[4];    // its float32 copy / double-float hi part
  const float* dl[4];    // its double-float lo part
  double* out[4];        // [N]
};

__device__ __forceinline__ double to_d(double v) { return v; }
__device__ __forceinline__ double to_d(float v) { return (double)v; }
__device__ __forceinline__ double to_d(F2 v) { return df_to_double(v); }

// Split-partial reduction and near-field correction SpMV of one pass, one
// warp per row.  The correction sums use the pass's own arithmetic: MODE 0
// float64 (weights vals), MODE 1 float32 (weights vh, densities dh), MODE 2
// double-float (weights vh + vl, densities dh + dl); float64 throughput on
// GB300 is a small fraction of float32, and the float32 / double-float sums
// match the accuracy of the pair sums they complete.
// The float copies are padded to npv float4 vectors per (block, kernel) and
// per patch (lb_lowp_vals, lowp_dens: zeros past np), so that every lane
// moves four nodes' weights and densities with single 16-byte loads; the
// weights are kernel-major (plane k at k * sp.kplane vectors), so that a
// row's blocks of one kernel are contiguous; four vectors per lane in flight.
// A row's loads form a chain (row offsets, near patches, weights, far sums),
// so the kernel is bound by latency: the float32 form is held to 40
// registers (six 256-thread CTAs, 48 warps per SM) to keep more rows in
// flight; the float64 and double-float forms would spill at that bound.
template <int MODE>
__global__ void __launch_bounds__(256, MODE == 1 ? 6 : 0) k_epilogue(int64_t N, int np, int npv, int nsplit, int nacc, const double* __restrict__ part,
                           const double* __restrict__ nrm, const int64_t* __restrict__ row_ptr,
                           const int32_t* __restrict__ near_patch, const double* __restrict__ vals,
                           const float4* __restrict__ vh, const float4* __restrict__ vl, EpiSpec sp) {
  using T = typename std::conditional<MODE == 0, double, typename std::conditional<MODE == 1, float, F2>::type>::type;
  const int lane = threadIdx.x & 31;
  const int64_t i = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  if (i >= N) return;
  T cs[4];
#pragma unroll
  for (int o = 0; o < 4; ++o) cs[o] = T{};
  const bool corr = MODE == 0 ? vals != nullptr : vh != nullptr;
  if constexpr (MODE != 0) {
   if (corr) {
    const int64_t rb = row_ptr[i];
    const int tot = (int)(row_ptr[i + 1] - rb) * npv;
    for (int e0 = lane; e0 < tot; e0 += 128) {
      int64_t bq[4], pq[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int e = e0 + 32 * u;
        const int bl = e < tot ? e / npv : 0;
        const int qv = e < tot ? e - bl * npv : 0;
        bq[u] = (rb + bl) * (int64_t)npv + qv;                        // weights, kernel plane 0
        pq[u] = e < tot ? (int64_t)near_patch[rb + bl] * npv + qv : -1;  // densities
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        if (pq[u] < 0) continue;
#pragma unroll
        for (int o = 0; o < 4; ++o) {
          if (o >= sp.nout || sp.kern[o] < 0) continue;
          const int64_t wi = bq[u] + sp.kern[o] * sp.kplane;
          const float4 w = __ldg(vh + wi);
          const float4 x = __ldg(reinterpret_cast<const float4*>(sp.dh[o]) + pq[u]);
          if constexpr (MODE == 1) {
            float t = cs[o];
            t = fmaf(w.x, x.x, t);
            t = fmaf(w.y, x.y, t);
            t = fmaf(w.z, x.z, t);
            t = fmaf(w.w, x.w, t);
            cs[o] = t;
          } else {
            const float4 wl = __ldg(vl + wi);
            const float4 xl = __ldg(reinterpret_cast<const float4*>(sp.dl[o]) + pq[u]);
            df_acc(cs[o], df_mul({w.x, wl.x}, {x.x, xl.x}));
            df_acc(cs[o], df_mul({w.y, wl.y}, {x.y, xl.y}));
            df_acc(cs[o], df_mul({w.z, wl.z}, {x.z, xl.z}));
            df_acc(cs[o], df_mul({w.w, wl.w}, {x.w, xl.w}));
          }
        }
      }
    }
    warp_reduce_scatter<4>(cs, lane);  // lane 8 o holds output o
  }
  } else {
   if (corr) {
    // the row's (block, node) pairs flattened; each lane walks them 32 apart,
    // four at a time so that their loads overlap, tracking (block, node)
    // incrementally instead of dividing
    const int64_t rb = row_ptr[i];
    const int ne = (int)((row_ptr[i + 1] - rb) * np);
    const int stride = LB_NKERNELS * np;
    int bo = lane / np, q = lane - (lane / np) * np;
    for (int e = lane; e < ne; e += 128) {
      int bl[4], ql[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        bl[u] = bo;
        ql[u] = q;
        q += 32;
        while (q >= np) { q -= np; ++bo; }
      }
      int64_t col[4], vo[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const bool ok = e + 32 * u < ne;
        const int64_t b = rb + (ok ? bl[u] : 0);
        col[u] = ok ? (int64_t)near_patch[b] * np + ql[u] : -1;
        vo[u] = b * stride + ql[u];
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        if (col[u] < 0) continue;
#pragma unroll
        for (int o = 0; o < 4; ++o) {
          if (o >= sp.nout || sp.kern[o] < 0) continue;
          const int64_t w = vo[u] + sp.kern[o] * np;
          if constexpr (MODE == 0) cs[o] = fma(__ldg(vals + w), sp.dens[o][col[u]], cs[o]);
        }
      }
    }
    warp_reduce_scatter<4>(cs, lane);  // lane 8 o holds output o
  }
  }
  // split partials of output o summed by lanes 8 o .. 8 o + 7, eight splits
  // apart (float64 for float64 passes, else (hi, lo) float pairs summed in
  // double-float arithmetic), then combined by three shuffles; nsplit < 0:
  // a single float64 sum per accumulator (the symmetric double-float kernels)
  const int o = lane >> 3, sub = lane & 7;
  const int oo = o < sp.nout ? o : 0;
  const int a0 = sp.acc[oo];
  using P = typename std::conditional<MODE == 0, double, F2>::type;
  P g[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) g[k] = P{};
  const int na = a0 >= 0 ? 1 : 3;
  const int ab = a0 >= 0 ? a0 : 1;
  if (nsplit < 0) {  // one float64 sum per accumulator, [nacc][N]
    if (sub == 0)
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        if (k >= na) break;
        const double v = part[(int64_t)(ab + k) * N + i];
        if constexpr (MODE == 0) {
          g[k] = v;
        } else {
          const float h = (float)v;
          g[k] = {h, (float)(v - (double)h)};
        }
      }
  } else {
    for (int s = sub; s < nsplit; s += 8)
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        if (k >= na) break;
        const int64_t idx = ((int64_t)s * nacc + ab + k) * N + i;
        if constexpr (MODE == 0) {
          g[k] += part[idx];
        } else {
          const float2 v = reinterpret_cast<const float2*>(part)[idx];
          g[k] = df_add(g[k], {v.x, v.y});
        }
      }
  }
#pragma unroll
  for (int off = 4; off > 0; off >>= 1)
#pragma unroll
    for (int k = 0; k < 3; ++k) g[k] = add_v(g[k], shfl_xor_v(g[k], off));
  if (sub != 0 || o >= sp.nout) return;
  double f;
  if (a0 >= 0) f = to_d(g[0]);
  else f = -(nrm[3 * i] * to_d(g[0]) + nrm[3 * i + 1] * to_d(g[1]) + nrm[3 * i + 2] * to_d(g[2]));
  sp.out[o][i] = f * sp.scale[o] + (corr ? to_d(cs[0]) : 0.0);
}

// hi = (float)x, lo = (float)(x - hi)
__global__ void k_split_f64(int64_t n, const double* __restrict__ x, float* __restrict__ hi, float* __restrict__ lo) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const double v = x[i];
    const float h = (float)v;
    hi[i] = h;
    if (lo) lo[i] = (float)(v - (double)h);
  }
}

int lb_split_f64(lb_ctx* c, int64_t n, const double* x, float* hi, float* lo) {
  const unsigned nb = (unsigned)std::min<int64_t>(8LL * c->sm_count, std::max<int64_t>(1, lb_div_up(n, 256)));
  k_split_f64<<<nb, 256, 0, c->stream>>>(n, x, hi, lo);
  LB_LAUNCH(c);
  return LB_OK;
}

// hi = (float)x, lo = (float)(x - hi) of rows of np values into rows of npp
// (the tail of each row zero): n_rows rows
__global__ void k_split_pad(int64_t nrows, int np, int npp, const double* __restrict__ x, float* __restrict__ hi,
                            float* __restrict__ lo) {
  const int64_t n = nrows * npp;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = t / npp;
    const int q = (int)(t - r * npp);
    const double v = q < np ? x[r * np + q] : 0.0;
    const float h = (float)v;
    hi[t] = h;
    if (lo) lo[t] = (float)(v - (double)h);
  }
}

static int split_pad(lb_ctx* c, int64_t nrows, const double* x, float* hi, float* lo) {
  const int npp = lb_np_pad(c->np);
  const unsigned nb = (unsigned)std::min<int64_t>(8LL * c->sm_count, std::max<int64_t>(1, lb_div_up(nrows * npp, 256)));
  k_split_pad<<<nb, 256, 0, c->stream>>>(nrows, c->np, npp, x, hi, lo);
  LB_LAUNCH(c);
  return LB_OK;
}

// hi / lo float copies of vals [nnzb][4][np] in kernel-major planes
// [4][nnzb][npp] (rows padded with zeros to npp)
__global__ void k_split_kmajor(int64_t nnzb, int np, int npp, const double* __restrict__ vals,
                               float* __restrict__ hi, float* __restrict__ lo) {
  const int64_t plane = nnzb * npp, n = LB_NKERNELS * plane;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t k = t / plane, rem = t - k * plane;
    const int64_t b = rem / npp;
    const int q = (int)(rem - b * npp);
    const double v = q < np ? vals[(b * LB_NKERNELS + k) * np + q] : 0.0;
    const float h = (float)v;
    hi[t] = h;
    lo[t] = (float)(v - (double)h);
  }
}

// float32 hi / lo copies of the correction weights, kernel-major
// [4][nnzb][npp] with the node index padded to a multiple of four, made on
// first use after the corrections were loaded or built: a pass reads each
// of its kernels' weights as one contiguous stream
int lb_lowp_vals(lb_ctx* c) {
  if (!c->have_corr || c->vals_hi) return LB_OK;
  const int npp = lb_np_pad(c->np);
  const int64_t n = c->nnzb * LB_NKERNELS * npp;
  LB_CHECK(lb_alloc(c, &c->vals_hi, (size_t)n));
  LB_CHECK(lb_alloc(c, &c->vals_lo, (size_t)n));
  const unsigned nb = (unsigned)std::min<int64_t>(8LL * c->sm_count, std::max<int64_t>(1, lb_div_up(n, 256)));
  k_split_kmajor<<<nb, 256, 0, c->stream>>>(c->nnzb, c->np, npp, c->vals, c->vals_hi, c->vals_lo);
  LB_LAUNCH(c);
  return LB_OK;
}

// float32 / double-float copies of the distinct correction densities of sp,
// [npatch][npp] each
static int lowp_dens(lb_ctx* c, int mode, EpiSpec& sp) {
  const int64_t M = c->npatch * lb_np_pad(c->np);
  LB_CHECK(lb_ensure(c, c->ws_dlow, (size_t)(8 * M) * sizeof(float)));
  float* base = (float*)c->ws_dlow.p;
  const double* uniq[4];
  int nu = 0;
  for (int o = 0; o < sp.nout; ++o) {
    if (sp.kern[o] < 0) continue;
    int j = 0;
    while (j < nu && uniq[j] != sp.dens[o]) ++j;
    if (j == nu) {
      uniq[nu++] = sp.dens[o];
      LB_CHECK(split_pad(c, c->npatch, sp.dens[o], base + 2 * j * M, mode == 2 ? base + (2 * j + 1) * M : nullptr));
    }
    sp.dh[o] = base + 2 * j * M;
    sp.dl[o] = base + (2 * j + 1) * M;
  }
  return LB_OK;
}

static int run_epilogue(lb_ctx* c, int prec, int nsplit, int nacc, const double* part, EpiSpec sp) {
  const unsigned grid = lb_div_up(c->N * 32, 256);
  // the pair precision fixes the partials' format and the correction arithmetic
  const int mode = prec == LB_FP64 ? 0 : (prec == LB_FP32 ? 1 : 2);
  const bool corr = c->have_corr;
  if (mode && corr) {
    LB_CHECK(lb_lowp_vals(c));
    LB_CHECK(lowp_dens(c, mode, sp));
  }
  ProfScope prof(c, LB_PROF_EPILOGUE);
  const int npv = lb_np_pad(c->np) / 4;
  const float4* vh = corr ? (const float4*)c->vals_hi : nullptr;
  const float4* vl = corr ? (const float4*)c->vals_lo : nullptr;
  sp.kplane = c->nnzb * (int64_t)npv;
  if (mode == 0)
    k_epilogue<0><<<grid, 256, 0, c->stream>>>(c->N, c->np, npv, nsplit, nacc, part, c->nrm, c->row_ptr,
                                               c->near_patch, corr ? c->vals : nullptr, nullptr, nullptr, sp);
  else if (mode == 1)
    k_epilogue<1><<<grid, 256, 0, c->stream>>>(c->N, c->np, npv, nsplit, nacc, part, c->nrm, c->row_ptr,
                                               c->near_patch, nullptr, vh, nullptr, sp);
  else
    k_epilogue<2><<<grid, 256, 0, c->stream>>>(c->N, c->np, npv, nsplit, nacc, part, c->nrm, c->row_ptr,
                                               c->near_patch, nullptr, vh, vl, sp);
  LB_LAUNCH(c);
  return LB_OK;
}

static int part_buffer(lb_ctx* c, double** part) {
  // up to 4 accumulators x up to ntiles splits
  const int64_t max_split = src_pad(c) / 64;
  const int64_t want = std::min<int64_t>(max_split, 32);
  LB_CHECK(lb_ensure(c, c->ws_part, (size_t)(want * 4 * c->N) * sizeof(double)));
  *part = (double*)c->ws_part.p;
  return LB_OK;
}

// ---------------------------------------------------------------------------
// deterministic weighted sums: partial per block, then a fixed-order total
#define RED_BLOCKS 256
__global__ void k_wdot_partial(int64_t N, const double* __restrict__ w, const double* __restrict__ v,
                               double* __restrict__ partial) {
  __shared__ double sh[256];
  double s = 0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x)
    s += (w ? w[i] : 1.0) * v[i];
  sh[threadIdx.x] = s;
  __syncthreads();
  for (int k = blockDim.x / 2; k > 0; k >>= 1) {
    if (threadIdx.x < k) sh[threadIdx.x] += sh[threadIdx.x + k];
    __syncthreads();
  }
  if (threadIdx.x == 0) partial[blockIdx.x] = sh[0];
}

__device__ __forceinline__ double sum_partials(const double* p, int n) {
  double s = 0;
  for (int k = 0; k < n; ++k) s += p[k];
  return s;
}

__global__ void k_sum_partials(const double* __restrict__ partial, int n, double* __restrict__ out) {
  if (threadIdx.x == 0 && blockIdx.x == 0) out[0] = sum_partials(partial, n);
}

int lb_wmean(lb_ctx* c, const double* f, double* mean_host) {
  LB_CHECK(lb_ensure(c, c->ws_red, (RED_BLOCKS + 8) * sizeof(double)));
  double* partial = (double*)c->ws_red.p;
  k_wdot_partial<<<RED_BLOCKS, 256, 0, c->stream>>>(c->N, c->w, f, partial);
  LB_LAUNCH(c);
  k_sum_partials<<<1, 32, 0, c->stream>>>(partial, RED_BLOCKS, partial + RED_BLOCKS);
  LB_LAUNCH(c);
  LB_CUDA(c, cudaMemcpyAsync(c->host_pinned, partial + RED_BLOCKS, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  LB_CUDA(c, cudaStreamSynchronize(c->stream));
  *mean_host = c->host_pinned[0] / c->area;
  return LB_OK;
}

// A3 final: out = -tau/4 + p0 - p3 - 2 H p2 + W p1  (p = S'mu1, S mu2, S'mu2, (S''+D')mu2)
__global__ void k_a3_final(int64_t N, const double* __restrict__ tau, const double* __restrict__ pot,
                           const double* __restrict__ H, const double* __restrict__ partial, int npart, double area,
                           double* __restrict__ out) {
  __shared__ double eta;
  if (threadIdx.x == 0) eta = sum_partials(partial, npart) / area;
  __syncthreads();
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = -0.25 * tau[i] + pot[i] - pot[3 * N + i] - 2.0 * H[i] * pot[2 * N + i] + eta;
}

// A2 middle: mu1 = D tau (in place), mu2 = -(S''+D') tau - 2 H S' tau + W S tau
__global__ void k_a2_mid(int64_t N, const double* __restrict__ pot, const double* __restrict__ H,
                         const double* __restrict__ partial, int npart, double area, double* __restrict__ mu2) {
  __shared__ double eta;
  if (threadIdx.x == 0) eta = sum_partials(partial, npart) / area;
  __syncthreads();
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x)
    mu2[i] = -pot[3 * N + i] - 2.0 * H[i] * pot[2 * N + i] + eta;
}

__global__ void k_a2_final(int64_t N, const double* __restrict__ tau, const double* __restrict__ q0,
                           const double* __restrict__ q1, double* __restrict__ out) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = -0.25 * tau[i] + q0[i] + q1[i];
}

// ---------------------------------------------------------------------------
int lb_potentials(lb_ctx* c, int prec, const double* sigma, double* pot, unsigned which) {
  void *A, *B;
  double* part;
  int nsplit = 0;
  LB_CHECK(part_buffer(c, &part));
  const bool only_s = (which & ~((1u << LB_K_S) | (1u << LB_K_SP))) == 0;
  LB_CHECK(pack_sources(c, prec, sigma, nullptr, &A, &B));
  const int kind = only_s ? FAR_K1 : FAR_KALL;
  LB_CHECK(lb_far_launch(c, kind, prec, A, B, part, &nsplit));
  EpiSpec sp{};
  int o = 0;
  for (int k = 0; k < LB_NKERNELS; ++k) {
    if (!(which & (1u << k))) continue;
    if (kind == FAR_K1) {
      sp.acc[o] = (k == LB_K_S) ? 0 : -1;
      sp.scale[o] = LB_INV4PI;
    } else {
      sp.acc[o] = k;
      sp.scale[o] = (k == LB_K_SP) ? -LB_INV4PI : LB_INV4PI;
    }
    sp.kern[o] = c->have_corr ? k : -1;
    sp.dens[o] = sigma;
    sp.out[o] = pot + (int64_t)k * c->N;
    ++o;
  }
  sp.nout = o;
  return run_epilogue(c, prec, nsplit, 4, part, sp);
}

int lb_apply_op(lb_ctx* c, int formulation, int prec, const double* tau, double* out) {
  if (formulation == LB_A1) return lb_apply_a1(c, prec, tau, out);
  const int64_t N = c->N;
  LB_CHECK(lb_ensure(c, c->ws_pot, (size_t)(8 * N) * sizeof(double)));
  double* pot = (double*)c->ws_pot.p;   // [4][N] pass-1 potentials, then pass-2
  double* mu = pot + 4 * N;             // mu1 [N], mu2 [N]
  double* q = pot + 6 * N;              // pass-2 outputs (A2: 2 of them)
  LB_CHECK(lb_ensure(c, c->ws_red, (RED_BLOCKS + 8) * sizeof(double)));
  double* partial = (double*)c->ws_red.p;
  double* part;
  LB_CHECK(part_buffer(c, &part));
  void *A, *B;
  int nsplit = 0;
  if (prec == LB_FP32) ++lb_apply32_counter; else ++lb_apply64_counter;
  const unsigned nb = 4 * (unsigned)std::min<int64_t>(c->sm_count, lb_div_up(N, 256));
  if (formulation == LB_A3) {
    // pass 1: charge tau -> S tau, S' tau
    LB_CHECK(pack_sources(c, prec, tau, nullptr, &A, &B));
    LB_CHECK(lb_far_launch(c, FAR_K1, prec, A, B, part, &nsplit));
    EpiSpec e1{};
    e1.nout = 2;
    e1.acc[0] = 0; e1.scale[0] = LB_INV4PI; e1.kern[0] = LB_K_S; e1.dens[0] = tau; e1.out[0] = mu + N;   // mu2
    e1.acc[1] = -1; e1.scale[1] = LB_INV4PI; e1.kern[1] = LB_K_SP; e1.dens[1] = tau; e1.out[1] = mu;     // mu1
    LB_CHECK(run_epilogue(c, prec, nsplit, 4, part, e1));
    // pass 2: charges mu1 (A.w), mu2 (B.w)
    LB_CHECK(pack_sources(c, prec, mu, mu + N, &A, &B));
    LB_CHECK(lb_far_launch(c, FAR_K2, prec, A, B, part, &nsplit));
    EpiSpec e2{};
    e2.nout = 4;
    e2.acc[0] = 0; e2.scale[0] = -LB_INV4PI; e2.kern[0] = LB_K_SP; e2.dens[0] = mu; e2.out[0] = pot;
    e2.acc[1] = 1; e2.scale[1] = LB_INV4PI; e2.kern[1] = LB_K_S; e2.dens[1] = mu + N; e2.out[1] = pot + N;
    e2.acc[2] = 2; e2.scale[2] = -LB_INV4PI; e2.kern[2] = LB_K_SP; e2.dens[2] = mu + N; e2.out[2] = pot + 2 * N;
    e2.acc[3] = 3; e2.scale[3] = LB_INV4PI; e2.kern[3] = LB_K_SPPDP; e2.dens[3] = mu + N; e2.out[3] = pot + 3 * N;
    LB_CHECK(run_epilogue(c, prec, nsplit, 4, part, e2));
    k_wdot_partial<<<RED_BLOCKS, 256, 0, c->stream>>>(N, c->w, pot + N, partial);
    LB_LAUNCH(c);
    k_a3_final<<<nb, 256, 0, c->stream>>>(N, tau, pot, c->H, partial, RED_BLOCKS, c->area, out);
    LB_LAUNCH(c);
    return LB_OK;
  }
  // A2, pass 1: all four potentials of tau
  LB_CHECK(pack_sources(c, prec, tau, nullptr, &A, &B));
  LB_CHECK(lb_far_launch(c, FAR_KALL, prec, A, B, part, &nsplit));
  EpiSpec e1{};
  e1.nout = 4;
  for (int k = 0; k < 4; ++k) {
    e1.acc[k] = k;
    e1.scale[k] = (k == LB_K_SP) ? -LB_INV4PI : LB_INV4PI;
    e1.kern[k] = k;
    e1.dens[k] = tau;
    e1.out[k] = pot + (int64_t)k * N;
  }
  LB_CHECK(run_epilogue(c, prec, nsplit, 4, part, e1));
  k_wdot_partial<<<RED_BLOCKS, 256, 0, c->stream>>>(N, c->w, pot, partial);
  LB_LAUNCH(c);
  k_a2_mid<<<nb, 256, 0, c->stream>>>(N, pot, c->H, partial, RED_BLOCKS, c->area, mu + N);
  LB_LAUNCH(c);
  // pass 2: dipole mu1 = D tau (A.w), charge mu2 (B.w)
  LB_CHECK(pack_sources(c, prec, pot + N, mu + N, &A, &B));
  LB_CHECK(lb_far_launch(c, FAR_K4, prec, A, B, part, &nsplit));
  EpiSpec e2{};
  e2.nout = 2;
  e2.acc[0] = 0; e2.scale[0] = LB_INV4PI; e2.kern[0] = LB_K_D; e2.dens[0] = pot + N; e2.out[0] = q;
  e2.acc[1] = 1; e2.scale[1] = LB_INV4PI; e2.kern[1] = LB_K_S; e2.dens[1] = mu + N; e2.out[1] = q + N;
  LB_CHECK(run_epilogue(c, prec, nsplit, 2, part, e2));
  k_a2_final<<<nb, 256, 0, c->stream>>>(N, tau, q, q + N, out);
  LB_LAUNCH(c);
  return LB_OK;
}

// ---------------------------------------------------------------------------
// public entry points
static int pair_prec(lb_ctx* c) {
  const int p = c->params.precision;
  return (p == LB_FP64 || p == LB_DF64) ? p : LB_FP32;
}

extern "C" int lb_far_sums(lb_ctx* c, int precision, int nrhs, const double* sigma, double* out) {
  if (!c) return lb_fail(nullptr, LB_EINVAL, "null context");
  if (!c->have_geom) return lb_fail(c, LB_ESTATE, "no geometry uploaded");
  if (!c->have_near) LB_CHECK(lb_build_near(c));
  if (nrhs < 1 || (precision != LB_FP64 && precision != LB_FP32 && precision != LB_DF64))
    return lb_fail(c, LB_EINVAL, "bad nrhs/precision");
  LB_CUDA(c, cudaSetDevice(c->device));
  const int64_t N = c->N;
  const double* din;
  double* dout;
  LB_CHECK(lb_stage_in(c, sigma, nrhs * N * sizeof(double), c->ws_stage_in, (const void**)&din));
  LB_CHECK(lb_stage_out(c, out, nrhs * 4 * N * sizeof(double), c->ws_stage_out, (void**)&dout));
  double* part;
  LB_CHECK(part_buffer(c, &part));
  for (int r = 0; r < nrhs; ++r) {
    void *A, *B;
    int nsplit = 0;
    LB_CHECK(pack_sources(c, precision, din + r * N, nullptr, &A, &B));
    LB_CHECK(lb_far_launch(c, FAR_KALL, precision, A, B, part, &nsplit));
    EpiSpec sp{};
    sp.nout = 4;
    for (int k = 0; k < 4; ++k) {
      sp.acc[k] = k;
      sp.scale[k] = (k == LB_K_SP) ? -LB_INV4PI : LB_INV4PI;
      sp.kern[k] = -1;
      sp.out[k] = dout + ((int64_t)r * 4 + k) * N;
    }
    const unsigned grid = lb_div_up(N * 32, 256);
    if (precision == LB_FP64)
      k_epilogue<0><<<grid, 256, 0, c->stream>>>(N, c->np, 1, nsplit, 4, part, c->nrm, c->row_ptr, c->near_patch, nullptr,
                                                 nullptr, nullptr, sp);
    else if (precision == LB_FP32)
      k_epilogue<1><<<grid, 256, 0, c->stream>>>(N, c->np, 1, nsplit, 4, part, c->nrm, c->row_ptr, c->near_patch, nullptr,
                                                 nullptr, nullptr, sp);
    else
      k_epilogue<2><<<grid, 256, 0, c->stream>>>(N, c->np, 1, nsplit, 4, part, c->nrm, c->row_ptr, c->near_patch, nullptr,
                                                 nullptr, nullptr, sp);
    LB_LAUNCH(c);
  }
  return lb_stage_out_finish(c, out, dout, nrhs * 4 * N * sizeof(double));
}

static int apply_kernel(lb_ctx* c, int k, int nrhs, const double* sigma, double* out) {
  LB_CHECK(lb_require_corr(c));
  if (nrhs < 1) return lb_fail(c, LB_EINVAL, "nrhs must be >= 1");
  LB_CUDA(c, cudaSetDevice(c->device));
  const int64_t N = c->N;
  const double* din;
  double* dout;
  LB_CHECK(lb_stage_in(c, sigma, nrhs * N * sizeof(double), c->ws_stage_in, (const void**)&din));
  LB_CHECK(lb_stage_out(c, out, nrhs * N * sizeof(double), c->ws_stage_out, (void**)&dout));
  LB_CHECK(lb_ensure(c, c->ws_vec, (size_t)(4 * N) * sizeof(double)));
  double* pot = (double*)c->ws_vec.p;
  for (int r = 0; r < nrhs; ++r) {
    LB_CHECK(lb_potentials(c, pair_prec(c), din + r * N, pot, 1u << k));
    LB_CUDA(c, cudaMemcpyAsync(dout + r * N, pot + (int64_t)k * N, N * sizeof(double), cudaMemcpyDeviceToDevice,
                               c->stream));
  }
  return lb_stage_out_finish(c, out, dout, nrhs * N * sizeof(double));
}

extern "C" int lb_apply_S(lb_ctx* c, int nrhs, const double* s, double* o) { return apply_kernel(c, LB_K_S, nrhs, s, o); }
extern "C" int lb_apply_Sp(lb_ctx* c, int nrhs, const double* s, double* o) { return apply_kernel(c, LB_K_SP, nrhs, s, o); }
extern "C" int lb_apply_D(lb_ctx* c, int nrhs, const double* s, double* o) { return apply_kernel(c, LB_K_D, nrhs, s, o); }
extern "C" int lb_apply_SppDp(lb_ctx* c, int nrhs, const double* s, double* o) {
  return apply_kernel(c, LB_K_SPPDP, nrhs, s, o);
}

extern "C" int lb_apply_A(lb_ctx* c, int nrhs, const double* tau, double* out) {
  LB_CHECK(lb_require_corr(c));
  if (nrhs < 1) return lb_fail(c, LB_EINVAL, "nrhs must be >= 1");
  LB_CUDA(c, cudaSetDevice(c->device));
  const int64_t N = c->N;
  const double* din;
  double* dout;
  LB_CHECK(lb_stage_in(c, tau, nrhs * N * sizeof(double), c->ws_stage_in, (const void**)&din));
  LB_CHECK(lb_stage_out(c, out, nrhs * N * sizeof(double), c->ws_stage_out, (void**)&dout));
  const int prec = pair_prec(c);
  if (c->params.formulation == LB_A3 && prec != LB_FP64 && nrhs >= 2 && !c->far_order) {
    // several densities per far-field pass
    LB_CHECK(lb_apply_a3_batch(c, prec, nrhs, din, dout, nullptr));
  } else {
    for (int r = 0; r < nrhs; ++r)
      LB_CHECK(lb_apply_op(c, c->params.formulation, prec, din + r * N, dout + r * N));
  }
  return lb_stage_out_finish(c, out, dout, nrhs * N * sizeof(double));
}

// ---------------------------------------------------------------------------
// Far sums without allocation.
//
// For callers that cannot allocate device memory themselves: code running
// inside another framework's memory pool that owns every allocation on the
// device, or a service that must keep a fixed device footprint after
// start-up.  Same float32 far-field
// kernel as lb_far_sums, with every piece of scratch (packed sources, the
// near-tile flag table, split partials) in one file-scope device array of
// fixed size.  Every GPU that loads the library holds this array until the
// process exits.

#define LB_NOALLOC_MAX_N 65536                      // nodes
#define LB_NOALLOC_SPLITS 4                         // source splits (partials)
#define LB_NOALLOC_TB 512                           // targets per block of the float32 kernel
#define LB_NOALLOC_TS 128                           // sources per tile of the float32 kernel
#define LB_NOALLOC_BYTES (12u << 20)                // 12 MiB

static __device__ __align__(256) unsigned char g_noalloc_scratch[LB_NOALLOC_BYTES];

static std::mutex g_noalloc_mutex;
static void* g_noalloc_addr[64] = {nullptr};

// mean node position (one block, fixed order) to recentre the float32 coordinates
__global__ void k_noalloc_center(int64_t N, const double* __restrict__ X, double* __restrict__ c) {
  __shared__ double sh[3][256];
  double a[3] = {0, 0, 0};
  for (int64_t i = threadIdx.x; i < N; i += blockDim.x)
    for (int k = 0; k < 3; ++k) a[k] += X[3 * i + k];
  for (int k = 0; k < 3; ++k) sh[k][threadIdx.x] = a[k];
  __syncthreads();
  if (threadIdx.x == 0)
    for (int k = 0; k < 3; ++k) {
      double t = 0;
      for (int j = 0; j < (int)blockDim.x; ++j) t += sh[k][j];
      c[k] = t / (double)N;
    }
}

// A = (x - c, w sigma), B = (n, 0); padding far away with zero charge
__global__ void k_noalloc_pack(int64_t N, int64_t Npad, const double* __restrict__ X, const double* __restrict__ n,
                               const double* __restrict__ w, const double* __restrict__ sigma,
                               const double* __restrict__ c, float4* __restrict__ A, float4* __restrict__ B) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= Npad) return;
  if (i < N) {
    A[i] = make_float4((float)(X[3 * i] - c[0]), (float)(X[3 * i + 1] - c[1]), (float)(X[3 * i + 2] - c[2]),
                       (float)(w[i] * sigma[i]));
    B[i] = make_float4((float)n[3 * i], (float)n[3 * i + 1], (float)n[3 * i + 2], 0.f);
  } else {
    A[i] = make_float4(1e15f, 1e15f, 1e15f, 0.f);
    B[i] = make_float4(0.f, 0.f, 0.f, 0.f);
  }
}

// Address of the scratch array on the current device, looked up once per
// device (host code cannot use the array's name as a device pointer).  With
// CUDA's lazy module loading the array itself is created on a device by this
// first lookup, so the first call on a device can fail for lack of memory.
static int noalloc_scratch(void** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
    cudaGetLastError();
    return lb_fail(nullptr, LB_ECUDA, "lb_far_sums_noalloc: no current CUDA device");
  }
  std::lock_guard<std::mutex> lock(g_noalloc_mutex);
  if (!g_noalloc_addr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p)
      return lb_fail(nullptr, LB_ECUDA, "lb_far_sums_noalloc: cudaGetSymbolAddress failed: %s",
                     cudaGetErrorString(e));
    g_noalloc_addr[dev] = p;
  }
  *out = g_noalloc_addr[dev];
  return LB_OK;
}

extern "C" int lb_far_sums_noalloc(int64_t npatch, int np, const double* X, const double* nrm, const double* w,
                                   const double* sigma, const int64_t* row_ptr, const int32_t* near_patch,
                                   double* out, void* stream) {
  if (npatch < 1 || np < 3 || !X || !nrm || !w || !sigma || !row_ptr || !near_patch || !out)
    return lb_fail(nullptr, LB_EINVAL, "lb_far_sums_noalloc: null pointer, npatch < 1 or np < 3");
  // compare before multiplying: npatch * np could overflow int64
  if (np > LB_NOALLOC_MAX_N || npatch > LB_NOALLOC_MAX_N / np)
    return lb_fail(nullptr, LB_EINVAL,
                   "lb_far_sums_noalloc: npatch = %lld patches of %d nodes exceeds the maximum of %d nodes",
                   (long long)npatch, np, LB_NOALLOC_MAX_N);
  const int64_t N = npatch * np;
  void* base = nullptr;
  LB_CHECK(noalloc_scratch(&base));
  cudaStream_t st = (cudaStream_t)stream;
  const int64_t Npad = ((N + 1023) / 1024) * 1024;
  const int64_t ntb = (N + LB_NOALLOC_TB - 1) / LB_NOALLOC_TB;
  const int64_t ntiles = Npad / LB_NOALLOC_TS;
  const int64_t nsplit = std::min<int64_t>(LB_NOALLOC_SPLITS, ntiles);
  const int tps = (int)((ntiles + nsplit - 1) / nsplit);
  // carve the array: centre | A | B | flags | partials (256-byte aligned pieces)
  auto align = [](size_t x) { return (x + 255) & ~(size_t)255; };
  char* p = (char*)base;
  size_t off = 0;
  double* cen = (double*)(p + off); off = align(off + 4 * sizeof(double));
  float4* A = (float4*)(p + off); off = align(off + Npad * sizeof(float4));
  float4* B = (float4*)(p + off); off = align(off + Npad * sizeof(float4));
  uint8_t* flags = (uint8_t*)(p + off); off = align(off + (size_t)(ntb * ntiles));
  double* part = (double*)(p + off); off = align(off + (size_t)(nsplit * 4 * N) * sizeof(double));
  if (off > LB_NOALLOC_BYTES)
    return lb_fail(nullptr, LB_EINVAL, "lb_far_sums_noalloc: scratch of %zu bytes exceeds %u", off,
                   LB_NOALLOC_BYTES);
  // the flag table is the only piece that must start at zero
  cudaError_t e = cudaMemsetAsync(flags, 0, (size_t)(ntb * ntiles), st);
  if (e != cudaSuccess) return lb_fail(nullptr, LB_ECUDA, "lb_far_sums_noalloc: %s", cudaGetErrorString(e));
  k_noalloc_center<<<1, 256, 0, st>>>(N, X, cen);
  k_noalloc_pack<<<lb_div_up(Npad, 256), 256, 0, st>>>(N, Npad, X, nrm, w, sigma, cen, A, B);
  k_mask_flags<<<lb_div_up(N, 256), 256, 0, st>>>(N, np, LB_NOALLOC_TB, LB_NOALLOC_TS, ntiles, row_ptr, near_patch,
                                                    flags);
  dim3 grid((unsigned)ntb, (unsigned)nsplit);
  k_far<float, FAR_KALL, 4, 128, LB_NOALLOC_TS><<<grid, 128, 0, st>>>(N, np, A, B, A, B, flags, ntiles, row_ptr,
                                                                      near_patch, tps, part);
  EpiSpec sp{};
  sp.nout = 4;
  for (int k = 0; k < 4; ++k) {
    sp.acc[k] = k;
    sp.scale[k] = (k == LB_K_SP) ? -LB_INV4PI : LB_INV4PI;
    sp.kern[k] = -1;
    sp.out[k] = out + (int64_t)k * N;
  }
  k_epilogue<1><<<lb_div_up(N * 32, 256), 256, 0, st>>>(N, np, 1, (int)nsplit, 4, part, nrm, row_ptr, near_patch,
                                                        nullptr, nullptr, nullptr, sp);
  e = cudaGetLastError();
  if (e != cudaSuccess) return lb_fail(nullptr, LB_ECUDA, "lb_far_sums_noalloc launch: %s", cudaGetErrorString(e));
  return LB_OK;
}
