// Batched applies: several densities per far-field pass.
//
// The paper's vector FMM (Section 4, the n_d densities of the FMM formula,
// Table 1) shares everything that does not depend on the density; the
// direct-sum analogue shares the pair geometry (d, 1/r, 1/r^3, the normal
// products of S''+D') between RC densities evaluated against the same
// (target, source) pair, and the correction SpMV reads each weight block once
// for all of them.  One thread per target, RC <= 8 densities per launch, the
// tile / split / near-mask structure of the single-density kernels; float32
// (compensated per tile) and double-float variants of A3's two passes
// (K1: S and grad S of tau; K2: S'[mu1], S[mu2], S'[mu2], (S''+D')[mu2]).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <map>
#include <mutex>
#include <tuple>
#include <type_traits>

#include "dfloat.cuh"
#include "internal.cuh"


namespace {

struct FFb {
  float hi, lo;
  __device__ __forceinline__ void add(float p) {
    const float s = hi + p;
    const float bp = s - hi;
    lo += (hi - (s - bp)) + (p - bp);
    hi = s;
  }
};

// bitmask of the near patches of target t among the 64 patches from P0
__device__ __forceinline__ unsigned long long near_bits(bool any, int64_t t, int64_t N, int64_t P0,
                                                        const int64_t* __restrict__ row_ptr,
                                                        const int32_t* __restrict__ near_patch) {
  unsigned long long m = 0ull;
  if (any && t < N)
    for (int64_t bb = row_ptr[t]; bb < row_ptr[t + 1]; ++bb) {
      const int64_t d = (int64_t)near_patch[bb] - P0;
      if (d >= 0 && d < 64) m |= 1ull << d;
    }
  return m;
}

}  // namespace

// ---------------------------------------------------------------------------
// float32.  P = (x - c, .), Nn = (n, .); charges Q[Npad][NPL*RC] (plane 0:
// tau or mu1, plane 1: mu2), weighted by the quadrature weights.
// part[split][r][o][N].
template <int KIND, int RC, int NTH, int TS>
__global__ void __launch_bounds__(NTH) k_farb32(int64_t N, int np, const float4* __restrict__ P,
                                                   const float4* __restrict__ Nn, const float4* __restrict__ Q,
                                                   const uint8_t* __restrict__ flags, int64_t ntiles,
                                                   const int64_t* __restrict__ row_ptr,
                                                   const int32_t* __restrict__ near_patch, int tiles_per_split,
                                                   double* __restrict__ part) {
  constexpr int NO = 4;
  constexpr bool K2 = KIND == FAR_K2;
  constexpr int NQ4 = (K2 ? 2 : 1) * RC / 4;  // float4 charge groups per source
  static_assert(NQ4 >= 1, "RC must allow a float4 of charges");
  __shared__ float4 sP[TS];
  __shared__ float4 sN[K2 ? TS : 1];
  __shared__ float4 sQ[TS * NQ4];
  __shared__ int sLp[TS];
  const int64_t t = (int64_t)blockIdx.x * NTH + threadIdx.x;
  const float4 tp = P[t];
  float nx = 0.f, ny = 0.f, nz = 0.f;
  if (K2) {
    const float4 tn = Nn[t];
    nx = tn.x; ny = tn.y; nz = tn.z;
  }
  float acc[RC][NO];
  FFb tot[RC][NO];
#pragma unroll
  for (int r = 0; r < RC; ++r)
#pragma unroll
    for (int o = 0; o < NO; ++o) {
      acc[r][o] = 0.f;
      tot[r][o].hi = tot[r][o].lo = 0.f;
    }
  const int64_t tile_b = (int64_t)blockIdx.y * tiles_per_split;
  const int64_t tile_e = min(ntiles, tile_b + tiles_per_split);
  for (int64_t tile = tile_b; tile < tile_e; ++tile) {
    const int64_t s0 = tile * TS;
    const int64_t P0 = s0 / np;
    for (int s = threadIdx.x; s < TS; s += NTH) {
      sP[s] = P[s0 + s];
      if (K2) sN[s] = Nn[s0 + s];
      sLp[s] = (int)((s0 + s) / np - P0);
    }
    for (int k = threadIdx.x; k < TS * NQ4; k += NTH) sQ[k] = Q[s0 * NQ4 + k];
    __syncthreads();
    const unsigned long long m =
        near_bits(flags[(int64_t)blockIdx.x * ntiles + tile] != 0, t, N, P0, row_ptr, near_patch);
#pragma unroll 2
    for (int s = 0; s < TS; ++s) {
      float q[NQ4 * 4];
#pragma unroll
      for (int g = 0; g < NQ4; ++g) {
        const float4 v = sQ[s * NQ4 + g];
        q[4 * g] = v.x; q[4 * g + 1] = v.y; q[4 * g + 2] = v.z; q[4 * g + 3] = v.w;
      }
      const float4 a = sP[s];
      const float dx = tp.x - a.x, dy = tp.y - a.y, dz = tp.z - a.z;
      float rinv = rsqrt_approx(dx * dx + dy * dy + dz * dz);
      if ((m >> sLp[s]) & 1ull) rinv = 0.f;
      if (!K2) {
        const float rinv3 = rinv * rinv * rinv;
#pragma unroll
        for (int r = 0; r < RC; ++r) {
          acc[r][0] = fmaf(q[r], rinv, acc[r][0]);
          const float qt = q[r] * rinv3;
          acc[r][1] = fmaf(qt, dx, acc[r][1]);
          acc[r][2] = fmaf(qt, dy, acc[r][2]);
          acc[r][3] = fmaf(qt, dz, acc[r][3]);
        }
      } else {
        const float4 b = sN[s];
        const float rinv2 = rinv * rinv, rinv3 = rinv2 * rinv;
        const float nxd = nx * dx + ny * dy + nz * dz;
        const float tt = nxd * rinv3;
        const float ex = nx - b.x, ey = ny - b.y, ez = nz - b.z;
        const float dnd = ex * dx + ey * dy + ez * dz;
        const float dn2 = ex * ex + ey * ey + ez * ez;
        const float kr3 = rinv3 * ((nxd * dnd) * (3.f * rinv2) - 0.5f * dn2);
#pragma unroll
        for (int r = 0; r < RC; ++r) {
          const float q1 = q[r], q2 = q[(K2 ? RC : 0) + r];
          acc[r][0] = fmaf(q1, tt, acc[r][0]);
          acc[r][1] = fmaf(q2, rinv, acc[r][1]);
          acc[r][2] = fmaf(q2, tt, acc[r][2]);
          acc[r][3] = fmaf(q2, kr3, acc[r][3]);
        }
      }
    }
#pragma unroll
    for (int r = 0; r < RC; ++r)
#pragma unroll
      for (int o = 0; o < NO; ++o) {
        tot[r][o].add(acc[r][o]);
        acc[r][o] = 0.f;
      }
    __syncthreads();
  }
  if (t >= N) return;
#pragma unroll
  for (int r = 0; r < RC; ++r)
#pragma unroll
    for (int o = 0; o < NO; ++o)
      reinterpret_cast<float2*>(part)[(((int64_t)blockIdx.y * RC + r) * NO + o) * N + t] =
          make_float2(tot[r][o].hi, tot[r][o].lo);
}

// double-float.  G: four planes of Npad float4 (x hi, x lo, n hi, n lo; the
// hi position on the exact-difference grid); charges Q[Npad][NPL*RC] of
// float2 (hi, lo).
template <int KIND, int RC, int NTH, int TS>
__global__ void __maxnreg__(200) k_farbdf(int64_t N, int64_t Npad, int np, const float4* __restrict__ G,
                                                   const float4* __restrict__ Q, const uint8_t* __restrict__ flags,
                                                   int64_t ntiles, const int64_t* __restrict__ row_ptr,
                                                   const int32_t* __restrict__ near_patch, int tiles_per_split,
                                                   double* __restrict__ part) {
  constexpr int NO = 4;
  constexpr bool K2 = KIND == FAR_K2;
  constexpr int NQ4 = (K2 ? 2 : 1) * RC / 2;  // float4 = two (hi, lo) charges
  __shared__ float4 sA[TS], sB[TS];
  __shared__ float4 sC[K2 ? TS : 1], sD[K2 ? TS : 1];
  __shared__ float4 sQ[TS * NQ4];
  __shared__ int sLp[TS];
  const float4* GA = G;
  const float4* GB = G + Npad;
  const float4* GC = G + 2 * Npad;
  const float4* GD = G + 3 * Npad;
  const int64_t t = (int64_t)blockIdx.x * NTH + threadIdx.x;
  const float4 ta = GA[t], tb = GB[t];
  F2 nxx = {0.f, 0.f}, nxy = {0.f, 0.f}, nxz = {0.f, 0.f};
  if (K2) {
    const float4 tc = GC[t], td = GD[t];
    nxx = {tc.x, td.x}; nxy = {tc.y, td.y}; nxz = {tc.z, td.z};
  }
  F2 acc[RC][NO];
#pragma unroll
  for (int r = 0; r < RC; ++r)
#pragma unroll
    for (int o = 0; o < NO; ++o) acc[r][o] = {0.f, 0.f};
  const int64_t tile_b = (int64_t)blockIdx.y * tiles_per_split;
  const int64_t tile_e = min(ntiles, tile_b + tiles_per_split);
  for (int64_t tile = tile_b; tile < tile_e; ++tile) {
    const int64_t s0 = tile * TS;
    const int64_t P0 = s0 / np;
    for (int s = threadIdx.x; s < TS; s += NTH) {
      sA[s] = GA[s0 + s];
      sB[s] = GB[s0 + s];
      if (K2) {
        sC[s] = GC[s0 + s];
        sD[s] = GD[s0 + s];
      }
      sLp[s] = (int)((s0 + s) / np - P0);
    }
    for (int k = threadIdx.x; k < TS * NQ4; k += NTH) sQ[k] = Q[s0 * NQ4 + k];
    __syncthreads();
    const unsigned long long m =
        near_bits(flags[(int64_t)blockIdx.x * ntiles + tile] != 0, t, N, P0, row_ptr, near_patch);
    for (int s = 0; s < TS; ++s) {
      const float4 A = sA[s], B = sB[s];
      // exact renormalisation of the grid-split difference (as in far_df.cu)
      const F2 dx = fast_two_sum(ta.x - A.x, tb.x - B.x);
      const F2 dy = fast_two_sum(ta.y - A.y, tb.y - B.y);
      const F2 dz = fast_two_sum(ta.z - A.z, tb.z - B.z);
      F2 rinv = df_rsqrt(df_add(df_add(df_sqr(dx), df_sqr(dy)), df_sqr(dz)));
      if ((m >> sLp[s]) & 1ull) rinv = {0.f, 0.f};
      const F2 rinv2 = df_sqr(rinv);
      const F2 rinv3 = df_mul(rinv2, rinv);
      F2 q[NQ4 * 2];
#pragma unroll
      for (int g = 0; g < NQ4; ++g) {
        const float4 v = sQ[s * NQ4 + g];
        q[2 * g] = {v.x, v.y};
        q[2 * g + 1] = {v.z, v.w};
      }
      if (!K2) {
#pragma unroll
        for (int r = 0; r < RC; ++r) {
          df_acc(acc[r][0], df_mul(q[r], rinv));
          const F2 qt = df_mul(q[r], rinv3);
          df_acc(acc[r][1], df_mul(qt, dx));
          df_acc(acc[r][2], df_mul(qt, dy));
          df_acc(acc[r][3], df_mul(qt, dz));
        }
      } else {
        const float4 C = sC[s], D = sD[s];
        const F2 nyx = {C.x, D.x}, nyy = {C.y, D.y}, nyz = {C.z, D.z};
        const F2 nxd = df_dot3(nxx, nxy, nxz, dx, dy, dz);
        const F2 ex = df_add(nxx, {-nyx.h, -nyx.l}), ey = df_add(nxy, {-nyy.h, -nyy.l}),
                 ez = df_add(nxz, {-nyz.h, -nyz.l});
        const F2 dnd = df_dot3(ex, ey, ez, dx, dy, dz);
        const F2 dn2 = df_dot3(ex, ey, ez, ex, ey, ez);
        // 3 (n_x.d)((n_x - n_y).d) / r^2 - |n_x - n_y|^2 / 2
        const F2 kk = df_add(df_scale(df_mul(df_mul(nxd, dnd), rinv2), 3.f), df_scale(dn2, -0.5f));
        const F2 tt = df_mul(nxd, rinv3);
        const F2 kr3 = df_mul(kk, rinv3);
#pragma unroll
        for (int r = 0; r < RC; ++r) {
          const F2 q1 = q[r], q2 = q[(K2 ? RC : 0) + r];
          df_acc(acc[r][0], df_mul(q1, tt));
          df_acc(acc[r][1], df_mul(q2, rinv));
          df_acc(acc[r][2], df_mul(q2, tt));
          df_acc(acc[r][3], df_mul(q2, kr3));
        }
      }
    }
    // renormalise the accumulators so that lo stays within an ulp of hi
#pragma unroll
    for (int r = 0; r < RC; ++r)
#pragma unroll
      for (int o = 0; o < NO; ++o) {
        const float s = acc[r][o].h + acc[r][o].l;
        acc[r][o] = {s, acc[r][o].l - (s - acc[r][o].h)};
      }
    __syncthreads();
  }
  if (t >= N) return;
#pragma unroll
  for (int r = 0; r < RC; ++r)
#pragma unroll
    for (int o = 0; o < NO; ++o)
      reinterpret_cast<float2*>(part)[(((int64_t)blockIdx.y * RC + r) * NO + o) * N + t] =
          make_float2(acc[r][o].h, acc[r][o].l);
}

// ---------------------------------------------------------------------------
// charge packing: Q[i][pl*RC + r] = w_i d_pl[r][i] for the far field and
// D[i][pl*RC + r] = d_pl[r][i] for the correction sums (zero for padding and
// for densities beyond R)
__global__ void k_packq32(int64_t N, int64_t Npad, int R, int RC, int npl, const double* __restrict__ w,
                          const double* __restrict__ d1, const double* __restrict__ d2, float* __restrict__ Q,
                          float* __restrict__ D) {
  const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int per = npl * RC;
  if (k >= Npad * per) return;
  const int64_t i = k / per;
  const int j = (int)(k - i * per), pl = j / RC, r = j - pl * RC;
  const double d = (i < N && r < R) ? (pl ? d2 : d1)[(int64_t)r * N + i] : 0.0;
  Q[k] = i < N ? (float)(w[i] * d) : 0.f;
  D[k] = (float)d;
}

__global__ void k_packqdf(int64_t N, int64_t Npad, int R, int RC, int npl, const double* __restrict__ w,
                          const double* __restrict__ d1, const double* __restrict__ d2, float2* __restrict__ Q,
                          float2* __restrict__ D) {
  const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int per = npl * RC;
  if (k >= Npad * per) return;
  const int64_t i = k / per;
  const int j = (int)(k - i * per), pl = j / RC, r = j - pl * RC;
  const double d = (i < N && r < R) ? (pl ? d2 : d1)[(int64_t)r * N + i] : 0.0;
  const double q = i < N ? w[i] * d : 0.0;
  const float qh = (float)q, dh = (float)d;
  Q[k] = make_float2(qh, (float)(q - (double)qh));
  D[k] = make_float2(dh, (float)(d - (double)dh));
}

// ---------------------------------------------------------------------------
// batched epilogue: one warp per row i.  The lanes stride over the row's
// correction entries (each weight block read once for all densities; the
// densities of a node are adjacent in D) in float32 (MODE 1) or double-float
// (MODE 2) arithmetic, a reduce-scatter leaves correction (r, k) in lanes
// (r NK + k) << (5 - log2(RC NK)), and lane 4r + o sums the split partials
// of density r, output o.
//   pass 1: mu1 = S' tau (out0), mu2 = S tau (out1)
//   pass 2: S' mu1, S mu2, S' mu2, (S''+D') mu2 (out0..out3)
template <int RC, bool PASS2, int MODE>
__global__ void k_epib(int64_t N, int np, int64_t nnzb, int R, int nsplit, const double* __restrict__ part,
                       const double* __restrict__ nrm, const int64_t* __restrict__ row_ptr,
                       const int32_t* __restrict__ near_patch, const float4* __restrict__ vh,
                       const float4* __restrict__ vl, const float4* __restrict__ D, double* __restrict__ out0,
                       double* __restrict__ out1, double* __restrict__ out2, double* __restrict__ out3) {
  using T = typename std::conditional<MODE == 1, float, F2>::type;
  constexpr int NK = PASS2 ? 4 : 2;
  constexpr int V = RC * NK;
  constexpr int SH = 5 - Log2<V>::value;
  constexpr int NPL = PASS2 ? 2 : 1;
  constexpr int NV = NPL * RC;                   // density values per node
  constexpr int NF4 = MODE == 1 ? NV / 4 : NV / 2;  // float4 loads per node
  const int lane = threadIdx.x & 31;
  const int64_t i = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  if (i >= N) return;
  T cs[V];
#pragma unroll
  for (int k = 0; k < V; ++k) cs[k] = T{};
  // the row's (block, node) pairs flattened; each lane walks them 32 apart,
  // so that a warp reads 32 consecutive nodes' densities per load; the float
  // weights are stored kernel-major [kernel][block][npp], npp = np rounded up
  // to four, so that a warp's weights of one kernel are contiguous
  const int npp = (np + 3) & ~3;
  const int64_t rb = row_ptr[i];
  const int ne = (int)((row_ptr[i + 1] - rb) * np);
  const int64_t kp = nnzb * (int64_t)npp;  // floats per kernel plane
  int bo = lane / np, q = lane - (lane / np) * np;
  const float* vhf = reinterpret_cast<const float*>(vh);
  const float* vlf = reinterpret_cast<const float*>(vl);
  for (int e = lane; e < ne; e += 32) {
    const int64_t b = rb + bo;
    const int64_t col = (int64_t)near_patch[b] * np + q;
    const int64_t wo = b * npp + q;
    float dv[NF4 * 4];
#pragma unroll
    for (int g = 0; g < NF4; ++g) {
      const float4 v = __ldg(D + col * NF4 + g);
      dv[4 * g] = v.x; dv[4 * g + 1] = v.y; dv[4 * g + 2] = v.z; dv[4 * g + 3] = v.w;
    }
    if constexpr (MODE == 1) {
      const float wS = __ldg(vhf + wo + LB_K_S * kp), wSp = __ldg(vhf + wo + LB_K_SP * kp);
      const float wSD = PASS2 ? __ldg(vhf + wo + LB_K_SPPDP * kp) : 0.f;
      float* c = cs;
#pragma unroll
      for (int r = 0; r < RC; ++r) {
        const float x1 = dv[r];
        if (!PASS2) {
          c[r * NK] = fmaf(wS, x1, c[r * NK]);
          c[r * NK + 1] = fmaf(wSp, x1, c[r * NK + 1]);
        } else {
          const float x2 = dv[RC + r];
          c[r * NK] = fmaf(wSp, x1, c[r * NK]);
          c[r * NK + 1] = fmaf(wS, x2, c[r * NK + 1]);
          c[r * NK + 2] = fmaf(wSp, x2, c[r * NK + 2]);
          c[r * NK + 3] = fmaf(wSD, x2, c[r * NK + 3]);
        }
      }
    } else {
      const F2 wS = {__ldg(vhf + wo + LB_K_S * kp), __ldg(vlf + wo + LB_K_S * kp)};
      const F2 wSp = {__ldg(vhf + wo + LB_K_SP * kp), __ldg(vlf + wo + LB_K_SP * kp)};
      F2 wSD = {0.f, 0.f};
      if (PASS2) wSD = {__ldg(vhf + wo + LB_K_SPPDP * kp), __ldg(vlf + wo + LB_K_SPPDP * kp)};
      F2* c = cs;
#pragma unroll
      for (int r = 0; r < RC; ++r) {
        const F2 x1 = {dv[2 * r], dv[2 * r + 1]};
        if (!PASS2) {
          df_acc(c[r * NK], df_mul(wS, x1));
          df_acc(c[r * NK + 1], df_mul(wSp, x1));
        } else {
          const F2 x2 = {dv[2 * (RC + r)], dv[2 * (RC + r) + 1]};
          df_acc(c[r * NK], df_mul(wSp, x1));
          df_acc(c[r * NK + 1], df_mul(wS, x2));
          df_acc(c[r * NK + 2], df_mul(wSp, x2));
          df_acc(c[r * NK + 3], df_mul(wSD, x2));
        }
      }
    }
    q += 32;
    while (q >= np) { q -= np; ++bo; }
  }
  warp_reduce_scatter<V>(cs, lane);
  double cmine;
  if constexpr (MODE == 1) cmine = (double)cs[0];
  else cmine = df_to_double(cs[0]);
  const int rr = lane >> 2, o = lane & 3;
  // split partials: (hi, lo) float pairs summed in double-float arithmetic
  F2 as = {0.f, 0.f};
  if (rr < RC && rr < R)
    for (int s = 0; s < nsplit; ++s) {
      const float2 v = reinterpret_cast<const float2*>(part)[(((int64_t)s * RC + rr) * 4 + o) * N + i];
      as = df_add(as, {v.x, v.y});
    }
  const double a = df_to_double(as);
  if (!PASS2) {
    const int base = lane & ~3;
    const double g1 = __shfl_sync(0xffffffffu, a, base + 1);
    const double g2 = __shfl_sync(0xffffffffu, a, base + 2);
    const double g3 = __shfl_sync(0xffffffffu, a, base + 3);
    const double cS = __shfl_sync(0xffffffffu, cmine, ((rr * NK) << SH) & 31);
    const double cSp = __shfl_sync(0xffffffffu, cmine, ((rr * NK + 1) << SH) & 31);
    if (o == 0 && rr < RC && rr < R) {
      out1[(int64_t)rr * N + i] = a * LB_INV4PI + cS;
      out0[(int64_t)rr * N + i] = -(nrm[3 * i] * g1 + nrm[3 * i + 1] * g2 + nrm[3 * i + 2] * g3) * LB_INV4PI + cSp;
    }
  } else {
    const double cv = __shfl_sync(0xffffffffu, cmine, ((rr * NK + o) << SH) & 31);
    if (rr < RC && rr < R) {
      double* dst = o == 0 ? out0 : (o == 1 ? out1 : (o == 2 ? out2 : out3));
      const double sgn = (o == 0 || o == 2) ? -LB_INV4PI : LB_INV4PI;
      dst[(int64_t)rr * N + i] = sgn * a + cv;
    }
  }
}

// weighted sums of R vectors: partial[r][blk]
__global__ void k_wdot_batch(int64_t N, const double* __restrict__ w, const double* __restrict__ v,
                             double* __restrict__ partial) {
  __shared__ double sh[256];
  const int r = blockIdx.y;
  double s = 0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x)
    s += w[i] * v[(int64_t)r * N + i];
  sh[threadIdx.x] = s;
  __syncthreads();
  for (int k = blockDim.x / 2; k > 0; k >>= 1) {
    if (threadIdx.x < k) sh[threadIdx.x] += sh[threadIdx.x + k];
    __syncthreads();
  }
  if (threadIdx.x == 0) partial[(int64_t)r * gridDim.x + blockIdx.x] = sh[0];
}

// out_r = -tau/4 + S'mu1 - (S''+D')mu2 - 2 H S'mu2 + W S mu2 (Section 4.3);
// optionally u_r = S mu2 = S[S[tau]], the solution potential of tau
__global__ void k_a3_final_batch(int64_t N, const double* __restrict__ tau, const double* __restrict__ p0,
                                 const double* __restrict__ p1, const double* __restrict__ p2,
                                 const double* __restrict__ p3, const double* __restrict__ H,
                                 const double* __restrict__ partial, int npart, double area, double* __restrict__ out,
                                 double* __restrict__ u) {
  const int r = blockIdx.y;
  __shared__ double eta;
  if (threadIdx.x == 0) {
    double s = 0;
    for (int k = 0; k < npart; ++k) s += partial[(int64_t)r * npart + k];
    eta = s / area;
  }
  __syncthreads();
  const int64_t o = (int64_t)r * N;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
    out[o + i] = -0.25 * tau[o + i] + p0[o + i] - p3[o + i] - 2.0 * H[i] * p2[o + i] + eta;
    if (u) u[o + i] = p1[o + i];
  }
}

// ---------------------------------------------------------------------------
// Launch shapes and their tuning.
//
// A batched pass can run with 128 or 256 threads per block (one target each)
// and 64 or 128 sources per shared-memory tile; the number of source splits
// (gridDim.y) is then chosen so that the grid fills whole waves of resident
// blocks.  Which shape is fastest depends on the kernel, the density count
// and N, so the first pass of each kind (not under a stream capture) times
// every shape once on the real data with CUDA events and keeps the fastest
// in a process-wide table: every later pass, every context of the process
// and every graph replay then run that shape.  GBLB_BATCH_SHAPE = 0, 1 or 2
// in the environment forces one shape.
struct BShape {
  int nth, ts;
};
static const BShape kShapes[3] = {{128, 64}, {128, 128}, {256, 64}};

// largest split count a batched launch can pick (workspace sizing)
static int64_t max_nsplit(lb_ctx* c) { return std::min<int64_t>(c->Npad / 64, 32); }

// one far-field pass of shape (NTH, TS); Q (and G for double-float) packed
template <int KIND, int RC, int NTH, int TS>
static int far_shape(lb_ctx* c, bool df, const void* G, const void* Q, double* part, int* nsplit_out, int cat,
                     int64_t pairs) {
  MaskTable* m = nullptr;
  LB_CHECK(lb_get_mask(c, NTH, TS, &m));
  const int64_t ntb = m->ntb, ntiles = m->ntiles;
  int nsplit = 1;
  if (!df) {
    auto kern = k_farb32<KIND, RC, NTH, TS>;
    LB_CHECK(lb_pick_nsplit(c, kern, NTH, ntb, ntiles, &nsplit));
    const int tps = (int)((ntiles + nsplit - 1) / nsplit);
    ProfScope prof(c, cat, pairs);
    kern<<<dim3((unsigned)ntb, (unsigned)nsplit), NTH, 0, c->stream>>>(
        c->N, c->np, c->pos32, c->nrm32, (const float4*)Q, m->flags, ntiles, c->row_ptr, c->near_patch, tps, part);
    LB_LAUNCH(c);
  } else {
    auto kern = k_farbdf<KIND, RC, NTH, TS>;
    LB_CHECK(lb_pick_nsplit(c, kern, NTH, ntb, ntiles, &nsplit));
    const int tps = (int)((ntiles + nsplit - 1) / nsplit);
    ProfScope prof(c, cat, pairs);
    kern<<<dim3((unsigned)ntb, (unsigned)nsplit), NTH, 0, c->stream>>>(
        c->N, c->Npad, c->np, (const float4*)G, (const float4*)Q, m->flags, ntiles, c->row_ptr, c->near_patch, tps,
        part);
    LB_LAUNCH(c);
  }
  *nsplit_out = nsplit;
  return LB_OK;
}

template <int KIND, int RC>
static int far_any_shape(lb_ctx* c, int shape, bool df, const void* G, const void* Q, double* part, int* nsplit,
                         int cat, int64_t pairs) {
  switch (shape) {
    case 1: return far_shape<KIND, RC, 128, 128>(c, df, G, Q, part, nsplit, cat, pairs);
    case 2: return far_shape<KIND, RC, 256, 64>(c, df, G, Q, part, nsplit, cat, pairs);
    default: return far_shape<KIND, RC, 128, 64>(c, df, G, Q, part, nsplit, cat, pairs);
  }
}

namespace {
struct TuneKey {
  int device;
  int64_t N;
  int np, RC, kind, prec;
  bool operator<(const TuneKey& o) const {
    return std::tie(device, N, np, RC, kind, prec) < std::tie(o.device, o.N, o.np, o.RC, o.kind, o.prec);
  }
};
std::mutex g_tune_mu;
std::map<TuneKey, int> g_tune;
}  // namespace

// the shape for this pass: forced, tuned earlier, tuned now, or (under a
// stream capture, where nothing may be timed) the first shape
template <int KIND, int RC>
static int tuned_shape(lb_ctx* c, bool df, const void* G, const void* Q, double* part, int* shape) {
  if (const char* env = getenv("GBLB_BATCH_SHAPE")) {
    const int s = atoi(env);
    if (s >= 0 && s < 3) { *shape = s; return LB_OK; }
  }
  const TuneKey key{c->device, c->N, c->np, RC, KIND, df ? LB_DF64 : LB_FP32};
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tune.find(key);
    if (it != g_tune.end()) { *shape = it->second; return LB_OK; }
  }
  *shape = 0;
  if (c->capturing) return LB_OK;
  cudaEvent_t e0, e1;
  LB_CUDA(c, cudaEventCreate(&e0));
  LB_CUDA(c, cudaEventCreate(&e1));
  float best_ms = 1e30f;
  int best = 0, rc = LB_OK;
  const int prof = c->prof_on;
  c->prof_on = 0;  // tuning launches are not part of any profile
  for (int s = 0; s < 3 && rc == LB_OK; ++s) {
    int ns = 0;
    rc = far_any_shape<KIND, RC>(c, s, df, G, Q, part, &ns, 0, 0);  // warm-up: mask table, caches
    if (rc != LB_OK) break;
    cudaEventRecord(e0, c->stream);
    rc = far_any_shape<KIND, RC>(c, s, df, G, Q, part, &ns, 0, 0);
    cudaEventRecord(e1, c->stream);
    if (rc != LB_OK) break;
    float ms = 0.f;
    if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
      rc = lb_fail(c, LB_ECUDA, "timing a batched launch shape failed");
      break;
    }
    if (ms < best_ms) { best_ms = ms; best = s; }
  }
  c->prof_on = prof;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc != LB_OK) return rc;
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tune[key] = best;
  }
  *shape = best;
  return LB_OK;
}

template <int RC>
static int launch_pass(lb_ctx* c, int prec, bool pass2, int R, const double* d1, const double* d2, double* part,
                       int* nsplit_out) {
  const int64_t Npad = c->Npad;
  const int npl = pass2 ? 2 : 1;
  const int64_t nq = Npad * npl * RC;
  const bool df = prec != LB_FP32;
  const void* G = nullptr;
  const void* Q = nullptr;
  if (!df) {
    LB_CHECK(lb_ensure(c, c->ws_src, (size_t)nq * sizeof(float)));
    LB_CHECK(lb_ensure(c, c->ws_dlow, (size_t)nq * sizeof(float)));
    float* q = (float*)c->ws_src.p;
    k_packq32<<<lb_div_up(nq, 256), 256, 0, c->stream>>>(c->N, Npad, R, RC, npl, c->w, d1, d2, q,
                                                          (float*)c->ws_dlow.p);
    LB_LAUNCH(c);
    Q = q;
  } else {
    // geometry planes of the double-float kernels, then the charges
    const size_t geo = 4 * (size_t)Npad * sizeof(float4);
    LB_CHECK(lb_ensure(c, c->ws_src, geo + (size_t)nq * sizeof(float2)));
    LB_CHECK(lb_ensure(c, c->ws_dlow, (size_t)nq * sizeof(float2)));
    void* g = c->ws_src.p;
    float2* q = (float2*)((char*)g + geo);
    LB_CHECK(lb_pack_df(c, d1, nullptr, g));  // positions and normals; its charge slots are not read
    k_packqdf<<<lb_div_up(nq, 256), 256, 0, c->stream>>>(c->N, Npad, R, RC, npl, c->w, d1, d2, q,
                                                          (float2*)c->ws_dlow.p);
    LB_LAUNCH(c);
    G = g;
    Q = q;
  }
  const int cat = df ? (pass2 ? LB_PROF_FARDF_K2 : LB_PROF_FARDF_K1) : (pass2 ? LB_PROF_FAR32_K2 : LB_PROF_FAR32_K1);
  int shape = 0;
  if (pass2) {
    LB_CHECK((tuned_shape<FAR_K2, RC>(c, df, G, Q, part, &shape)));
    LB_CHECK((far_any_shape<FAR_K2, RC>(c, shape, df, G, Q, part, nsplit_out, cat, c->N * c->N * R)));
  } else {
    LB_CHECK((tuned_shape<FAR_K1, RC>(c, df, G, Q, part, &shape)));
    LB_CHECK((far_any_shape<FAR_K1, RC>(c, shape, df, G, Q, part, nsplit_out, cat, c->N * c->N * R)));
  }
  lb_pair_counter += c->N * c->N * R;
  return LB_OK;
}

// the epilogue of a batched pass in the pass's arithmetic; densities in the
// layout the pack kernel left in ws_dlow
template <int RC, bool PASS2>
static int run_epib(lb_ctx* c, int prec, int R, int nsplit, const double* part, double* o0, double* o1, double* o2,
                    double* o3) {
  LB_CHECK(lb_lowp_vals(c));
  const int64_t N = c->N;
  const unsigned eb = lb_div_up(N * 32, 256);
  const float4* D = (const float4*)c->ws_dlow.p;
  ProfScope prof(c, LB_PROF_EPILOGUE);
  const float4* vh = (const float4*)c->vals_hi;
  const float4* vl = (const float4*)c->vals_lo;
  if (prec == LB_FP32)
    k_epib<RC, PASS2, 1><<<eb, 256, 0, c->stream>>>(N, c->np, c->nnzb, R, nsplit, part, c->nrm, c->row_ptr,
                                                     c->near_patch, vh, nullptr, D, o0, o1, o2, o3);
  else
    k_epib<RC, PASS2, 2><<<eb, 256, 0, c->stream>>>(N, c->np, c->nnzb, R, nsplit, part, c->nrm, c->row_ptr,
                                                     c->near_patch, vh, vl, D, o0, o1, o2, o3);
  LB_LAUNCH(c);
  return LB_OK;
}

template <int RC>
static int apply_a3_chunk(lb_ctx* c, int prec, int R, const double* tau, double* out, double* u) {
  const int64_t N = c->N;
  LB_CHECK(lb_ensure(c, c->ws_bpot, (size_t)(6 * RC * N) * sizeof(double)));
  double* mu1 = (double*)c->ws_bpot.p;
  double* mu2 = mu1 + RC * N;
  double* p0 = mu2 + RC * N;
  double* p1 = p0 + RC * N;
  double* p2 = p1 + RC * N;
  double* p3 = p2 + RC * N;
  LB_CHECK(lb_ensure(c, c->ws_part, (size_t)(max_nsplit(c) * RC * 4 * N) * sizeof(double)));
  double* part = (double*)c->ws_part.p;
  const int RB = 64;
  LB_CHECK(lb_ensure(c, c->ws_red, (size_t)(RB * RC + 8) * sizeof(double)));
  double* partial = (double*)c->ws_red.p;
  int nsplit = 0;
  // pass 1: charges tau -> mu1 = S' tau, mu2 = S tau
  LB_CHECK(launch_pass<RC>(c, prec, false, R, tau, nullptr, part, &nsplit));
  LB_CHECK((run_epib<RC, false>(c, prec, R, nsplit, part, mu1, mu2, nullptr, nullptr)));
  // pass 2: charges mu1, mu2
  LB_CHECK(launch_pass<RC>(c, prec, true, R, mu1, mu2, part, &nsplit));
  LB_CHECK((run_epib<RC, true>(c, prec, R, nsplit, part, p0, p1, p2, p3)));
  k_wdot_batch<<<dim3(RB, R), 256, 0, c->stream>>>(N, c->w, p1, partial);
  LB_LAUNCH(c);
  const unsigned nb = (unsigned)std::min<int64_t>(2 * c->sm_count, lb_div_up(N, 256));
  k_a3_final_batch<<<dim3(nb, R), 256, 0, c->stream>>>(N, tau, p0, p1, p2, p3, c->H, partial, RB, c->area, out, u);
  LB_LAUNCH(c);
  if (prec == LB_FP32) lb_apply32_counter += R; else lb_apply64_counter += R;
  return LB_OK;
}

template <int RC>
static int apply_s_chunk(lb_ctx* c, int prec, int R, const double* sig, double* out) {
  const int64_t N = c->N;
  LB_CHECK(lb_ensure(c, c->ws_part, (size_t)(max_nsplit(c) * RC * 4 * N) * sizeof(double)));
  LB_CHECK(lb_ensure(c, c->ws_bpot, (size_t)(6 * RC * N) * sizeof(double)));
  double* part = (double*)c->ws_part.p;
  double* sp = (double*)c->ws_bpot.p;  // S' of the densities (not returned)
  int nsplit = 0;
  LB_CHECK(launch_pass<RC>(c, prec, false, R, sig, nullptr, part, &nsplit));
  return run_epib<RC, false>(c, prec, R, nsplit, part, sp, out, nullptr, nullptr);
}

// densities in chunks of 8, the remainder by 4
template <typename F8, typename F4>
static int chunked(int R, F8 f8, F4 f4) {
  for (int r0 = 0; r0 < R;) {
    const int left = R - r0;
    if (left > 4) { const int k = std::min(left, 8); LB_CHECK(f8(r0, k)); r0 += k; }
    else { LB_CHECK(f4(r0, left)); r0 += left; }
  }
  return LB_OK;
}

int lb_apply_a3_batch(lb_ctx* c, int prec, int R, const double* tau, double* out, double* u) {
  if (prec != LB_FP32 && prec != LB_DF64) return lb_fail(c, LB_EINVAL, "batched applies take LB_FP32 or LB_DF64");
  const int64_t N = c->N;
  auto um = [&](int r0) { return u ? u + (int64_t)r0 * N : nullptr; };
  return chunked(
      R, [&](int r0, int k) { return apply_a3_chunk<8>(c, prec, k, tau + (int64_t)r0 * N, out + (int64_t)r0 * N, um(r0)); },
      [&](int r0, int k) { return apply_a3_chunk<4>(c, prec, k, tau + (int64_t)r0 * N, out + (int64_t)r0 * N, um(r0)); });
}

int lb_apply_s_batch(lb_ctx* c, int prec, int R, const double* sig, double* out) {
  if (prec != LB_FP32 && prec != LB_DF64) return lb_fail(c, LB_EINVAL, "batched applies take LB_FP32 or LB_DF64");
  const int64_t N = c->N;
  return chunked(
      R, [&](int r0, int k) { return apply_s_chunk<8>(c, prec, k, sig + (int64_t)r0 * N, out + (int64_t)r0 * N); },
      [&](int r0, int k) { return apply_s_chunk<4>(c, prec, k, sig + (int64_t)r0 * N, out + (int64_t)r0 * N); });
}

// the tuned launch shapes for this context's surface: shapes[8] indexed by
// precision (0 float32, 1 double-float) * 4 + pass (0 K1, 1 K2) * 2 +
// (0: 4 densities, 1: 8 densities); -1 where that pass has not run yet
extern "C" int lb_get_tuning(lb_ctx* c, int* shapes) {
  if (!c || !shapes) return lb_fail(c, LB_EINVAL, "null argument");
  std::lock_guard<std::mutex> lk(g_tune_mu);
  for (int p = 0; p < 2; ++p)
    for (int k = 0; k < 2; ++k)
      for (int r = 0; r < 2; ++r) {
        const TuneKey key{c->device, c->N, c->np, r ? 8 : 4, k ? FAR_K2 : FAR_K1, p ? LB_DF64 : LB_FP32};
        auto it = g_tune.find(key);
        shapes[p * 4 + k * 2 + r] = it == g_tune.end() ? -1 : it->second;
      }
  for (int kind = 0; kind < 4; ++kind) shapes[8 + kind] = lb_far_tuned_variant(c, kind);
  shapes[12] = lb_tuned_choice(c, LB_TUNE_DFSYM + FAR_K1);
  shapes[13] = lb_tuned_choice(c, LB_TUNE_DFSYM + FAR_K2);
  return LB_OK;
}
