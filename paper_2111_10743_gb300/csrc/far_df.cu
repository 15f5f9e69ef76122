// Far-field pair sums in double-float arithmetic (float32 pairs, ~1e-14).
//
// GB300 executes float64 at a small fraction of its float32 rate, so the
// accurate pair sums (refinement residuals, the solution potentials u =
// S[S[sigma]], LB_DF64 solves) carry every quantity as an unevaluated sum of
// two floats, hi + lo, and use the error-free transformations of Knuth
// (TwoSum), Dekker (FastTwoSum) and the fused-multiply-add TwoProduct, with a
// Newton step for the reciprocal square root (y <- y + y (1 - x y^2) / 2).
// Positions are split on a common grid: hi is an integer multiple of
// h = 2^(e-23) with 2^e above every recentred coordinate, so that hi
// differences between nodes are exact in float32 and d = (x_hi - y_hi) +
// (x_lo - y_lo) needs no error correction.  The sums and kernels are those of
// far.cu (Section 3 kernels, Section 4.2/4.3 passes); only the arithmetic
// differs.  Accumulation: hi by TwoSum, lo collects the errors and the lo
// parts of the terms.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>

#include "dfloat.cuh"
#include "internal.cuh"

template <int KIND> struct DfOut { static const int n = 4; };
template <> struct DfOut<FAR_K4> { static const int n = 2; };

// sources: A = (x_hi, q1_hi), B = (x_lo, q1_lo), C = (n_hi, q2_hi), D = (n_lo, q2_lo)
template <int KIND>
__device__ __forceinline__ void df_pair(const float* t, const float4& A, const float4& B, const float4& C,
                                        const float4& D, bool masked, F2* acc) {
  // t: x_hi[3], x_lo[3], n_hi[3], n_lo[3] of the target
  const F2 dx = {t[0] - A.x, t[3] - B.x};
  const F2 dy = {t[1] - A.y, t[4] - B.y};
  const F2 dz = {t[2] - A.z, t[5] - B.z};
  const F2 r2 = df_add(df_add(df_sqr(dx), df_sqr(dy)), df_sqr(dz));
  F2 rinv = df_rsqrt(r2);
  if (masked) rinv = {0.f, 0.f};
  const F2 q1 = {A.w, B.w};
  if (KIND == FAR_K1) {
    df_acc(acc[0], df_mul(q1, rinv));
    const F2 tt = df_mul(q1, df_mul(df_sqr(rinv), rinv));
    df_acc(acc[1], df_mul(tt, dx));
    df_acc(acc[2], df_mul(tt, dy));
    df_acc(acc[3], df_mul(tt, dz));
    return;
  }
  const F2 rinv2 = df_sqr(rinv);
  const F2 rinv3 = df_mul(rinv2, rinv);
  const F2 nyx = {C.x, D.x}, nyy = {C.y, D.y}, nyz = {C.z, D.z};
  if (KIND == FAR_K4) {
    const F2 nyd = df_dot3(nyx, nyy, nyz, dx, dy, dz);
    df_acc(acc[0], df_mul(q1, df_mul(nyd, rinv3)));
    df_acc(acc[1], df_mul({C.w, D.w}, rinv));
    return;
  }
  const F2 nxx = {t[6], t[9]}, nxy = {t[7], t[10]}, nxz = {t[8], t[11]};
  const F2 nxd = df_dot3(nxx, nxy, nxz, dx, dy, dz);
  const F2 nyd = df_dot3(nyx, nyy, nyz, dx, dy, dz);
  // (n_x - n_y).d = n_x.d - n_y.d, and for unit normals |n_x - n_y|^2 / 2 =
  // 1 - n_x.n_y (double-float keeps its absolute error near 1e-16)
  const F2 dnd = df_sub(nxd, nyd);
  const F2 hdn2 = df_sub({1.f, 0.f}, df_dot3(nxx, nxy, nxz, nyx, nyy, nyz));
  // 3 (n_x.d)((n_x - n_y).d) / r^2 - |n_x - n_y|^2 / 2
  const F2 kk = df_sub(df_scale(df_mul(df_mul(nxd, dnd), rinv2), 3.f), hdn2);
  if (KIND == FAR_KALL) {
    const F2 qr3 = df_mul(q1, rinv3);
    df_acc(acc[0], df_mul(q1, rinv));
    df_acc(acc[1], df_mul(qr3, nyd));
    df_acc(acc[2], df_mul(qr3, nxd));
    df_acc(acc[3], df_mul(qr3, kk));
  } else {  // FAR_K2: q1 = mu1, q2 = mu2
    const F2 q2 = {C.w, D.w};
    const F2 tt = df_mul(nxd, rinv3);
    df_acc(acc[0], df_mul(q1, tt));
    df_acc(acc[1], df_mul(q2, rinv));
    df_acc(acc[2], df_mul(q2, tt));
    df_acc(acc[3], df_mul(df_mul(q2, rinv3), kk));
  }
}

template <int KIND, int NT, int NTH, int TS>
__global__ void __launch_bounds__(NTH) k_far_df(int64_t N, int np, const float4* __restrict__ S,
                                                const uint8_t* __restrict__ flags, int64_t ntiles,
                                                const int64_t* __restrict__ row_ptr,
                                                const int32_t* __restrict__ near_patch, int tiles_per_split,
                                                int64_t Npad, const float4* __restrict__ T, int64_t Tpad,
                                                double* __restrict__ part) {
  constexpr int NO = DfOut<KIND>::n;
  // S holds four planes of Npad float4: A, B, C, D (sources, np per patch);
  // T four planes of Tpad float4 in the same layout (targets: the nodes)
  const float4* __restrict__ SA = S;
  const float4* __restrict__ SB = S + Npad;
  const float4* __restrict__ SC = S + 2 * Npad;
  const float4* __restrict__ SD = S + 3 * Npad;
  __shared__ float4 sA[TS], sB[TS], sC[TS], sD[TS];
  __shared__ int sLp[TS];
  const int64_t t0 = (int64_t)blockIdx.x * (NTH * NT);
  float tv[NT][12];
  F2 acc[NT][NO];
#pragma unroll
  for (int j = 0; j < NT; ++j) {
    const int64_t t = t0 + threadIdx.x + j * NTH;
    const float4 a = T[t], b = T[Tpad + t], c = T[2 * Tpad + t], d = T[3 * Tpad + t];
    tv[j][0] = a.x; tv[j][1] = a.y; tv[j][2] = a.z;
    tv[j][3] = b.x; tv[j][4] = b.y; tv[j][5] = b.z;
    tv[j][6] = c.x; tv[j][7] = c.y; tv[j][8] = c.z;
    tv[j][9] = d.x; tv[j][10] = d.y; tv[j][11] = d.z;
#pragma unroll
    for (int o = 0; o < NO; ++o) acc[j][o] = {0.f, 0.f};
  }
  const int64_t tile_b = (int64_t)blockIdx.y * tiles_per_split;
  const int64_t tile_e = min(ntiles, tile_b + tiles_per_split);
  for (int64_t tile = tile_b; tile < tile_e; ++tile) {
    const int64_t s0 = tile * TS;
    const int64_t P0 = s0 / np;
    for (int s = threadIdx.x; s < TS; s += NTH) {
      sA[s] = SA[s0 + s];
      sB[s] = SB[s0 + s];
      sC[s] = SC[s0 + s];
      sD[s] = SD[s0 + s];
      sLp[s] = (int)((s0 + s) / np - P0);
    }
    __syncthreads();
    const bool any_near = flags[(int64_t)blockIdx.x * ntiles + tile] != 0;
    unsigned long long m[NT];
#pragma unroll
    for (int j = 0; j < NT; ++j) {
      m[j] = 0ull;
      const int64_t t = t0 + threadIdx.x + j * NTH;
      if (any_near && t < N)
        for (int64_t bb = row_ptr[t]; bb < row_ptr[t + 1]; ++bb) {
          const int64_t d = (int64_t)near_patch[bb] - P0;
          if (d >= 0 && d < 64) m[j] |= 1ull << d;
        }
    }
    for (int s = 0; s < TS; ++s) {
      const float4 a = sA[s], b = sB[s], c = sC[s], d = sD[s];
      const int lp = sLp[s];
#pragma unroll
      for (int j = 0; j < NT; ++j) df_pair<KIND>(tv[j], a, b, c, d, (m[j] >> lp) & 1ull, acc[j]);
    }
    // renormalise the accumulators so that lo stays within an ulp of hi
#pragma unroll
    for (int j = 0; j < NT; ++j)
#pragma unroll
      for (int o = 0; o < NO; ++o) acc[j][o] = fast_two_sum(acc[j][o].h, acc[j][o].l);
    __syncthreads();
  }
#pragma unroll
  for (int j = 0; j < NT; ++j) {
    const int64_t t = t0 + threadIdx.x + j * NTH;
    if (t >= N) continue;
#pragma unroll
    for (int o = 0; o < NO; ++o)
      reinterpret_cast<float2*>(part)[((int64_t)blockIdx.y * NO + o) * N + t] = make_float2(acc[j][o].h, acc[j][o].l);
  }
}

// four planes (A, B, C, D) of Npad float4: hi/lo position on the grid h,
// hi/lo normal, hi/lo charges w d1 (A, B) and w d2 (C, D)
__global__ void k_pack_df(int64_t N, int64_t Npad, const double* __restrict__ X, const double* __restrict__ nrm,
                          const double* __restrict__ w, const double* __restrict__ d1, const double* __restrict__ d2,
                          double cx, double cy, double cz, double h, float4* __restrict__ S) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= Npad) return;
  float4 A, B, C, D;
  if (i < N) {
    const double c[3] = {cx, cy, cz};
    float hi[3], lo[3], nh[3], nl[3];
    for (int k = 0; k < 3; ++k) {
      const double x = X[3 * i + k] - c[k];
      const double xh = rint(x / h) * h;
      hi[k] = (float)xh;
      lo[k] = (float)(x - xh);
      const double n = nrm[3 * i + k];
      nh[k] = (float)n;
      nl[k] = (float)(n - (double)nh[k]);
    }
    const double q1 = w[i] * d1[i];
    const double q2 = d2 ? w[i] * d2[i] : 0.0;
    const float q1h = (float)q1, q2h = (float)q2;
    A = make_float4(hi[0], hi[1], hi[2], q1h);
    B = make_float4(lo[0], lo[1], lo[2], (float)(q1 - (double)q1h));
    C = make_float4(nh[0], nh[1], nh[2], q2h);
    D = make_float4(nl[0], nl[1], nl[2], (float)(q2 - (double)q2h));
  } else {
    A = make_float4(1e15f, 1e15f, 1e15f, 0.f);
    B = make_float4(0.f, 0.f, 0.f, 0.f);
    C = B;
    D = B;
  }
  S[i] = A;
  S[Npad + i] = B;
  S[2 * Npad + i] = C;
  S[3 * Npad + i] = D;
}

int lb_pack_df(lb_ctx* c, const double* d1, const double* d2, void* S) {
  k_pack_df<<<lb_div_up(c->Npad, 256), 256, 0, c->stream>>>(c->N, c->Npad, c->X, c->nrm, c->w, d1, d2, c->center[0],
                                                             c->center[1], c->center[2], c->df_grid, (float4*)S);
  LB_LAUNCH(c);
  return LB_OK;
}

// the same planes for n explicit points (padded to npad): positions Y, normals
// nY, weights wY (the oversampled far rule's sources)
int lb_pack_df_points(lb_ctx* c, int64_t n, int64_t npad, const double* Y, const double* nY, const double* wY,
                      const double* d1, const double* d2, void* S) {
  k_pack_df<<<lb_div_up(npad, 256), 256, 0, c->stream>>>(n, npad, Y, nY, wY, d1, d2, c->center[0], c->center[1],
                                                         c->center[2], c->df_grid, (float4*)S);
  LB_LAUNCH(c);
  return LB_OK;
}

template <int KIND>
static int launch_df_t(lb_ctx* c, const void* S, double* part, int* nsplit_out) {
  constexpr int NT = 2, NTH = 128, TS = 64;
  const int tb = NT * NTH;
  // sources: the nodes, or the oversampled far rule's points followed by the
  // nodes' own planes as targets (lb_far_rule_pack)
  const int snp = c->far_order ? c->nps : c->np;
  const int64_t spad = c->far_order ? c->Nspad : c->Npad;
  const float4* T = c->far_order ? (const float4*)S + 4 * spad : (const float4*)S;
  const int64_t pairs = c->N * (c->far_order ? c->Ns : c->N);
  if (snp * 62 < TS) return lb_fail(c, LB_EINVAL, "patch too small for the source tile");
  MaskTable* m = nullptr;
  LB_CHECK(lb_get_mask_src(c, tb, TS, snp, spad, &m));
  const int64_t ntb = m->ntb, ntiles = m->ntiles;
  int nsplit = 1;
  LB_CHECK(lb_pick_nsplit(c, k_far_df<KIND, NT, NTH, TS>, NTH, ntb, ntiles, &nsplit));
  const int tps = (int)((ntiles + nsplit - 1) / nsplit);
  dim3 grid((unsigned)ntb, (unsigned)nsplit);
  ProfScope prof(c, LB_PROF_FARDF_K1 + KIND, pairs);
  k_far_df<KIND, NT, NTH, TS><<<grid, NTH, 0, c->stream>>>(c->N, snp, (const float4*)S, m->flags, ntiles,
                                                           c->row_ptr, c->near_patch, tps, spad, T, c->Npad, part);
  LB_LAUNCH(c);
  lb_pair_counter += pairs;
  *nsplit_out = (int)nsplit;
  return LB_OK;
}

int lb_far_launch_df(lb_ctx* c, int kind, const void* S, double* part, int* nsplit) {
  switch (kind) {
    case FAR_K1: return launch_df_t<FAR_K1>(c, S, part, nsplit);
    case FAR_KALL: return launch_df_t<FAR_KALL>(c, S, part, nsplit);
    case FAR_K2: return launch_df_t<FAR_K2>(c, S, part, nsplit);
    default: return launch_df_t<FAR_K4>(c, S, part, nsplit);
  }
}
