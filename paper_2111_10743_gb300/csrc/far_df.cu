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
  // t: x_hi[3], x_lo[3], n_hi[3], n_lo[3] of the target.  The grid
  // difference is exact and either zero or at least h, the lo difference at
  // most h, so FastTwoSum renormalises d exactly; without it |lo| / |hi| can
  // reach h / r (2e-5 for close pairs on a large surface), and the products
  // below, which drop lo * lo and round hi * lo to float, would lose that
  // ratio squared.
  const F2 dx = fast_two_sum(t[0] - A.x, t[3] - B.x);
  const F2 dy = fast_two_sum(t[1] - A.y, t[4] - B.y);
  const F2 dz = fast_two_sum(t[2] - A.z, t[5] - B.z);
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

// ---------------------------------------------------------------------------
// Symmetric pair sums (node sources, passes K1 and K2).  The kernels are
// functions of d = x_i - y_j, r and the two normals, so one evaluation of an
// unordered pair {i, j} serves both directions: d, r, 1/r, 1/r^3, n_i.d,
// n_j.d and 1 - n_i.n_j are shared, and only the charges and the signs of
// the odd terms differ (for target j: d -> -d, so n_j.d' = -n_j.d and
// (n_j - n_i).d' = (n_i - n_j).d).  Each CTA takes one pair of node blocks
// (I, J), I <= J, B nodes each: thread t holds target i = I B + t and loops
// over the sources j of block J, accumulating its own (i-side) sums in
// registers.  The j-side sums circulate: in each 32 x 32 warp tile lane t
// takes source (t + k) mod 32 at step k and hands its j-side sums one lane
// down after it (eight shuffles per step), so that after 32 steps lane t
// holds the warp's sums for source t; a sum over the CTA's warps in shared
// memory follows.  Diagonal blocks (I = J) take the i-side only, so every
// ordered pair is evaluated exactly once.  The near mask
// holds per direction (Near is not symmetric): bit patch(j) of Near(i) for
// the i-side, bit patch(i) of Near(j), gathered per source into shared
// memory, for the j-side.  Sums leave each CTA as float64 additions to
// out[4][N] (red.global.add.f64): the order of those additions, and so the
// last bit of the result, is not fixed from run to run.
template <int KIND, bool MASKED = true>
__device__ __forceinline__ void df_pair_sym(const float* t, const float4& A, const float4& B, const float4& C,
                                            const float4& D, bool mi, bool mj, F2* acci, F2* accj) {
  // t: x_hi[3], x_lo[3], n_hi[3], n_lo[3], q1 (hi, lo), q2 (hi, lo) of the target
  const F2 dx = fast_two_sum(t[0] - A.x, t[3] - B.x);
  const F2 dy = fast_two_sum(t[1] - A.y, t[4] - B.y);
  const F2 dz = fast_two_sum(t[2] - A.z, t[5] - B.z);
  const F2 r2 = df_add(df_add(df_sqr(dx), df_sqr(dy)), df_sqr(dz));
  F2 rinv = df_rsqrt(r2);
  if (MASKED && mi && mj) rinv = {0.f, 0.f};  // both directions masked (the self pair, padding)
  const F2 zero = {0.f, 0.f};
  const F2 q1j = MASKED && mi ? zero : F2{A.w, B.w};    // source charges, i-side
  const F2 q1i = MASKED && mj ? zero : F2{t[12], t[13]};  // target charges, j-side
  const F2 rinv2 = df_sqr(rinv);
  const F2 rinv3 = df_mul(rinv2, rinv);
  if (KIND == FAR_K1) {
    // S: q / r; gradient sums: q d / r^3 (d' = -d for the j-side)
    df_acc(acci[0], df_mul(q1j, rinv));
    df_acc(accj[0], df_mul(q1i, rinv));
    const F2 tj = df_mul(q1j, rinv3);
    const F2 ti = df_mul(F2{-q1i.h, -q1i.l}, rinv3);
    df_acc(acci[1], df_mul(tj, dx));
    df_acc(acci[2], df_mul(tj, dy));
    df_acc(acci[3], df_mul(tj, dz));
    df_acc(accj[1], df_mul(ti, dx));
    df_acc(accj[2], df_mul(ti, dy));
    df_acc(accj[3], df_mul(ti, dz));
    return;
  }
  // FAR_K2: q1 = mu1, q2 = mu2
  const F2 q2j = MASKED && mi ? zero : F2{C.w, D.w};
  const F2 q2i = MASKED && mj ? zero : F2{t[14], t[15]};
  const F2 nxx = {t[6], t[9]}, nxy = {t[7], t[10]}, nxz = {t[8], t[11]};
  const F2 nyx = {C.x, D.x}, nyy = {C.y, D.y}, nyz = {C.z, D.z};
  const F2 a = df_dot3(nxx, nxy, nxz, dx, dy, dz);  // n_i.d
  const F2 b = df_dot3(nyx, nyy, nyz, dx, dy, dz);  // n_j.d
  const F2 cc = df_sub(a, b);                       // (n_i - n_j).d
  const F2 hdn2 = df_sub({1.f, 0.f}, df_dot3(nxx, nxy, nxz, nyx, nyy, nyz));
  const F2 c3 = df_scale(df_mul(cc, rinv2), 3.f);   // 3 (n_i - n_j).d / r^2
  // i-side: K = 3 a c / r^2 - (1 - n_i.n_j); j-side: -(3 b c / r^2 + 1 - n_i.n_j)
  const F2 kki = df_sub(df_mul(a, c3), hdn2);
  const F2 kkj = df_add(df_mul(b, c3), hdn2);
  const F2 tti = df_mul(a, rinv3);
  const F2 ttj = df_mul(F2{-b.h, -b.l}, rinv3);
  df_acc(acci[0], df_mul(q1j, tti));
  df_acc(acci[1], df_mul(q2j, rinv));
  df_acc(acci[2], df_mul(q2j, tti));
  df_acc(acci[3], df_mul(df_mul(q2j, rinv3), kki));
  df_acc(accj[0], df_mul(q1i, ttj));
  df_acc(accj[1], df_mul(q2i, rinv));
  df_acc(accj[2], df_mul(q2i, ttj));
  df_acc(accj[3], df_mul(df_mul(F2{-q2i.h, -q2i.l}, rinv3), kkj));
}

// NT: targets per lane (the CTA has 128 / NT threads for a 128-node block)
template <int KIND, int NT>
__global__ void __launch_bounds__(128 / NT) k_far_df_sym(int64_t N, int np, int nb, const float4* __restrict__ S,
                                                         int64_t Npad, const uint8_t* __restrict__ flags,
                                                         int64_t ntiles, const int64_t* __restrict__ row_ptr,
                                                         const int32_t* __restrict__ near_patch,
                                                         double* __restrict__ out) {
  constexpr int NO = 4, B = 128, NTH = B / NT, NW = NTH / 32;
  __shared__ float4 sA[B], sB[B], sC[B], sD[B];
  __shared__ unsigned long long sMask[B];
  __shared__ int sLp[B];
  __shared__ F2 sRed[NW][B][NO];
  int64_t I, J;
  tri_pair(blockIdx.x, I, J);
  const bool diag = I == J;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int64_t P0I = (I * B) / np, P0J = (J * B) / np;
  const bool any = flags[I * ntiles + J] != 0 || flags[J * ntiles + I] != 0;
  // stage block J with its j-side masks (bit p: patch P0I + p in Near(j))
#pragma unroll
  for (int u = 0; u < NT; ++u) {
    const int ls = tid + u * NTH;
    const int64_t j = J * B + ls;
    sA[ls] = S[j];
    sB[ls] = S[Npad + j];
    sC[ls] = S[2 * Npad + j];
    sD[ls] = S[3 * Npad + j];
    sLp[ls] = (int)(j / np - P0J);
    unsigned long long mj = 0ull;
    if (any && !diag && j < N)
      for (int64_t bb = row_ptr[j]; bb < row_ptr[j + 1]; ++bb) {
        const int64_t d = (int64_t)near_patch[bb] - P0I;
        if (d >= 0 && d < 64) mj |= 1ull << d;
      }
    sMask[ls] = mj;
  }
  // the targets i = I B + tid + t NTH: data, i-side masks over block J's
  // patches, patch offsets
  float tv[NT][16];
  unsigned long long mi[NT];
  int lpi[NT];
  bool pad[NT];
  F2 acci[NT][NO];
#pragma unroll
  for (int t = 0; t < NT; ++t) {
    const int64_t i = I * B + tid + t * NTH;
    const float4 a = S[i], b = S[Npad + i], c = S[2 * Npad + i], d = S[3 * Npad + i];
    tv[t][0] = a.x; tv[t][1] = a.y; tv[t][2] = a.z;
    tv[t][3] = b.x; tv[t][4] = b.y; tv[t][5] = b.z;
    tv[t][6] = c.x; tv[t][7] = c.y; tv[t][8] = c.z;
    tv[t][9] = d.x; tv[t][10] = d.y; tv[t][11] = d.z;
    tv[t][12] = a.w; tv[t][13] = b.w; tv[t][14] = c.w; tv[t][15] = d.w;
    mi[t] = 0ull;
    if (any && i < N)
      for (int64_t bb = row_ptr[i]; bb < row_ptr[i + 1]; ++bb) {
        const int64_t dd = (int64_t)near_patch[bb] - P0J;
        if (dd >= 0 && dd < 64) mi[t] |= 1ull << dd;
      }
    lpi[t] = (int)(i / np - P0I);
    pad[t] = i >= N;
#pragma unroll
    for (int o = 0; o < NO; ++o) acci[t][o] = {0.f, 0.f};
  }
  __syncthreads();
  if (diag) {  // the target side only, every source of the block in turn
    F2 none[NO] = {};  // j-side sums of the diagonal: charges masked, never read
    for (int s = 0; s < B; ++s)
#pragma unroll
      for (int t = 0; t < NT; ++t) {
        const bool msk_i = pad[t] || ((mi[t] >> sLp[s]) & 1ull);
        df_pair_sym<KIND>(tv[t], sA[s], sB[s], sC[s], sD[s], msk_i, true, acci[t], none);
      }
  } else {
    // 32 x 32 warp tiles: at step k lane t takes source (t + k) mod 32 of the
    // tile, and the source-side sums move one lane down after each step, so
    // that lane t holds the sums of source (t + k) mod 32 throughout and of
    // source t after the 32nd step
    for (int r = 0; r < B / 32; ++r) {
      F2 accj[NO];
#pragma unroll
      for (int o = 0; o < NO; ++o) accj[o] = {0.f, 0.f};
      if (!any) {  // no near pair in either direction (and no padded target off the diagonal)
#pragma unroll 2
        for (int k = 0; k < 32; ++k) {
          const int s = 32 * r + ((lane + k) & 31);
          const float4 a = sA[s], b = sB[s], c = sC[s], d = sD[s];
#pragma unroll
          for (int t = 0; t < NT; ++t) df_pair_sym<KIND, false>(tv[t], a, b, c, d, false, false, acci[t], accj);
#pragma unroll
          for (int o = 0; o < NO; ++o) accj[o] = shfl_idx_v(accj[o], (lane + 1) & 31);
        }
      } else {
        for (int k = 0; k < 32; ++k) {
          const int s = 32 * r + ((lane + k) & 31);
          const float4 a = sA[s], b = sB[s], c = sC[s], d = sD[s];
          const int lp = sLp[s];
          const unsigned long long ms = sMask[s];
#pragma unroll
          for (int t = 0; t < NT; ++t) {
            const bool msk_i = (mi[t] >> lp) & 1ull;
            const bool msk_j = (ms >> lpi[t]) & 1ull;
            df_pair_sym<KIND>(tv[t], a, b, c, d, msk_i, msk_j, acci[t], accj);
          }
#pragma unroll
          for (int o = 0; o < NO; ++o) accj[o] = shfl_idx_v(accj[o], (lane + 1) & 31);
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
      for (int o = 0; o < NO; ++o) red_add_f64(out + o * N + i, df_to_double(acci[t][o]));
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
      F2 v = sRed[0][ls][o];
#pragma unroll
      for (int w = 1; w < NW; ++w) v = df_add(v, sRed[w][ls][o]);
      red_add_f64(out + o * N + j, df_to_double(v));
    }
  }
}

template <int KIND, int NT>
static int launch_df_sym(lb_ctx* c, const void* S, double* part) {
  constexpr int B = 128;
  if (c->np * 62 < B) return lb_fail(c, LB_EINVAL, "patch too small for the source tile");
  if (c->Npad % B) return lb_fail(c, LB_EINVAL, "node padding is not a multiple of the block");
  MaskTable* m = nullptr;
  LB_CHECK(lb_get_mask_src(c, B, B, c->np, c->Npad, &m));
  const int64_t nb = m->ntb;  // blocks holding nodes; the rest are padding
  const int64_t nblk = nb * (nb + 1) / 2;
  if (nblk > 0x7fffffffLL) return lb_fail(c, LB_EINVAL, "too many node blocks for one launch");
  LB_CUDA(c, cudaMemsetAsync(part, 0, 4 * c->N * sizeof(double), c->stream));
  const int64_t pairs = c->N * c->N;
  ProfScope prof(c, LB_PROF_FARDF_K1 + KIND, pairs);
  k_far_df_sym<KIND, NT><<<(unsigned)nblk, B / NT, 0, c->stream>>>(c->N, c->np, (int)nb, (const float4*)S, c->Npad,
                                                                  m->flags, m->ntiles, c->row_ptr, c->near_patch,
                                                                  part);
  LB_LAUNCH(c);
  lb_pair_counter += pairs;
  return LB_OK;
}

struct DfSymLaunch {
  int kind;
  const void* S;
  double* part;
};
// variant 0: one target per lane, 1: two
static int df_sym_cb(lb_ctx* c, int v, void* arg) {
  const DfSymLaunch* a = (const DfSymLaunch*)arg;
  if (a->kind == FAR_K1)
    return v == 0 ? launch_df_sym<FAR_K1, 1>(c, a->S, a->part) : launch_df_sym<FAR_K1, 2>(c, a->S, a->part);
  return v == 0 ? launch_df_sym<FAR_K2, 1>(c, a->S, a->part) : launch_df_sym<FAR_K2, 2>(c, a->S, a->part);
}

int lb_far_launch_df(lb_ctx* c, int kind, const void* S, double* part, int* nsplit) {
  if ((kind == FAR_K1 || kind == FAR_K2) && !c->far_order) {
    *nsplit = -1;
    // one or two targets per lane, timed on first use
    DfSymLaunch a{kind, S, part};
    int v = 0;
    LB_CHECK(lb_tune_choice(c, LB_TUNE_DFSYM + kind, 2, df_sym_cb, &a, &v));
    return df_sym_cb(c, v, &a);
  }
  switch (kind) {
    case FAR_K1: return launch_df_t<FAR_K1>(c, S, part, nsplit);
    case FAR_KALL: return launch_df_t<FAR_KALL>(c, S, part, nsplit);
    case FAR_K2: return launch_df_t<FAR_K2>(c, S, part, nsplit);
    default: return launch_df_t<FAR_K4>(c, S, part, nsplit);
  }
}
