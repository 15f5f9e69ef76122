// Transposed applies, the adjoint (density) solve and the pair sums of the
// node-position gradient (at the end of this file).
//
// The discrete operators are matrices: S_ij = w_j G(x_i, x_j) for far pairs
// (patch(j) not in Near(i)) plus the correction weights C_ij for near ones,
// and likewise for S', D, S''+D' (Sections 3, 4).  Their transposes act on a
// vector y as
//   (S^T y)_j       = w_j sum_i G(x_i, x_j) y_i       + sum_i C^S_ij y_i,
//   (S'^T y)_j      = w_j sum_i n_i.d / (4 pi r^3) y_i + sum_i C^S'_ij y_i,
//   ((S''+D')^T y)_j = w_j sum_i [3 (n_i.d)((n_i - n_j).d)/r^2 - |n_i - n_j|^2/2]
//                      / (4 pi r^3) y_i               + sum_i C^SD_ij y_i,
// with d = x_j - x_i and the sums over i with patch(j) not in Near(i): the
// near relation is not symmetric, so the far sums skip, for target j, the
// sources i whose near list holds j's patch.  Those sources are a 64-bit mask
// per (target patch, 64-source tile), built exactly from the near lists, and
// the correction sums walk the near lists transposed to patch-major order.
// Everything here is float64.
//
// A3^T y = -y/4 + S'^T S'^T y - S^T (S''+D')^T y - S^T S'^T (2 H y)
//          + (sum y / |Gamma|) S^T S^T w,
// the transpose of A3 = -I/4 + S'S' - (S''+D')S - 2H S'S + W S S with
// W = 1 w^T / |Gamma|.  The adjoint of the solve u = S S A3^-1 P f, P the
// weighted mean projection I - 1 w^T / |Gamma|, is g_f = P^T A3^-T S^T S^T g_u.
//
// A2 = -I/4 + D D + S (-(S''+D') - 2H S' + 1 w^T S / |Gamma|) has
// A2^T y = -y/4 + D^T D^T y - (S''+D')^T t - S'^T (2 H t) + (sum t / |Gamma|) S^T w
// with t = S^T y, and (D^T y)_j = w_j sum_i -(n_j.d) / (4 pi r^3) y_i + ...;
// the A2 solve u = S A2^-1 S P f has the adjoint g_f = P^T S^T A2^-T S^T g_u.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <vector>

#include "internal.cuh"

#define TT_NT 2
#define TT_NTH 128
#define TT_TS 64  // one 64-bit source mask per tile
#define TT_TB (TT_NT * TT_NTH)

enum TKind { T_S = 0, T_P1 = 1, T_P2 = 2, T_DS = 3 };
template <int K> struct TOut { static const int n = 1; };
template <> struct TOut<T_P1> { static const int n = 3; };
template <> struct TOut<T_P2> { static const int n = 2; };
template <> struct TOut<T_DS> { static const int n = 2; };

// ---------------------------------------------------------------------------
// transposed near structure

// tmask[P][tile] bit s: source i = 64 tile + s has P in Near(i)
__global__ void k_tmask(int64_t N, const int64_t* __restrict__ row_ptr, const int32_t* __restrict__ near_patch,
                        int64_t ntiles, unsigned long long* __restrict__ tmask) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= N) return;
  for (int64_t b = row_ptr[i]; b < row_ptr[i + 1]; ++b)
    atomicOr(&tmask[(int64_t)near_patch[b] * ntiles + i / 64], 1ull << (i % 64));
}

// tflag[block][tile]: some target of the block has a masked source in the tile
__global__ void k_tflag(int64_t N, int np, int64_t npatch, int64_t ntb, int64_t ntiles,
                        const unsigned long long* __restrict__ tmask, uint8_t* __restrict__ tflag) {
  const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (k >= ntb * ntiles) return;
  const int64_t blk = k / ntiles, tile = k - blk * ntiles;
  const int64_t t0 = blk * TT_TB;
  uint8_t f = 0;
  if (t0 < N) {
    const int64_t p0 = t0 / np, p1 = (std::min<int64_t>(N, t0 + TT_TB) - 1) / np;
    for (int64_t p = p0; p <= p1 && p < npatch; ++p) f |= tmask[p * ntiles + tile] != 0ull;
  }
  tflag[k] = f;
}

int lb_build_transpose(lb_ctx* c) {
  if (c->have_trans) return LB_OK;
  LB_CHECK(lb_require_corr(c));
  const int64_t N = c->N, np = c->np, npatch = c->npatch, nnzb = c->nnzb;
  // patch-major lists of (row, block), rows ascending within each patch
  std::vector<int64_t> rp(N + 1);
  std::vector<int32_t> pl(nnzb);
  LB_CUDA(c, cudaMemcpyAsync(rp.data(), c->row_ptr, (N + 1) * sizeof(int64_t), cudaMemcpyDeviceToHost, c->stream));
  LB_CUDA(c, cudaMemcpyAsync(pl.data(), c->near_patch, nnzb * sizeof(int32_t), cudaMemcpyDeviceToHost, c->stream));
  LB_CUDA(c, cudaStreamSynchronize(c->stream));
  std::vector<int64_t> tp(npatch + 1, 0);
  for (int64_t b = 0; b < nnzb; ++b) ++tp[pl[b] + 1];
  for (int64_t p = 0; p < npatch; ++p) tp[p + 1] += tp[p];
  std::vector<int64_t> fill(tp.begin(), tp.end() - 1);
  std::vector<int32_t> trow(nnzb);
  std::vector<int64_t> tblk(nnzb);
  for (int64_t i = 0; i < N; ++i)
    for (int64_t b = rp[i]; b < rp[i + 1]; ++b) {
      const int64_t e = fill[pl[b]]++;
      trow[e] = (int32_t)i;
      tblk[e] = b;
    }
  LB_CHECK(lb_alloc(c, &c->tptr, (size_t)(npatch + 1)));
  LB_CHECK(lb_alloc(c, &c->trow, (size_t)std::max<int64_t>(nnzb, 1)));
  LB_CHECK(lb_alloc(c, &c->tblk, (size_t)std::max<int64_t>(nnzb, 1)));
  LB_CUDA(c, cudaMemcpyAsync(c->tptr, tp.data(), (npatch + 1) * sizeof(int64_t), cudaMemcpyHostToDevice, c->stream));
  LB_CUDA(c, cudaMemcpyAsync(c->trow, trow.data(), nnzb * sizeof(int32_t), cudaMemcpyHostToDevice, c->stream));
  LB_CUDA(c, cudaMemcpyAsync(c->tblk, tblk.data(), nnzb * sizeof(int64_t), cudaMemcpyHostToDevice, c->stream));
  // source masks and the tile flags of the target blocks
  c->t_ntiles = c->Npad / TT_TS;
  c->t_ntb = (N + TT_TB - 1) / TT_TB;
  LB_CHECK(lb_alloc(c, &c->tmask, (size_t)(npatch * c->t_ntiles)));
  LB_CHECK(lb_alloc(c, &c->tflag, (size_t)(c->t_ntb * c->t_ntiles)));
  LB_CUDA(c, cudaMemsetAsync(c->tmask, 0, (size_t)(npatch * c->t_ntiles) * sizeof(unsigned long long), c->stream));
  k_tmask<<<lb_div_up(N, 256), 256, 0, c->stream>>>(N, c->row_ptr, c->near_patch, c->t_ntiles, c->tmask);
  LB_LAUNCH(c);
  k_tflag<<<lb_div_up(c->t_ntb * c->t_ntiles, 256), 256, 0, c->stream>>>(N, (int)np, npatch, c->t_ntb, c->t_ntiles,
                                                                           c->tmask, c->tflag);
  LB_LAUNCH(c);
  LB_CUDA(c, cudaStreamSynchronize(c->stream));  // the host lists above are freed on return
  c->have_trans = true;
  return LB_OK;
}

// ---------------------------------------------------------------------------
// transposed far sums (float64)

// sources: A = (x - c, q1), B = (n, q2), unweighted densities
__global__ void k_pack_t(int64_t N, int64_t Npad, const double4_32a* __restrict__ pos,
                         const double4_32a* __restrict__ nrm, const double* __restrict__ d1,
                         const double* __restrict__ d2, double4_32a* __restrict__ A, double4_32a* __restrict__ B) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= Npad) return;
  if (i < N) {
    const double4_32a p = pos[i], n = nrm[i];
    A[i] = make_double4_32a(p.x, p.y, p.z, d1[i]);
    B[i] = make_double4_32a(n.x, n.y, n.z, d2 ? d2[i] : 0.0);
  } else {
    A[i] = make_double4_32a(1e15, 1e15, 1e15, 0.0);
    B[i] = make_double4_32a(0.0, 0.0, 0.0, 0.0);
  }
}

template <int KIND>
__device__ __forceinline__ void pair_t(const double* x, const double* nx, const double4_32a& a,
                                       const double4_32a& b, bool masked, double* acc) {
  const double dx = x[0] - a.x, dy = x[1] - a.y, dz = x[2] - a.z;  // d = x_j - x_i
  const double r2 = dx * dx + dy * dy + dz * dz;
  const double rinv = masked ? 0.0 : rsqrt(r2);
  if (KIND == T_S) {
    acc[0] += a.w * rinv;
    return;
  }
  if (KIND == T_DS) {  // D^T q1 (target normal), S^T q1
    const double nxd = nx[0] * dx + nx[1] * dy + nx[2] * dz;
    acc[0] -= a.w * nxd * rinv * rinv * rinv;
    acc[1] += a.w * rinv;
    return;
  }
  const double rinv2 = rinv * rinv, rinv3 = rinv2 * rinv;
  const double nyd = b.x * dx + b.y * dy + b.z * dz;  // n_i . d
  if (KIND == T_P2) {
    acc[0] += a.w * nyd * rinv3;  // S'^T q1
    acc[1] += b.w * rinv;         // S^T q2
    return;
  }
  // T_P1: S'^T q1, (S''+D')^T q1, S'^T q2
  const double ex = b.x - nx[0], ey = b.y - nx[1], ez = b.z - nx[2];  // n_i - n_j
  const double ed = ex * dx + ey * dy + ez * dz;
  const double e2 = ex * ex + ey * ey + ez * ez;
  acc[0] += a.w * nyd * rinv3;
  acc[1] += a.w * (3.0 * nyd * ed * rinv2 - 0.5 * e2) * rinv3;
  acc[2] += b.w * nyd * rinv3;
}

template <int KIND>
__global__ void __launch_bounds__(TT_NTH) k_far_t(int64_t N, int np, const double4_32a* __restrict__ tpos,
                                                  const double4_32a* __restrict__ tnrm,
                                                  const double4_32a* __restrict__ A, const double4_32a* __restrict__ B,
                                                  const uint8_t* __restrict__ tflag,
                                                  const unsigned long long* __restrict__ tmask, int64_t ntiles,
                                                  int tiles_per_split, double* __restrict__ part) {
  constexpr int NO = TOut<KIND>::n;
  __shared__ double4_32a sA[TT_TS], sB[TT_TS];
  const int64_t t0 = (int64_t)blockIdx.x * TT_TB;
  double x[TT_NT][3], nx[TT_NT][3], acc[TT_NT][NO];
  int64_t pj[TT_NT];
#pragma unroll
  for (int k = 0; k < TT_NT; ++k) {
    const int64_t t = t0 + threadIdx.x + k * TT_NTH;
    const double4_32a p = tpos[t], n = tnrm[t];
    x[k][0] = p.x; x[k][1] = p.y; x[k][2] = p.z;
    nx[k][0] = n.x; nx[k][1] = n.y; nx[k][2] = n.z;
    pj[k] = t < N ? t / np : -1;
#pragma unroll
    for (int o = 0; o < NO; ++o) acc[k][o] = 0.0;
  }
  const int64_t tile_b = (int64_t)blockIdx.y * tiles_per_split;
  const int64_t tile_e = min(ntiles, tile_b + tiles_per_split);
  for (int64_t tile = tile_b; tile < tile_e; ++tile) {
    for (int s = threadIdx.x; s < TT_TS; s += TT_NTH) {
      sA[s] = A[tile * TT_TS + s];
      sB[s] = B[tile * TT_TS + s];
    }
    __syncthreads();
    const bool any = tflag[(int64_t)blockIdx.x * ntiles + tile] != 0;
    unsigned long long m[TT_NT];
#pragma unroll
    for (int k = 0; k < TT_NT; ++k) m[k] = (any && pj[k] >= 0) ? tmask[pj[k] * ntiles + tile] : 0ull;
    for (int s = 0; s < TT_TS; ++s) {
      const double4_32a a = sA[s], b = sB[s];
#pragma unroll
      for (int k = 0; k < TT_NT; ++k) pair_t<KIND>(x[k], nx[k], a, b, (m[k] >> s) & 1ull, acc[k]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int k = 0; k < TT_NT; ++k) {
    const int64_t t = t0 + threadIdx.x + k * TT_NTH;
    if (t >= N) continue;
#pragma unroll
    for (int o = 0; o < NO; ++o) part[((int64_t)blockIdx.y * NO + o) * N + t] = acc[k][o];
  }
}

// out_o[j] = w_j / (4 pi) sum_s part[s][o][j]
__global__ void k_reduce_t(int64_t N, int nsplit, int nout, const double* __restrict__ part,
                           const double* __restrict__ w, double* __restrict__ out) {
  const int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (j >= N) return;
  for (int o = 0; o < nout; ++o) {
    double s = 0;
    for (int k = 0; k < nsplit; ++k) s += part[((int64_t)k * nout + o) * N + j];
    out[(int64_t)o * N + j] = w[j] * s * LB_INV4PI;
  }
}

// transposed correction sums: one warp per patch P, lanes over its nodes;
// out_o[P np + q] += sum over (i, b) listed for P of vals[b][kern_o][q] dens_o[i]
struct CorrT {
  int nout;
  int kern[3];
  const double* dens[3];
  double* out[3];
};

__global__ void k_corr_t(int64_t npatch, int np, const int64_t* __restrict__ tptr, const int32_t* __restrict__ trow,
                         const int64_t* __restrict__ tblk, const double* __restrict__ vals, CorrT sp) {
  const int lane = threadIdx.x & 31;
  const int64_t P = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  if (P >= npatch) return;
  for (int q = lane; q < np; q += 32) {
    double acc[3] = {0, 0, 0};
    for (int64_t e = tptr[P]; e < tptr[P + 1]; ++e) {
      const int64_t i = trow[e], b = tblk[e];
      const double* vb = vals + b * LB_NKERNELS * np + q;
#pragma unroll
      for (int o = 0; o < 3; ++o)
        if (o < sp.nout) acc[o] = fma(__ldg(vb + sp.kern[o] * np), sp.dens[o][i], acc[o]);
    }
#pragma unroll
    for (int o = 0; o < 3; ++o)
      if (o < sp.nout) sp.out[o][P * np + q] += acc[o];
  }
}

// ---------------------------------------------------------------------------
// one transposed pass: far sums of kind KIND for densities d1 (and d2) plus
// the transposed corrections spec; outputs out [nout][N]
struct TWork {
  double* part;
  double4_32a* A;
  double4_32a* B;
};

static int work_t(lb_ctx* c, TWork* w) {
  const int64_t N = c->N, Npad = c->Npad;
  const size_t part = (size_t)32 * 3 * N * sizeof(double);
  const size_t packed = 2 * (size_t)Npad * sizeof(double4_32a);
  LB_CHECK(lb_ensure(c, c->ws_adj, part + packed + (size_t)(12 * N + 256) * sizeof(double)));
  char* p = (char*)c->ws_adj.p;
  w->part = (double*)p;
  w->A = (double4_32a*)(p + part);
  w->B = w->A + Npad;
  return LB_OK;
}

// vectors for the passes, after the part and packed areas
static double* vec_t(lb_ctx* c, int k) {
  const size_t part = (size_t)32 * 3 * c->N * sizeof(double);
  const size_t packed = 2 * (size_t)c->Npad * sizeof(double4_32a);
  return (double*)((char*)c->ws_adj.p + part + packed) + (int64_t)k * c->N;
}

template <int KIND>
static int pass_t(lb_ctx* c, const double* d1, const double* d2, const CorrT& corr, double* out) {
  constexpr int NO = TOut<KIND>::n;
  const int64_t N = c->N;
  TWork w;
  LB_CHECK(work_t(c, &w));
  k_pack_t<<<lb_div_up(c->Npad, 256), 256, 0, c->stream>>>(N, c->Npad, c->pos64, c->nrm64, d1, d2, w.A, w.B);
  LB_LAUNCH(c);
  const int64_t ntb = c->t_ntb, ntiles = c->t_ntiles;
  const int64_t want = 6LL * c->sm_count;
  int64_t nsplit = std::max<int64_t>(1, std::min<int64_t>({ntiles, (want + ntb - 1) / ntb, (int64_t)32}));
  const int tps = (int)((ntiles + nsplit - 1) / nsplit);
  nsplit = (ntiles + tps - 1) / tps;
  {
    ProfScope prof(c, LB_PROF_FAR64_K1 + (KIND == T_S || KIND == T_DS ? 0 : 2), N * N);
    k_far_t<KIND><<<dim3((unsigned)ntb, (unsigned)nsplit), TT_NTH, 0, c->stream>>>(
        N, c->np, c->pos64, c->nrm64, w.A, w.B, c->tflag, c->tmask, ntiles, tps, w.part);
    LB_LAUNCH(c);
  }
  lb_pair_counter += N * N;
  k_reduce_t<<<lb_div_up(N, 256), 256, 0, c->stream>>>(N, (int)nsplit, NO, w.part, c->w, out);
  LB_LAUNCH(c);
  ProfScope prof(c, LB_PROF_EPILOGUE);
  k_corr_t<<<lb_div_up(c->npatch * 32, 256), 256, 0, c->stream>>>(c->npatch, c->np, c->tptr, c->trow, c->tblk,
                                                                   c->vals, corr);
  LB_LAUNCH(c);
  return LB_OK;
}

// S^T y -> out (device)
static int apply_st(lb_ctx* c, const double* y, double* out) {
  CorrT cs{};
  cs.nout = 1;
  cs.kern[0] = LB_K_S; cs.dens[0] = y; cs.out[0] = out;
  return pass_t<T_S>(c, y, nullptr, cs, out);
}

__global__ void k_scale_h(int64_t N, const double* __restrict__ H, const double* __restrict__ y,
                          double* __restrict__ out) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < N) out[i] = 2.0 * H[i] * y[i];
}

__global__ void k_add_t(int64_t N, const double* __restrict__ a, const double* __restrict__ b, double* __restrict__ s) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < N) s[i] = a[i] + b[i];
}

// out = -y/4 + b1 - b2 + (sum y / area) v0
__global__ void k_a3t_final(int64_t N, const double* __restrict__ y, const double* __restrict__ b1,
                            const double* __restrict__ b2, const double* __restrict__ v0,
                            const double* __restrict__ partial, int npart, double area, double* __restrict__ out) {
  __shared__ double eta;
  if (threadIdx.x == 0) {
    double s = 0;
    for (int k = 0; k < npart; ++k) s += partial[k];
    eta = s / area;
  }
  __syncthreads();
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = -0.25 * y[i] + b1[i] - b2[i] + eta * v0[i];
}

// plain sums of y in per-block partials (fixed order)
__global__ void k_sum_t(int64_t N, const double* __restrict__ y, double* __restrict__ partial) {
  __shared__ double sh[256];
  double s = 0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x)
    s += y[i];
  sh[threadIdx.x] = s;
  __syncthreads();
  for (int k = blockDim.x / 2; k > 0; k >>= 1) {
    if (threadIdx.x < k) sh[threadIdx.x] += sh[threadIdx.x + k];
    __syncthreads();
  }
  if (threadIdx.x == 0) partial[blockIdx.x] = sh[0];
}

#define T_RB 128

// v0 = S^T S^T w, kept until the corrections change
static int ensure_v0(lb_ctx* c) {
  if (c->v0) return LB_OK;
  LB_CHECK(lb_build_transpose(c));
  LB_CHECK(lb_alloc(c, &c->v0, (size_t)c->N));
  TWork w;
  LB_CHECK(work_t(c, &w));
  double* t = vec_t(c, 11);
  LB_CHECK(apply_st(c, c->w, t));
  LB_CHECK(apply_st(c, t, c->v0));
  return LB_OK;
}

int lb_apply_a3t(lb_ctx* c, const double* y, double* out) {
  LB_CHECK(lb_build_transpose(c));
  LB_CHECK(ensure_v0(c));
  const int64_t N = c->N;
  TWork w;
  LB_CHECK(work_t(c, &w));
  double* y2 = vec_t(c, 0);   // 2 H y
  double* o = vec_t(c, 1);    // [3][N]: S'^T y, (S''+D')^T y, S'^T (2Hy)
  double* s = vec_t(c, 4);    // (S''+D')^T y + S'^T (2Hy)
  double* b = vec_t(c, 5);    // [2][N]: S'^T o0, S^T s
  double* partial = vec_t(c, 12);  // T_RB doubles past the twelve vectors
  k_scale_h<<<lb_div_up(N, 256), 256, 0, c->stream>>>(N, c->H, y, y2);
  LB_LAUNCH(c);
  CorrT c1{};
  c1.nout = 3;
  c1.kern[0] = LB_K_SP; c1.dens[0] = y; c1.out[0] = o;
  c1.kern[1] = LB_K_SPPDP; c1.dens[1] = y; c1.out[1] = o + N;
  c1.kern[2] = LB_K_SP; c1.dens[2] = y2; c1.out[2] = o + 2 * N;
  LB_CHECK(pass_t<T_P1>(c, y, y2, c1, o));
  k_add_t<<<lb_div_up(N, 256), 256, 0, c->stream>>>(N, o + N, o + 2 * N, s);
  LB_LAUNCH(c);
  CorrT c2{};
  c2.nout = 2;
  c2.kern[0] = LB_K_SP; c2.dens[0] = o; c2.out[0] = b;
  c2.kern[1] = LB_K_S; c2.dens[1] = s; c2.out[1] = b + N;
  LB_CHECK(pass_t<T_P2>(c, o, s, c2, b));
  k_sum_t<<<T_RB, 256, 0, c->stream>>>(N, y, partial);
  LB_LAUNCH(c);
  const unsigned nb = (unsigned)std::min<int64_t>(4 * c->sm_count, lb_div_up(N, 256));
  k_a3t_final<<<nb, 256, 0, c->stream>>>(N, y, b, b + N, c->v0, partial, T_RB, c->area, out);
  LB_LAUNCH(c);
  ++lb_apply64_counter;
  return LB_OK;
}

// v1 = S^T w, kept until the corrections change
static int ensure_v1(lb_ctx* c) {
  if (c->v1) return LB_OK;
  LB_CHECK(lb_build_transpose(c));
  LB_CHECK(lb_alloc(c, &c->v1, (size_t)c->N));
  TWork w;
  LB_CHECK(work_t(c, &w));
  return apply_st(c, c->w, c->v1);
}

__global__ void k_a2t_final(int64_t N, const double* __restrict__ y, const double* __restrict__ b1,
                            const double* __restrict__ sd, const double* __restrict__ sp2h,
                            const double* __restrict__ v1, const double* __restrict__ partial, int npart,
                            double area, double* __restrict__ out) {
  __shared__ double eta;
  if (threadIdx.x == 0) {
    double s = 0;
    for (int k = 0; k < npart; ++k) s += partial[k];
    eta = s / area;
  }
  __syncthreads();
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = -0.25 * y[i] + b1[i] - sd[i] - sp2h[i] + eta * v1[i];
}

int lb_apply_a2t(lb_ctx* c, const double* y, double* out) {
  LB_CHECK(lb_build_transpose(c));
  LB_CHECK(ensure_v1(c));
  const int64_t N = c->N;
  TWork w;
  LB_CHECK(work_t(c, &w));
  double* a = vec_t(c, 0);    // [2][N]: D^T y, t = S^T y
  double* t2 = vec_t(c, 2);   // 2 H t
  double* o = vec_t(c, 3);    // [3][N]: S'^T t (unused), (S''+D')^T t, S'^T (2 H t)
  double* b = vec_t(c, 6);    // [2][N]: D^T a0, S^T a0 (unused)
  double* partial = vec_t(c, 12);
  CorrT c1{};
  c1.nout = 2;
  c1.kern[0] = LB_K_D; c1.dens[0] = y; c1.out[0] = a;
  c1.kern[1] = LB_K_S; c1.dens[1] = y; c1.out[1] = a + N;
  LB_CHECK(pass_t<T_DS>(c, y, nullptr, c1, a));
  k_scale_h<<<lb_div_up(N, 256), 256, 0, c->stream>>>(N, c->H, a + N, t2);
  LB_LAUNCH(c);
  CorrT c2{};
  c2.nout = 3;
  c2.kern[0] = LB_K_SP; c2.dens[0] = a + N; c2.out[0] = o;
  c2.kern[1] = LB_K_SPPDP; c2.dens[1] = a + N; c2.out[1] = o + N;
  c2.kern[2] = LB_K_SP; c2.dens[2] = t2; c2.out[2] = o + 2 * N;
  LB_CHECK(pass_t<T_P1>(c, a + N, t2, c2, o));
  CorrT c3{};
  c3.nout = 2;
  c3.kern[0] = LB_K_D; c3.dens[0] = a; c3.out[0] = b;
  c3.kern[1] = LB_K_S; c3.dens[1] = a; c3.out[1] = b + N;
  LB_CHECK(pass_t<T_DS>(c, a, nullptr, c3, b));
  k_sum_t<<<T_RB, 256, 0, c->stream>>>(N, a + N, partial);
  LB_LAUNCH(c);
  const unsigned nb = (unsigned)std::min<int64_t>(4 * c->sm_count, lb_div_up(N, 256));
  k_a2t_final<<<nb, 256, 0, c->stream>>>(N, y, b, o + N, o + 2 * N, c->v1, partial, T_RB, c->area, out);
  LB_LAUNCH(c);
  ++lb_apply64_counter;
  return LB_OK;
}

int lb_apply_st_dev(lb_ctx* c, const double* y, double* out) {
  LB_CHECK(lb_build_transpose(c));
  return apply_st(c, y, out);
}

// ---------------------------------------------------------------------------
// public entry points

static int check_adjoint(lb_ctx* c) {
  LB_CHECK(lb_require_corr(c));
  if (c->params.formulation != LB_A3 && c->params.formulation != LB_A2)
    return lb_fail(c, LB_EINVAL, "transposed applies take the A3 or A2 formulation");
  return LB_OK;
}

int lb_apply_at_op(lb_ctx* c, const double* y, double* out) {
  return c->params.formulation == LB_A2 ? lb_apply_a2t(c, y, out) : lb_apply_a3t(c, y, out);
}

extern "C" int lb_apply_St(lb_ctx* c, int nrhs, const double* y, double* out) {
  LB_CHECK(lb_require_corr(c));
  if (c->far_order) return lb_fail(c, LB_EINVAL, "transposed applies use the node rule: clear the far rule");
  if (nrhs < 1) return lb_fail(c, LB_EINVAL, "nrhs must be >= 1");
  LB_CUDA(c, cudaSetDevice(c->device));
  const int64_t N = c->N;
  const double* din;
  double* dout;
  LB_CHECK(lb_stage_in(c, y, nrhs * N * sizeof(double), c->ws_stage_in, (const void**)&din));
  LB_CHECK(lb_stage_out(c, out, nrhs * N * sizeof(double), c->ws_stage_out, (void**)&dout));
  for (int r = 0; r < nrhs; ++r) LB_CHECK(lb_apply_st_dev(c, din + (int64_t)r * N, dout + (int64_t)r * N));
  return lb_stage_out_finish(c, out, dout, nrhs * N * sizeof(double));
}

extern "C" int lb_apply_At(lb_ctx* c, int nrhs, const double* y, double* out) {
  LB_CHECK(check_adjoint(c));
  if (c->far_order) return lb_fail(c, LB_EINVAL, "transposed applies use the node rule: clear the far rule");
  if (nrhs < 1) return lb_fail(c, LB_EINVAL, "nrhs must be >= 1");
  LB_CUDA(c, cudaSetDevice(c->device));
  const int64_t N = c->N;
  const double* din;
  double* dout;
  LB_CHECK(lb_stage_in(c, y, nrhs * N * sizeof(double), c->ws_stage_in, (const void**)&din));
  LB_CHECK(lb_stage_out(c, out, nrhs * N * sizeof(double), c->ws_stage_out, (void**)&dout));
  for (int r = 0; r < nrhs; ++r) LB_CHECK(lb_apply_at_op(c, din + (int64_t)r * N, dout + (int64_t)r * N));
  return lb_stage_out_finish(c, out, dout, nrhs * N * sizeof(double));
}

// ---------------------------------------------------------------------------
// Node-position gradient of a loss of the A3 solve (float64).
//
// The positions enter A3 only through the far pair sums; the corrections, the
// near lists, w, n and H are held fixed.  With A3 sigma = P f, u = S S sigma,
// mu1 = S' sigma, mu2 = S sigma, q1 = S^T g_u and z = A3^-T S^T S^T g_u,
//   dL = g_u.dS(mu2) + q1.dS(sigma) - z.(dA3 sigma),
// and every term is a.dK(b) = sum over far pairs of a_i w_j b_j
// grad_d K(x_i, x_j).(dx_i - dx_j), d = x_i - x_j, normals fixed.  Grouped by
// (K, b) the six terms are
//   (S, sigma):  a0 = q1 + (S''+D')^T z + S'^T (2 H z) - eta S^T w,
//   (S, mu2):    a1 = g_u - eta w,
//   (S', mu1):   a2 = -z,
//   (S', sigma): a3 = -S'^T z,
//   (S', mu2):   a4 = 2 H z,
//   (S''+D', mu2): a5 = z,
// eta = sum z / |Gamma|, and grad_i = sum_m a_m,i T_m,i - b_m,i U_m,i with the
// forward sums T_m,i = sum_j w_j b_m,j grad K_m(x_i, x_j) and the transposed
// sums U_m,j = w_j sum_i a_m,i grad K_m(x_i, x_j).  The kernels' gradients in
// d, with a = n_i.d, e = n_i - n_j, b = e.d and 1/(4 pi) applied at the end:
//   grad S      = -d / r^3,
//   grad S'     = -n_i / r^3 + 3 a d / r^5,
//   grad S''+D' = [3 (b n_i + a e) / r^2 - 6 a b d / r^4] / r^3
//                 - 3 (3 a b / r^2 - |e|^2 / 2) d / r^5.
#define GR_NTH 128
#define GR_NO 18  // six (kernel, density) sums x three components

__device__ __forceinline__ void grad_kernels(const double* d, const double* ni, const double* nj, double rinv,
                                             double* gS, double* gSp, double* gSD) {
  const double rinv2 = rinv * rinv, rinv3 = rinv2 * rinv, rinv5 = rinv3 * rinv2;
  const double a = ni[0] * d[0] + ni[1] * d[1] + ni[2] * d[2];
  const double e[3] = {ni[0] - nj[0], ni[1] - nj[1], ni[2] - nj[2]};
  const double b = e[0] * d[0] + e[1] * d[1] + e[2] * d[2];
  const double e2 = e[0] * e[0] + e[1] * e[1] + e[2] * e[2];
  const double c1 = 3.0 * rinv5;
  const double c2 = 6.0 * a * b * rinv2 * rinv5 + 3.0 * (3.0 * a * b * rinv2 - 0.5 * e2) * rinv5;
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    gS[k] = -d[k] * rinv3;
    gSp[k] = -ni[k] * rinv3 + 3.0 * a * d[k] * rinv5;
    gSD[k] = c1 * (b * ni[k] + a * e[k]) - c2 * d[k];
  }
}

// forward sums: targets i, sources j with patch(j) not in Near(i).
// Q [Npad][3] = w (sigma, mu1, mu2); part [split][18][N]
__global__ void __launch_bounds__(GR_NTH) k_grad_fwd(int64_t N, int np, const double4_32a* __restrict__ pos,
                                                     const double4_32a* __restrict__ nrm, const double* __restrict__ Q,
                                                     const uint8_t* __restrict__ flags, int64_t ntiles,
                                                     const int64_t* __restrict__ row_ptr,
                                                     const int32_t* __restrict__ near_patch, int tiles_per_split,
                                                     double* __restrict__ part) {
  __shared__ double4_32a sP[TT_TS], sN[TT_TS];
  __shared__ double sQ[TT_TS][3];
  __shared__ int sLp[TT_TS];
  const int64_t t = (int64_t)blockIdx.x * GR_NTH + threadIdx.x;  // < Npad
  const double4_32a p = pos[t], n = nrm[t];
  const double xi[3] = {p.x, p.y, p.z}, ni[3] = {n.x, n.y, n.z};
  double acc[GR_NO];
#pragma unroll
  for (int o = 0; o < GR_NO; ++o) acc[o] = 0.0;
  const int64_t tile_b = (int64_t)blockIdx.y * tiles_per_split;
  const int64_t tile_e = min(ntiles, tile_b + tiles_per_split);
  for (int64_t tile = tile_b; tile < tile_e; ++tile) {
    const int64_t s0 = tile * TT_TS;
    const int64_t P0 = s0 / np;
    for (int s = threadIdx.x; s < TT_TS; s += GR_NTH) {
      sP[s] = pos[s0 + s];
      sN[s] = nrm[s0 + s];
#pragma unroll
      for (int k = 0; k < 3; ++k) sQ[s][k] = Q[(s0 + s) * 3 + k];
      sLp[s] = (int)((s0 + s) / np - P0);  // < 64: a tile spans at most 64 patches
    }
    __syncthreads();
    // bit L: patch P0 + L is in Near(t)
    unsigned long long m = 0ull;
    if (flags[(int64_t)blockIdx.x * ntiles + tile] != 0 && t < N)
      for (int64_t bb = row_ptr[t]; bb < row_ptr[t + 1]; ++bb) {
        const int64_t dd = (int64_t)near_patch[bb] - P0;
        if (dd >= 0 && dd < 64) m |= 1ull << dd;
      }
    for (int s = 0; s < TT_TS; ++s) {
      const double4_32a a = sP[s], b = sN[s];
      const double d[3] = {xi[0] - a.x, xi[1] - a.y, xi[2] - a.z};
      const double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
      const bool masked = ((m >> sLp[s]) & 1ull) || t >= N;
      const double rinv = masked ? 0.0 : rsqrt(r2);
      const double nj[3] = {b.x, b.y, b.z};
      double gS[3], gSp[3], gSD[3];
      grad_kernels(d, ni, nj, rinv, gS, gSp, gSD);
      const double qs = sQ[s][0], q1 = sQ[s][1], q2 = sQ[s][2];
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        acc[k] += qs * gS[k];
        acc[3 + k] += q2 * gS[k];
        acc[6 + k] += q1 * gSp[k];
        acc[9 + k] += qs * gSp[k];
        acc[12 + k] += q2 * gSp[k];
        acc[15 + k] += q2 * gSD[k];
      }
    }
    __syncthreads();
  }
  if (t >= N) return;
#pragma unroll
  for (int o = 0; o < GR_NO; ++o) part[((int64_t)blockIdx.y * GR_NO + o) * N + t] = acc[o];
}

// transposed sums: outputs j, sources i with patch(j) not in Near(i).
// A [Npad][6] = (a0 .. a5) at the sources; part [split][18][N]
__global__ void __launch_bounds__(GR_NTH) k_grad_tr(int64_t N, int np, const double4_32a* __restrict__ pos,
                                                    const double4_32a* __restrict__ nrm, const double* __restrict__ A,
                                                    const uint8_t* __restrict__ tflag,
                                                    const unsigned long long* __restrict__ tmask, int64_t ntiles,
                                                    int tiles_per_split, double* __restrict__ part) {
  __shared__ double4_32a sP[TT_TS], sN[TT_TS];
  __shared__ double sA[TT_TS][6];
  const int64_t t = (int64_t)blockIdx.x * GR_NTH + threadIdx.x;  // < Npad
  const double4_32a p = pos[t], n = nrm[t];
  const double xj[3] = {p.x, p.y, p.z}, nj[3] = {n.x, n.y, n.z};
  const int64_t pj = t < N ? t / np : -1;
  double acc[GR_NO];
#pragma unroll
  for (int o = 0; o < GR_NO; ++o) acc[o] = 0.0;
  const int64_t tile_b = (int64_t)blockIdx.y * tiles_per_split;
  const int64_t tile_e = min(ntiles, tile_b + tiles_per_split);
  for (int64_t tile = tile_b; tile < tile_e; ++tile) {
    const int64_t s0 = tile * TT_TS;
    for (int s = threadIdx.x; s < TT_TS; s += GR_NTH) {
      sP[s] = pos[s0 + s];
      sN[s] = nrm[s0 + s];
#pragma unroll
      for (int k = 0; k < 6; ++k) sA[s][k] = A[(s0 + s) * 6 + k];
    }
    __syncthreads();
    // the flag table is per block of TT_TB outputs, which holds this block's GR_NTH
    const bool any = tflag[((int64_t)blockIdx.x * GR_NTH / TT_TB) * ntiles + tile] != 0;
    const unsigned long long m = (any && pj >= 0) ? tmask[pj * ntiles + tile] : 0ull;
    for (int s = 0; s < TT_TS; ++s) {
      const double4_32a a = sP[s], b = sN[s];
      const double d[3] = {a.x - xj[0], a.y - xj[1], a.z - xj[2]};  // x_i - x_j
      const double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
      const bool masked = ((m >> s) & 1ull) || pj < 0;
      const double rinv = masked ? 0.0 : rsqrt(r2);
      const double ni[3] = {b.x, b.y, b.z};
      double gS[3], gSp[3], gSD[3];
      grad_kernels(d, ni, nj, rinv, gS, gSp, gSD);
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        acc[k] += sA[s][0] * gS[k];
        acc[3 + k] += sA[s][1] * gS[k];
        acc[6 + k] += sA[s][2] * gSp[k];
        acc[9 + k] += sA[s][3] * gSp[k];
        acc[12 + k] += sA[s][4] * gSp[k];
        acc[15 + k] += sA[s][5] * gSD[k];
      }
    }
    __syncthreads();
  }
  if (t >= N) return;
#pragma unroll
  for (int o = 0; o < GR_NO; ++o) part[((int64_t)blockIdx.y * GR_NO + o) * N + t] = acc[o];
}

// out[o][j] = scale_j / (4 pi) sum_s part[s][o][j], scale = w_j or 1
__global__ void k_reduce_g(int64_t N, int nsplit, const double* __restrict__ part, const double* __restrict__ w,
                           double* __restrict__ out) {
  const int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (j >= N) return;
  const double sc = (w ? w[j] : 1.0) * LB_INV4PI;
  for (int o = 0; o < GR_NO; ++o) {
    double s = 0;
    for (int k = 0; k < nsplit; ++k) s += part[((int64_t)k * GR_NO + o) * N + j];
    out[(int64_t)o * N + j] = s * sc;
  }
}

struct GradVecs {
  const double* v[6];
};

// out[i][k] = scale_i v_k[i] for i < N, 0 in the padding
__global__ void k_pack_g(int64_t N, int64_t Npad, int nv, const double* __restrict__ scale, GradVecs gv,
                         double* __restrict__ out) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= Npad) return;
  for (int k = 0; k < nv; ++k) out[i * nv + k] = i < N ? (scale ? scale[i] : 1.0) * gv.v[k][i] : 0.0;
}

// a vectors of the six terms; eta = sum z / area from per-block partials
__global__ void k_grad_avec(int64_t N, const double* __restrict__ gu, const double* __restrict__ q1,
                            const double* __restrict__ z, const double* __restrict__ h2z,
                            const double* __restrict__ tp, const double* __restrict__ v1,
                            const double* __restrict__ w, const double* __restrict__ partial, int npart, double area,
                            double* __restrict__ a) {
  __shared__ double eta;
  if (threadIdx.x == 0) {
    double s = 0;
    for (int k = 0; k < npart; ++k) s += partial[k];
    eta = s / area;
  }
  __syncthreads();
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
    a[i] = q1[i] + tp[N + i] + tp[2 * N + i] - eta * v1[i];
    a[N + i] = gu[i] - eta * w[i];
    a[2 * N + i] = -z[i];
    a[3 * N + i] = -tp[i];
  }
}

struct GradB {
  const double* a[6];
  const double* b[6];
};

// grad[i][k] = sum_m a_m[i] T[m][k][i] - b_m[i] U[m][k][i]
__global__ void k_grad_combine(int64_t N, GradB ab, const double* __restrict__ T, const double* __restrict__ U,
                               double* __restrict__ grad) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= N) return;
  double g[3] = {0, 0, 0};
#pragma unroll
  for (int m = 0; m < 6; ++m) {
    const double am = ab.a[m][i], bm = ab.b[m][i];
#pragma unroll
    for (int k = 0; k < 3; ++k) g[k] += am * T[(int64_t)(3 * m + k) * N + i] - bm * U[(int64_t)(3 * m + k) * N + i];
  }
#pragma unroll
  for (int k = 0; k < 3; ++k) grad[i * 3 + k] = g[k];
}

int lb_shape_grad_pairs(lb_ctx* c, const double* gu, const double* sg, const double* mu1, const double* mu2,
                        const double* q1, const double* z, double* grad) {
  LB_CHECK(lb_build_transpose(c));
  LB_CHECK(ensure_v1(c));
  const int64_t N = c->N, Npad = c->Npad;
  MaskTable* mt = nullptr;
  LB_CHECK(lb_get_mask(c, GR_NTH, TT_TS, &mt));
  const uint8_t* fflags = mt->flags;
  const int64_t ntb = (N + GR_NTH - 1) / GR_NTH, ntiles = Npad / TT_TS;
  if (mt->ntb != ntb || mt->ntiles != ntiles || c->t_ntiles != ntiles)
    return lb_fail(c, LB_EINVAL, "gradient tile tables disagree");
  const int64_t want = 6LL * c->sm_count;
  int64_t nsplit = std::max<int64_t>(1, std::min<int64_t>({ntiles, (want + ntb - 1) / ntb, (int64_t)32}));
  const int tps = (int)((ntiles + nsplit - 1) / nsplit);
  nsplit = (ntiles + tps - 1) / tps;
  // vectors: h2z, tp [3], a0..a3 [4], T [18], U [18], partial; scratch: packed [Npad][6], part
  const size_t nvec = (size_t)(1 + 3 + 4 + 2 * GR_NO) * N + T_RB;
  LB_CHECK(lb_ensure(c, c->ws_grad, (nvec + (size_t)Npad * 6 + (size_t)nsplit * GR_NO * N) * sizeof(double)));
  double* h2z = (double*)c->ws_grad.p;
  double* tp = h2z + N;
  double* av = tp + 3 * N;
  double* T = av + 4 * N;
  double* U = T + GR_NO * N;
  double* partial = U + GR_NO * N;
  double* packed = partial + T_RB;
  double* part = packed + Npad * 6;
  const unsigned nb = (unsigned)std::min<int64_t>(4 * c->sm_count, lb_div_up(N, 256));
  k_scale_h<<<lb_div_up(N, 256), 256, 0, c->stream>>>(N, c->H, z, h2z);
  LB_LAUNCH(c);
  // S'^T z, (S''+D')^T z, S'^T (2 H z)
  CorrT c1{};
  c1.nout = 3;
  c1.kern[0] = LB_K_SP; c1.dens[0] = z; c1.out[0] = tp;
  c1.kern[1] = LB_K_SPPDP; c1.dens[1] = z; c1.out[1] = tp + N;
  c1.kern[2] = LB_K_SP; c1.dens[2] = h2z; c1.out[2] = tp + 2 * N;
  LB_CHECK(pass_t<T_P1>(c, z, h2z, c1, tp));
  k_sum_t<<<T_RB, 256, 0, c->stream>>>(N, z, partial);
  LB_LAUNCH(c);
  k_grad_avec<<<nb, 256, 0, c->stream>>>(N, gu, q1, z, h2z, tp, c->v1, c->w, partial, T_RB, c->area, av);
  LB_LAUNCH(c);
  GradB ab{};
  const double* avs[6] = {av, av + N, av + 2 * N, av + 3 * N, h2z, z};
  const double* bvs[6] = {sg, mu2, mu1, sg, mu2, mu2};
  for (int m = 0; m < 6; ++m) {
    ab.a[m] = avs[m];
    ab.b[m] = bvs[m];
  }
  // forward sums of w (sigma, mu1, mu2)
  GradVecs gf{};
  gf.v[0] = sg; gf.v[1] = mu1; gf.v[2] = mu2;
  k_pack_g<<<lb_div_up(Npad, 256), 256, 0, c->stream>>>(N, Npad, 3, c->w, gf, packed);
  LB_LAUNCH(c);
  {
    ProfScope prof(c, LB_PROF_SHAPE, N * N);
    k_grad_fwd<<<dim3((unsigned)ntb, (unsigned)nsplit), GR_NTH, 0, c->stream>>>(
        N, c->np, c->pos64, c->nrm64, packed, fflags, ntiles, c->row_ptr, c->near_patch, tps, part);
    LB_LAUNCH(c);
  }
  lb_pair_counter += N * N;
  k_reduce_g<<<lb_div_up(N, 256), 256, 0, c->stream>>>(N, (int)nsplit, part, nullptr, T);
  LB_LAUNCH(c);
  // transposed sums of a0 .. a5
  GradVecs gt{};
  for (int m = 0; m < 6; ++m) gt.v[m] = avs[m];
  k_pack_g<<<lb_div_up(Npad, 256), 256, 0, c->stream>>>(N, Npad, 6, nullptr, gt, packed);
  LB_LAUNCH(c);
  {
    ProfScope prof(c, LB_PROF_SHAPE, N * N);
    k_grad_tr<<<dim3((unsigned)ntb, (unsigned)nsplit), GR_NTH, 0, c->stream>>>(
        N, c->np, c->pos64, c->nrm64, packed, c->tflag, c->tmask, ntiles, tps, part);
    LB_LAUNCH(c);
  }
  lb_pair_counter += N * N;
  k_reduce_g<<<lb_div_up(N, 256), 256, 0, c->stream>>>(N, (int)nsplit, part, c->w, U);
  LB_LAUNCH(c);
  k_grad_combine<<<lb_div_up(N, 256), 256, 0, c->stream>>>(N, ab, T, U, grad);
  LB_LAUNCH(c);
  return LB_OK;
}

// ---------------------------------------------------------------------------
// Gradient with respect to the chart tangents X_u, X_v (not in the paper).
// Input model: X, X_u, X_v are the upload's independent inputs; the
// correction blocks and the near lists are held fixed.  X_u, X_v enter A3
// through the unit normals n = X_u x X_v / |X_u x X_v| (target normal of S'
// and S''+D', source normal of S''+D'), the weights w = w_ref |X_u x X_v|
// (every far sum, the mean W, the projection P f = f - W f) and the mean
// curvature H = -1/2 tr(g^-1 L), L_ab = X_ab . n, X_uu = D_u X_u,
// X_vv = D_v X_v, X_uv = (D_v X_u + D_u X_v)/2 (Section 2).  With the six
// bilinear terms a_m . K_m b_m of the node-position gradient (same a_m, b_m):
//   dL/dw_j = sum_m b_m,j U_m,j - eta_z [(S mu2)_j - W S mu2 + (P f)_j],
//     U_m,j = sum_{i far} a_m,i K_m(x_i, x_j),  eta_z = sum z / |Gamma|;
//   dL/dn_i = a_2,i V1_i + a_3,i V2_i + a_4,i V3_i + z_i V4_i,
//     V1, V2, V3 = sum_{j far} w_j (mu1, sigma, mu2)_j dS'/dn_x,
//     V4 = sum_{j far} w_j mu2_j d(S''+D')/dn_x;
//   dL/dn_j += w_j mu2_j sum_{i far} z_i d(S''+D')/dn_y;
//   dL/dH_i = 2 z_i (S' mu2)_i;
// then the chain rule through n, |X_u x X_v| and H.  With a = n_x.d,
// e = n_x - n_y, b = e.d (d = x_i - x_j, 1/(4 pi) applied at the end):
//   dS'/dn_x = -d / r^3,
//   d(S''+D')/dn_x = [3 (a + b) d / r^2 - e] / r^3,
//   d(S''+D')/dn_y = [-3 a d / r^2 + e] / r^3.
#define TG_NF 12  // forward: V1 .. V4, three components each
#define TG_NT 9   // transposed: U_0 .. U_5, then the source-normal vector

// forward sums: Q [Npad][3] = w (sigma, mu1, mu2); part [split][12][N]
__global__ void __launch_bounds__(GR_NTH) k_tan_fwd(int64_t N, int np, const double4_32a* __restrict__ pos,
                                                    const double4_32a* __restrict__ nrm, const double* __restrict__ Q,
                                                    const uint8_t* __restrict__ flags, int64_t ntiles,
                                                    const int64_t* __restrict__ row_ptr,
                                                    const int32_t* __restrict__ near_patch, int tiles_per_split,
                                                    double* __restrict__ part) {
  __shared__ double4_32a sP[TT_TS], sN[TT_TS];
  __shared__ double sQ[TT_TS][3];
  __shared__ int sLp[TT_TS];
  const int64_t t = (int64_t)blockIdx.x * GR_NTH + threadIdx.x;  // < Npad
  const double4_32a p = pos[t], n = nrm[t];
  const double xi[3] = {p.x, p.y, p.z}, ni[3] = {n.x, n.y, n.z};
  double acc[TG_NF];
#pragma unroll
  for (int o = 0; o < TG_NF; ++o) acc[o] = 0.0;
  const int64_t tile_b = (int64_t)blockIdx.y * tiles_per_split;
  const int64_t tile_e = min(ntiles, tile_b + tiles_per_split);
  for (int64_t tile = tile_b; tile < tile_e; ++tile) {
    const int64_t s0 = tile * TT_TS;
    const int64_t P0 = s0 / np;
    for (int s = threadIdx.x; s < TT_TS; s += GR_NTH) {
      sP[s] = pos[s0 + s];
      sN[s] = nrm[s0 + s];
#pragma unroll
      for (int k = 0; k < 3; ++k) sQ[s][k] = Q[(s0 + s) * 3 + k];
      sLp[s] = (int)((s0 + s) / np - P0);
    }
    __syncthreads();
    unsigned long long m = 0ull;
    if (flags[(int64_t)blockIdx.x * ntiles + tile] != 0 && t < N)
      for (int64_t bb = row_ptr[t]; bb < row_ptr[t + 1]; ++bb) {
        const int64_t dd = (int64_t)near_patch[bb] - P0;
        if (dd >= 0 && dd < 64) m |= 1ull << dd;
      }
    for (int s = 0; s < TT_TS; ++s) {
      const double4_32a a4 = sP[s], b4 = sN[s];
      const double d[3] = {xi[0] - a4.x, xi[1] - a4.y, xi[2] - a4.z};
      const double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
      const bool masked = ((m >> sLp[s]) & 1ull) || t >= N;
      const double rinv = masked ? 0.0 : rsqrt(r2);
      const double rinv2 = rinv * rinv, rinv3 = rinv2 * rinv;
      const double e[3] = {ni[0] - b4.x, ni[1] - b4.y, ni[2] - b4.z};
      const double a = ni[0] * d[0] + ni[1] * d[1] + ni[2] * d[2];
      const double b = e[0] * d[0] + e[1] * d[1] + e[2] * d[2];
      const double cd = 3.0 * (a + b) * rinv2 * rinv3;
      const double qs = sQ[s][0], q1 = sQ[s][1], q2 = sQ[s][2];
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        const double gp = -d[k] * rinv3;                     // dS'/dn_x
        const double gx = cd * d[k] - e[k] * rinv3;          // d(S''+D')/dn_x
        acc[k] += q1 * gp;
        acc[3 + k] += qs * gp;
        acc[6 + k] += q2 * gp;
        acc[9 + k] += q2 * gx;
      }
    }
    __syncthreads();
  }
  if (t >= N) return;
#pragma unroll
  for (int o = 0; o < TG_NF; ++o) part[((int64_t)blockIdx.y * TG_NF + o) * N + t] = acc[o];
}

// transposed sums: outputs j, sources i with patch(j) not in Near(i).
// A [Npad][6] = (a0 .. a5) at the sources; part [split][9][N]
__global__ void __launch_bounds__(GR_NTH) k_tan_tr(int64_t N, int np, const double4_32a* __restrict__ pos,
                                                   const double4_32a* __restrict__ nrm, const double* __restrict__ A,
                                                   const uint8_t* __restrict__ tflag,
                                                   const unsigned long long* __restrict__ tmask, int64_t ntiles,
                                                   int tiles_per_split, double* __restrict__ part) {
  __shared__ double4_32a sP[TT_TS], sN[TT_TS];
  __shared__ double sA[TT_TS][6];
  const int64_t t = (int64_t)blockIdx.x * GR_NTH + threadIdx.x;  // < Npad
  const double4_32a p = pos[t], n = nrm[t];
  const double xj[3] = {p.x, p.y, p.z}, nj[3] = {n.x, n.y, n.z};
  const int64_t pj = t < N ? t / np : -1;
  double acc[TG_NT];
#pragma unroll
  for (int o = 0; o < TG_NT; ++o) acc[o] = 0.0;
  const int64_t tile_b = (int64_t)blockIdx.y * tiles_per_split;
  const int64_t tile_e = min(ntiles, tile_b + tiles_per_split);
  for (int64_t tile = tile_b; tile < tile_e; ++tile) {
    const int64_t s0 = tile * TT_TS;
    for (int s = threadIdx.x; s < TT_TS; s += GR_NTH) {
      sP[s] = pos[s0 + s];
      sN[s] = nrm[s0 + s];
#pragma unroll
      for (int k = 0; k < 6; ++k) sA[s][k] = A[(s0 + s) * 6 + k];
    }
    __syncthreads();
    const bool any = tflag[((int64_t)blockIdx.x * GR_NTH / TT_TB) * ntiles + tile] != 0;
    const unsigned long long m = (any && pj >= 0) ? tmask[pj * ntiles + tile] : 0ull;
    for (int s = 0; s < TT_TS; ++s) {
      const double4_32a a4 = sP[s], b4 = sN[s];
      const double d[3] = {a4.x - xj[0], a4.y - xj[1], a4.z - xj[2]};  // x_i - x_j
      const double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
      const bool masked = ((m >> s) & 1ull) || pj < 0;
      const double rinv = masked ? 0.0 : rsqrt(r2);
      const double rinv2 = rinv * rinv, rinv3 = rinv2 * rinv;
      const double ni[3] = {b4.x, b4.y, b4.z};
      const double e[3] = {ni[0] - nj[0], ni[1] - nj[1], ni[2] - nj[2]};
      const double a = ni[0] * d[0] + ni[1] * d[1] + ni[2] * d[2];
      const double b = e[0] * d[0] + e[1] * d[1] + e[2] * d[2];
      const double e2 = e[0] * e[0] + e[1] * e[1] + e[2] * e[2];
      const double kS = rinv, kSp = -a * rinv3, kSD = (3.0 * a * b * rinv2 - 0.5 * e2) * rinv3;
      acc[0] += sA[s][0] * kS;
      acc[1] += sA[s][1] * kS;
      acc[2] += sA[s][2] * kSp;
      acc[3] += sA[s][3] * kSp;
      acc[4] += sA[s][4] * kSp;
      acc[5] += sA[s][5] * kSD;
      const double ca = -3.0 * a * rinv2 * rinv3 * sA[s][5];
#pragma unroll
      for (int k = 0; k < 3; ++k) acc[6 + k] += ca * d[k] + sA[s][5] * e[k] * rinv3;  // d(S''+D')/dn_y
    }
    __syncthreads();
  }
  if (t >= N) return;
#pragma unroll
  for (int o = 0; o < TG_NT; ++o) part[((int64_t)blockIdx.y * TG_NT + o) * N + t] = acc[o];
}

// out[o][j] = 1/(4 pi) sum_s part[s][o][j]
__global__ void k_reduce_tg(int64_t N, int nsplit, int nout, const double* __restrict__ part,
                            double* __restrict__ out) {
  const int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (j >= N) return;
  for (int o = 0; o < nout; ++o) {
    double s = 0;
    for (int k = 0; k < nsplit; ++k) s += part[((int64_t)k * nout + o) * N + j];
    out[(int64_t)o * N + j] = s * LB_INV4PI;
  }
}

struct TanIn {
  const double *a[6], *b[6];   // the bilinear terms
  const double* V;             // [12][N] forward sums
  const double* U;             // [9][N] transposed sums
  const double* z;             // adjoint solution
  const double* mu2;
  const double* Smu2;          // S mu2 (far + near)
  const double* Spmu2;         // S' mu2 (far + near)
  const double* pf;            // P f
  const double* partial;       // [3][nblk] partial sums: z, w S mu2 (the weighted mean)
  int npart;
};

// per node: dL/dn, dL/dw, dL/dH -> the local parts of dL/dX_u, dL/dX_v and
// the vectors gXuu, gXvv, gXuv that the patch differentiation distributes
__global__ void k_tan_local(int64_t N, int np, TanIn in, const double* __restrict__ Xu, const double* __restrict__ Xv,
                            const double* __restrict__ nrm, const double* __restrict__ w,
                            const double* __restrict__ Jn, const double* __restrict__ ginv,
                            const double* __restrict__ ref, const double* __restrict__ Du,
                            const double* __restrict__ Dv, double area, double* __restrict__ gXu,
                            double* __restrict__ gXv, double* __restrict__ g2) {
  __shared__ double eta_z, eta;
  if (threadIdx.x == 0) {
    double s0 = 0, s1 = 0;
    for (int k = 0; k < in.npart; ++k) {
      s0 += in.partial[k];
      s1 += in.partial[in.npart + k];
    }
    eta_z = s0 / area;
    eta = s1 / area;
  }
  __syncthreads();
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= N) return;
  const int64_t P = i / np;
  const int q = (int)(i - P * np);
  // weights
  double gw = -eta_z * (in.Smu2[i] - eta + in.pf[i]);
#pragma unroll
  for (int m = 0; m < 6; ++m) gw += in.b[m][i] * in.U[(int64_t)m * N + i];
  // normals
  double gn[3];
#pragma unroll
  for (int k = 0; k < 3; ++k)
    gn[k] = in.a[2][i] * in.V[(int64_t)k * N + i] + in.a[3][i] * in.V[(int64_t)(3 + k) * N + i] +
            in.a[4][i] * in.V[(int64_t)(6 + k) * N + i] + in.z[i] * in.V[(int64_t)(9 + k) * N + i] +
            w[i] * in.mu2[i] * in.U[(int64_t)(6 + k) * N + i];
  // curvature
  const double gH = 2.0 * in.z[i] * in.Spmu2[i];
  const double* xu = Xu + 3 * i;
  const double* xv = Xv + 3 * i;
  const double n[3] = {nrm[3 * i], nrm[3 * i + 1], nrm[3 * i + 2]};
  double xuu[3] = {0, 0, 0}, xvv[3] = {0, 0, 0}, xuv[3] = {0, 0, 0};
  for (int bq = 0; bq < np; ++bq) {
    const double du = Du[q * np + bq], dv = Dv[q * np + bq];
    const double* pu = Xu + 3 * (P * np + bq);
    const double* pv = Xv + 3 * (P * np + bq);
    for (int k = 0; k < 3; ++k) {
      xuu[k] += du * pu[k];
      xvv[k] += dv * pv[k];
      xuv[k] += 0.5 * (dv * pu[k] + du * pv[k]);
    }
  }
  const double G11 = ginv[3 * i], G12 = ginv[3 * i + 1], G22 = ginv[3 * i + 2];
  const double L11 = xuu[0] * n[0] + xuu[1] * n[1] + xuu[2] * n[2];
  const double L12 = xuv[0] * n[0] + xuv[1] * n[1] + xuv[2] * n[2];
  const double L22 = xvv[0] * n[0] + xvv[1] * n[1] + xvv[2] * n[2];
  // M = 1/2 G L G (symmetric)
  const double GL11 = G11 * L11 + G12 * L12, GL12 = G11 * L12 + G12 * L22;
  const double GL21 = G12 * L11 + G22 * L12, GL22 = G12 * L12 + G22 * L22;
  const double M11 = 0.5 * (GL11 * G11 + GL12 * G12);
  const double M12 = 0.5 * (GL11 * G12 + GL12 * G22);
  const double M22 = 0.5 * (GL21 * G12 + GL22 * G22);
  double gu_[3], gv_[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    gn[k] += -0.5 * gH * (G11 * xuu[k] + 2.0 * G12 * xuv[k] + G22 * xvv[k]);
    g2[(int64_t)k * N + i] = -0.5 * gH * G11 * n[k];        // dL/dX_uu
    g2[(int64_t)(3 + k) * N + i] = -0.5 * gH * G22 * n[k];  // dL/dX_vv
    g2[(int64_t)(6 + k) * N + i] = -gH * G12 * n[k];        // dL/dX_uv
    gu_[k] = gH * (2.0 * M11 * xu[k] + 2.0 * M12 * xv[k]);
    gv_[k] = gH * (2.0 * M22 * xv[k] + 2.0 * M12 * xu[k]);
  }
  // n = c / |c|, w = w_ref |c|, c = X_u x X_v
  const double gJ = ref[3 * q + 2] * gw;
  const double ng = n[0] * gn[0] + n[1] * gn[1] + n[2] * gn[2];
  const double iJ = 1.0 / Jn[i];
  double gc[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) gc[k] = (gn[k] - ng * n[k]) * iJ + gJ * n[k];
  gu_[0] += xv[1] * gc[2] - xv[2] * gc[1];
  gu_[1] += xv[2] * gc[0] - xv[0] * gc[2];
  gu_[2] += xv[0] * gc[1] - xv[1] * gc[0];
  gv_[0] += gc[1] * xu[2] - gc[2] * xu[1];
  gv_[1] += gc[2] * xu[0] - gc[0] * xu[2];
  gv_[2] += gc[0] * xu[1] - gc[1] * xu[0];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    gXu[3 * i + k] = gu_[k];
    gXv[3 * i + k] = gv_[k];
  }
}

// patch differentiation transposed: gX_u[P,q] += sum_i Du[i][q] gXuu[P,i] + 1/2 Dv[i][q] gXuv[P,i],
// gX_v[P,q] += sum_i Dv[i][q] gXvv[P,i] + 1/2 Du[i][q] gXuv[P,i]
__global__ void k_tan_diff(int64_t N, int np, const double* __restrict__ Du, const double* __restrict__ Dv,
                           const double* __restrict__ g2, double* __restrict__ gXu, double* __restrict__ gXv) {
  const int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (j >= N) return;
  const int64_t P = j / np;
  const int q = (int)(j - P * np);
  double su[3] = {0, 0, 0}, sv[3] = {0, 0, 0};
  for (int ii = 0; ii < np; ++ii) {
    const int64_t i = P * np + ii;
    const double du = Du[ii * np + q], dv = Dv[ii * np + q];
    for (int k = 0; k < 3; ++k) {
      const double uu = g2[(int64_t)k * N + i], vv = g2[(int64_t)(3 + k) * N + i], uv = g2[(int64_t)(6 + k) * N + i];
      su[k] += du * uu + 0.5 * dv * uv;
      sv[k] += dv * vv + 0.5 * du * uv;
    }
  }
  for (int k = 0; k < 3; ++k) {
    gXu[3 * j + k] += su[k];
    gXv[3 * j + k] += sv[k];
  }
}

// partials of sum z (first row) and sum w S mu2 (second row)
__global__ void k_tan_sums(int64_t N, const double* __restrict__ z, const double* __restrict__ w,
                           const double* __restrict__ s, double* __restrict__ partial) {
  __shared__ double sh[2][256];
  double a = 0, b = 0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
    a += z[i];
    b += w[i] * s[i];
  }
  sh[0][threadIdx.x] = a;
  sh[1][threadIdx.x] = b;
  __syncthreads();
  for (int k = blockDim.x / 2; k > 0; k >>= 1) {
    if (threadIdx.x < k) {
      sh[0][threadIdx.x] += sh[0][threadIdx.x + k];
      sh[1][threadIdx.x] += sh[1][threadIdx.x + k];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    partial[blockIdx.x] = sh[0][0];
    partial[gridDim.x + blockIdx.x] = sh[1][0];
  }
}

int lb_tangent_grad_pairs(lb_ctx* c, const double* gu, const double* pf, const double* sg, const double* mu1,
                          const double* mu2, const double* q1, const double* z, double* gXu, double* gXv) {
  LB_CHECK(lb_build_transpose(c));
  LB_CHECK(ensure_v1(c));
  const int64_t N = c->N, Npad = c->Npad;
  MaskTable* mt = nullptr;
  LB_CHECK(lb_get_mask(c, GR_NTH, TT_TS, &mt));
  const int64_t ntb = (N + GR_NTH - 1) / GR_NTH, ntiles = Npad / TT_TS;
  if (mt->ntb != ntb || mt->ntiles != ntiles || c->t_ntiles != ntiles)
    return lb_fail(c, LB_EINVAL, "gradient tile tables disagree");
  const int64_t want = 6LL * c->sm_count;
  int64_t nsplit = std::max<int64_t>(1, std::min<int64_t>({ntiles, (want + ntb - 1) / ntb, (int64_t)32}));
  const int tps = (int)((ntiles + nsplit - 1) / nsplit);
  nsplit = (ntiles + tps - 1) / tps;
  // vectors: h2z, tp [3], a0..a3 [4], V [12], U [9], pot2 [4], g2 [9], partial [2 T_RB];
  // scratch: packed [Npad][6], part [nsplit][12][N]
  const size_t nvec = (size_t)(1 + 3 + 4 + TG_NF + TG_NT + 4 + 9) * N + 2 * T_RB;
  LB_CHECK(lb_ensure(c, c->ws_grad, (nvec + (size_t)Npad * 6 + (size_t)nsplit * TG_NF * N) * sizeof(double)));
  double* h2z = (double*)c->ws_grad.p;
  double* tp = h2z + N;
  double* av = tp + 3 * N;
  double* V = av + 4 * N;
  double* U = V + TG_NF * N;
  double* pot2 = U + TG_NT * N;
  double* g2 = pot2 + 4 * N;
  double* partial = g2 + 9 * N;
  double* packed = partial + 2 * T_RB;
  double* part = packed + Npad * 6;
  const unsigned nb = (unsigned)std::min<int64_t>(4 * c->sm_count, lb_div_up(N, 256));
  k_scale_h<<<lb_div_up(N, 256), 256, 0, c->stream>>>(N, c->H, z, h2z);
  LB_LAUNCH(c);
  CorrT c1{};
  c1.nout = 3;
  c1.kern[0] = LB_K_SP; c1.dens[0] = z; c1.out[0] = tp;
  c1.kern[1] = LB_K_SPPDP; c1.dens[1] = z; c1.out[1] = tp + N;
  c1.kern[2] = LB_K_SP; c1.dens[2] = h2z; c1.out[2] = tp + 2 * N;
  LB_CHECK(pass_t<T_P1>(c, z, h2z, c1, tp));
  k_sum_t<<<T_RB, 256, 0, c->stream>>>(N, z, partial);
  LB_LAUNCH(c);
  k_grad_avec<<<nb, 256, 0, c->stream>>>(N, gu, q1, z, h2z, tp, c->v1, c->w, partial, T_RB, c->area, av);
  LB_LAUNCH(c);
  const double* avs[6] = {av, av + N, av + 2 * N, av + 3 * N, h2z, z};
  const double* bvs[6] = {sg, mu2, mu1, sg, mu2, mu2};
  // S mu2 and S' mu2 (far + near), and the sums giving eta_z and W S mu2
  LB_CHECK(lb_potentials(c, LB_FP64, mu2, pot2, (1u << LB_K_S) | (1u << LB_K_SP)));
  k_tan_sums<<<T_RB, 256, 0, c->stream>>>(N, z, c->w, pot2 + (int64_t)LB_K_S * N, partial);
  LB_LAUNCH(c);
  // forward sums of w (sigma, mu1, mu2)
  GradVecs gf{};
  gf.v[0] = sg; gf.v[1] = mu1; gf.v[2] = mu2;
  k_pack_g<<<lb_div_up(Npad, 256), 256, 0, c->stream>>>(N, Npad, 3, c->w, gf, packed);
  LB_LAUNCH(c);
  {
    ProfScope prof(c, LB_PROF_SHAPE, N * N);
    k_tan_fwd<<<dim3((unsigned)ntb, (unsigned)nsplit), GR_NTH, 0, c->stream>>>(
        N, c->np, c->pos64, c->nrm64, packed, mt->flags, ntiles, c->row_ptr, c->near_patch, tps, part);
    LB_LAUNCH(c);
  }
  lb_pair_counter += N * N;
  k_reduce_tg<<<lb_div_up(N, 256), 256, 0, c->stream>>>(N, (int)nsplit, TG_NF, part, V);
  LB_LAUNCH(c);
  // transposed sums of a0 .. a5
  GradVecs gt{};
  for (int m = 0; m < 6; ++m) gt.v[m] = avs[m];
  k_pack_g<<<lb_div_up(Npad, 256), 256, 0, c->stream>>>(N, Npad, 6, nullptr, gt, packed);
  LB_LAUNCH(c);
  {
    ProfScope prof(c, LB_PROF_SHAPE, N * N);
    k_tan_tr<<<dim3((unsigned)ntb, (unsigned)nsplit), GR_NTH, 0, c->stream>>>(
        N, c->np, c->pos64, c->nrm64, packed, c->tflag, c->tmask, ntiles, tps, part);
    LB_LAUNCH(c);
  }
  lb_pair_counter += N * N;
  k_reduce_tg<<<lb_div_up(N, 256), 256, 0, c->stream>>>(N, (int)nsplit, TG_NT, part, U);
  LB_LAUNCH(c);
  TanIn in{};
  for (int m = 0; m < 6; ++m) {
    in.a[m] = avs[m];
    in.b[m] = bvs[m];
  }
  in.V = V;
  in.U = U;
  in.z = z;
  in.mu2 = mu2;
  in.Smu2 = pot2 + (int64_t)LB_K_S * N;
  in.Spmu2 = pot2 + (int64_t)LB_K_SP * N;
  in.pf = pf;
  in.partial = partial;
  in.npart = T_RB;
  k_tan_local<<<lb_div_up(N, 128), 128, 0, c->stream>>>(N, c->np, in, c->Xu, c->Xv, c->nrm, c->w, c->J, c->ginv,
                                                         c->dref, c->dDu, c->dDv, c->area, gXu, gXv, g2);
  LB_LAUNCH(c);
  k_tan_diff<<<lb_div_up(N, 128), 128, 0, c->stream>>>(N, c->np, c->dDu, c->dDv, g2, gXu, gXv);
  LB_LAUNCH(c);
  return LB_OK;
}
