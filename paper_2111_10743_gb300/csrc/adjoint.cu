// Transposed applies and the adjoint (density) solve.
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
