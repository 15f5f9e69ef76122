// GMRES, the mean-zero Laplace-Beltrami solve (single and lockstep), mixed-
// precision refinement, surface differential operators, harmonic vector
// fields, the A1 apply, the adjoint solve and the node-position gradient
// (whose pair sums live in the adjoint module).
//
// GMRES (Section 6: relative residual below tol, at most max_iter = 100
// iterations): x0 = 0, no restart, Euclidean inner product.  The Arnoldi
// basis lives on the device in float64; orthogonalisation is classical
// Gram-Schmidt applied twice (CGS2), whose two passes are each one multi-dot
// and one multi-axpy over all previous vectors; the Hessenberg column, the
// Givens rotations and the residual estimate |g_{j+1}| / |b| are updated by
// a single-thread kernel, and only that scalar is read back per iteration.
// Reductions are fixed-order (per-block partials, then an ordered sum).
//
// Mixed precision (LB_FP32_REFINED): float32 pair sums are accurate to about
// 1e-6, so an inner GMRES on the float32 operator to inner_tol is wrapped in
// iterative refinement whose residual b - A x uses double-float pair sums
// (about 1e-14, several times faster than float64 on GB300).  The solution
// potential is that apply's S[S[x1]] plus the float32 potentials that the
// later update applies compute on the way.
//
// Several right-hand sides (A3) advance in lockstep with one batched apply
// per iteration, each iteration replayed as a captured CUDA graph; see the
// Lockstep section below.
//
// Surface operators (Section 2), by nodal differentiation within a patch:
//   grad_Gamma f = (g^11 f_u + g^12 f_v) X_u + (g^21 f_u + g^22 f_v) X_v,
//   div_Gamma F = |X_u x X_v|^-1 (d_u(|X_u x X_v| F^1) + d_v(|X_u x X_v| F^2)),
//   F^a = g^ab (F . X_b).
// Harmonic fields (Section 5): Delta alpha = div F, Delta beta =
// -div(n x F), H = F - grad alpha - n x grad beta, and n x H.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <vector>

#include "internal.cuh"

#define GM_RB 128  // reduction blocks of the multi-dot

__global__ void k_multidot(int64_t N, int nvec, const double* __restrict__ V, int64_t ldv,
                           const double* __restrict__ w, double* __restrict__ partial) {
  __shared__ double sh[256];
  for (int v = 0; v < nvec; ++v) {
    const double* Vv = V + (int64_t)v * ldv;
    double s = 0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x)
      s += Vv[i] * w[i];
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int k = blockDim.x / 2; k > 0; k >>= 1) {
      if (threadIdx.x < k) sh[threadIdx.x] += sh[threadIdx.x + k];
      __syncthreads();
    }
    if (threadIdx.x == 0) partial[(int64_t)v * gridDim.x + blockIdx.x] = sh[0];
    __syncthreads();
  }
}

// out[v] (+)= ordered sum of the partials of vector v
__global__ void k_reduce_cols(int nvec, int nblk, const double* __restrict__ partial, double* __restrict__ out,
                              int accumulate) {
  int v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= nvec) return;
  double s = 0;
  for (int b = 0; b < nblk; ++b) s += partial[(int64_t)v * nblk + b];
  out[v] = accumulate ? out[v] + s : s;
}

// w -= sum_v h[v] V[v]
__global__ void k_axpy_multi(int64_t N, int nvec, const double* __restrict__ V, int64_t ldv,
                             const double* __restrict__ h, double* __restrict__ w) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
    double s = w[i];
    for (int v = 0; v < nvec; ++v) s -= h[v] * V[(int64_t)v * ldv + i];
    w[i] = s;
  }
}

// y = x / *s  (s on the device; zero output when *s == 0); y may equal x
__global__ void k_scale_by(int64_t N, const double* __restrict__ x, const double* __restrict__ s, double* y) {
  const double d = s[0] != 0.0 ? 1.0 / s[0] : 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x)
    y[i] = x[i] * d;
}

__global__ void k_add_small(int n, const double* __restrict__ a, double* __restrict__ b) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) b[i] += a[i];
}

// x = sum_v y[v] V[v]  (+ x when accumulate)
__global__ void k_combine(int64_t N, int nvec, const double* __restrict__ V, int64_t ldv,
                          const double* __restrict__ y, double* __restrict__ x, int accumulate) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
    double s = accumulate ? x[i] : 0.0;
    for (int v = 0; v < nvec; ++v) s += y[v] * V[(int64_t)v * ldv + i];
    x[i] = s;
  }
}

__global__ void k_sqrt_to(const double* __restrict__ a, double* __restrict__ b) {
  if (threadIdx.x == 0) b[0] = sqrt(a[0]);
}

// Hessenberg column j (h[0..j], hn = h[j+1]) -> rotations, g, residual
__global__ void k_givens(int j, int ldh, const double* __restrict__ h, double* __restrict__ Hm,
                         double* __restrict__ cs, double* __restrict__ sn, double* __restrict__ g, double beta,
                         double* __restrict__ resid) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double* col = Hm + (int64_t)j * ldh;
  for (int i = 0; i <= j + 1; ++i) col[i] = h[i];
  for (int i = 0; i < j; ++i) {
    const double t = cs[i] * col[i] + sn[i] * col[i + 1];
    col[i + 1] = -sn[i] * col[i] + cs[i] * col[i + 1];
    col[i] = t;
  }
  const double a = col[j], b = col[j + 1];
  const double r = hypot(a, b);
  const double c = r > 0 ? a / r : 1.0, s = r > 0 ? b / r : 0.0;
  cs[j] = c;
  sn[j] = s;
  col[j] = r;
  col[j + 1] = 0.0;
  g[j + 1] = -s * g[j];
  g[j] = c * g[j];
  resid[0] = fabs(g[j + 1]) / beta;
  resid[1] = r;
}

__global__ void k_backsolve(int k, int ldh, const double* __restrict__ Hm, const double* __restrict__ g,
                            double* __restrict__ y) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  for (int i = k - 1; i >= 0; --i) {
    double s = g[i];
    for (int l = i + 1; l < k; ++l) s -= Hm[(int64_t)l * ldh + i] * y[l];
    const double d = Hm[(int64_t)i * ldh + i];
    y[i] = d != 0.0 ? s / d : 0.0;
  }
}

__global__ void k_sub_scalar(int64_t N, const double* __restrict__ x, double m, double* __restrict__ y) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x)
    y[i] = x[i] - m;
}

__global__ void k_axpby(int64_t N, double a, const double* __restrict__ x, double b, double* __restrict__ y) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x)
    y[i] = a * x[i] + b * y[i];
}

__global__ void k_check_finite(int64_t N, const double* __restrict__ x, int* __restrict__ bad) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x)
    if (!isfinite(x[i])) atomicExch(bad, 1);
}

// ---------------------------------------------------------------------------
struct Gm {
  int m, ldh;
  int64_t ldv;  // distance between consecutive basis vectors of this system
  double *V, *h, *Hm, *cs, *sn, *g, *y, *partial, *scal, *w;
};

static int gm_work(lb_ctx* c, int m, Gm* G) {
  const int64_t N = c->N;
  const int ldh = m + 1;
  size_t need = (size_t)(m + 1) * N + (size_t)(m + 2) + (size_t)ldh * m + 3 * (size_t)(m + 2) + (size_t)(m + 2) +
                (size_t)GM_RB * (m + 2) + 8 + N;
  LB_CHECK(lb_ensure(c, c->ws_gm, need * sizeof(double)));
  double* p = (double*)c->ws_gm.p;
  G->m = m;
  G->ldh = ldh;
  G->ldv = N;
  G->V = p; p += (size_t)(m + 1) * N;
  G->h = p; p += m + 2;
  G->Hm = p; p += (size_t)ldh * m;
  G->cs = p; p += m + 2;
  G->sn = p; p += m + 2;
  G->g = p; p += m + 2;
  G->y = p; p += m + 2;
  G->partial = p; p += (size_t)GM_RB * (m + 2);
  G->scal = p; p += 8;
  G->w = p;
  return LB_OK;
}

static unsigned vec_blocks(lb_ctx* c) { return (unsigned)std::min<int64_t>(4 * c->sm_count, lb_div_up(c->N, 256)); }

// squared norm / dots into dst (device) via fixed-order partials
static int dots(lb_ctx* c, Gm& G, int nvec, const double* V, const double* w, double* dst, int accumulate) {
  k_multidot<<<GM_RB, 256, 0, c->stream>>>(c->N, nvec, V, G.ldv, w, G.partial);
  LB_LAUNCH(c);
  k_reduce_cols<<<lb_div_up(nvec, 64), 64, 0, c->stream>>>(nvec, GM_RB, G.partial, dst, accumulate);
  LB_LAUNCH(c);
  return LB_OK;
}

static int read_scalar(lb_ctx* c, const double* d, double* h) {
  LB_CUDA(c, cudaMemcpyAsync(c->host_pinned, d, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  LB_CUDA(c, cudaStreamSynchronize(c->stream));
  *h = c->host_pinned[0];
  return LB_OK;
}

// After w = A v_j: classical Gram-Schmidt twice (h = V^T w, w -= V h,
// h2 = V^T w, w -= V h2, h += h2), v_{j+1} = w / |w|, and the Givens update
// of column j; G.scal[0] then holds the residual estimate.
static int arnoldi_step(lb_ctx* c, Gm& G, int j, double beta) {
  const int64_t N = c->N;
  const unsigned nb = vec_blocks(c);
  double* vn = G.V + (int64_t)(j + 1) * G.ldv;
  LB_CHECK(dots(c, G, j + 1, G.V, G.w, G.h, 0));
  k_axpy_multi<<<nb, 256, 0, c->stream>>>(N, j + 1, G.V, G.ldv, G.h, G.w);
  LB_LAUNCH(c);
  LB_CHECK(dots(c, G, j + 1, G.V, G.w, G.y, 0));
  k_axpy_multi<<<nb, 256, 0, c->stream>>>(N, j + 1, G.V, G.ldv, G.y, G.w);
  LB_LAUNCH(c);
  k_add_small<<<lb_div_up(j + 1, 128), 128, 0, c->stream>>>(j + 1, G.y, G.h);
  LB_LAUNCH(c);
  LB_CHECK(dots(c, G, 1, G.w, G.w, G.scal + 2, 0));
  k_sqrt_to<<<1, 32, 0, c->stream>>>(G.scal + 2, G.h + j + 1);
  LB_LAUNCH(c);
  k_scale_by<<<nb, 256, 0, c->stream>>>(N, G.w, G.h + j + 1, vn);
  LB_LAUNCH(c);
  k_givens<<<1, 32, 0, c->stream>>>(j, G.ldh, G.h, G.Hm, G.cs, G.sn, G.g, beta, G.scal);
  LB_LAUNCH(c);
  return LB_OK;
}

// GMRES on the formulation operator with pair precision prec.
// x (device) receives the solution; *iters the iteration count, *res the
// final residual estimate; hist (may be null) the estimates per iteration.
static int gmres(lb_ctx* c, int prec, const double* b, double* x, double tol, int max_iter, int* iters, double* res,
                 std::vector<double>* hist) {
  const int64_t N = c->N;
  Gm G;
  LB_CHECK(gm_work(c, max_iter, &G));
  const unsigned nb = vec_blocks(c);
  double beta2 = 0;
  LB_CHECK(dots(c, G, 1, b, b, G.scal + 2, 0));
  LB_CHECK(read_scalar(c, G.scal + 2, &beta2));
  const double beta = sqrt(beta2);
  *iters = 0;
  *res = 0;
  if (!std::isfinite(beta)) return lb_fail(c, LB_EINVAL, "non-finite right-hand side");
  if (!(beta > 0)) {
    LB_CUDA(c, cudaMemsetAsync(x, 0, N * sizeof(double), c->stream));
    return LB_OK;
  }
  LB_CUDA(c, cudaMemsetAsync(G.g, 0, (G.m + 2) * sizeof(double), c->stream));
  c->host_pinned[8] = beta;
  LB_CUDA(c, cudaMemcpyAsync(G.g, c->host_pinned + 8, sizeof(double), cudaMemcpyHostToDevice, c->stream));
  k_sqrt_to<<<1, 32, 0, c->stream>>>(G.scal + 2, G.scal + 3);
  LB_LAUNCH(c);
  k_scale_by<<<nb, 256, 0, c->stream>>>(N, b, G.scal + 3, G.V);
  LB_LAUNCH(c);
  if (hist) hist->push_back(1.0);
  int k = 0;
  double r = 1.0;
  for (int j = 0; j < max_iter; ++j) {
    const double* vj = G.V + (int64_t)j * N;
    if (c->adjoint) LB_CHECK(lb_apply_at_op(c, vj, G.w));
    else LB_CHECK(lb_apply_op(c, c->params.formulation, prec, vj, G.w));
    LB_CHECK(arnoldi_step(c, G, j, beta));
    LB_CHECK(read_scalar(c, G.scal, &r));
    if (hist) hist->push_back(r);
    k = j + 1;
    if (!std::isfinite(r)) return lb_fail(c, LB_EINVAL, "GMRES breakdown: non-finite residual");
    if (r < tol || r == 0.0) break;
  }
  k_backsolve<<<1, 32, 0, c->stream>>>(k, G.ldh, G.Hm, G.g, G.y);
  LB_LAUNCH(c);
  k_combine<<<nb, 256, 0, c->stream>>>(N, k, G.V, N, G.y, x, 0);
  LB_LAUNCH(c);
  *iters = k;
  *res = r;
  return LB_OK;
}

// ---------------------------------------------------------------------------
// norms and mean projection helpers on the context stream
static int norm2(lb_ctx* c, const double* v, double* out) {
  Gm G;
  LB_CHECK(gm_work(c, 1, &G));
  LB_CHECK(dots(c, G, 1, v, v, G.scal + 2, 0));
  double s = 0;
  LB_CHECK(read_scalar(c, G.scal + 2, &s));
  *out = sqrt(s);
  return LB_OK;
}

static int project_mean_zero(lb_ctx* c, const double* f, double* out, double* removed) {
  double m = 0;
  LB_CHECK(lb_wmean(c, f, &m));
  k_sub_scalar<<<vec_blocks(c), 256, 0, c->stream>>>(c->N, f, m, out);
  LB_LAUNCH(c);
  if (removed) *removed = m;
  return LB_OK;
}

// S applied with precision prec (far + near), device in/out
static int apply_S_dev(lb_ctx* c, int prec, const double* s, double* out) {
  LB_CHECK(lb_ensure(c, c->ws_vec, (size_t)(4 * c->N) * sizeof(double)));
  double* pot = (double*)c->ws_vec.p;
  LB_CHECK(lb_potentials(c, prec, s, pot, 1u << LB_K_S));
  LB_CUDA(c, cudaMemcpyAsync(out, pot, c->N * sizeof(double), cudaMemcpyDeviceToDevice, c->stream));
  return LB_OK;
}

// ---------------------------------------------------------------------------
// Recycling the first inner solve's Krylov space in the later ones of the
// refinement (GCRO, de Sturler 1996; the augmented GMRES of Saad 1997).  The
// first inner GMRES leaves V (k + 1 basis vectors) and, in the Hessenberg
// storage, R with the Givens rotations Omega_j that produced it:
// Omega_k ... Omega_1 H_k = [R; 0], so H_k = Q R with Q the first k columns
// of Omega_1^T ... Omega_k^T.  Then C = V Q has orthonormal columns and
// A32 U = C for U = V_k R^-1.  A later inner solve of A32 delta = r is
// minimised over span(U) + K_m((I - C C^T) A32, r'), r' = r - C C^T r:
// with B = C^T A32 V2 collected during its Arnoldi process,
// delta = U (C^T r - B y) + V2 y, and its residual is that of the small
// least-squares problem.  A restarted GMRES would rebuild the directions
// that the first solve already found (two iterations on the benchmark
// surface: plain float32 GMRES takes 9 iterations to 3e-11, the
// restarted refinement 5 + 6).
struct Recycle {
  int k = 0;
  double* V = nullptr;   // [k + 1][N] the first solve's basis
  double* C = nullptr;   // [k][N] C = V Q
  double* sm = nullptr;  // device scratch: alpha [k], B [k][max_iter], two k-vectors
  std::vector<double> R;  // k x k upper triangle, column-major
};

// after the first inner gmres (k iterations, workspace of max_iter)
static int recycle_capture(lb_ctx* c, int k, int max_iter, Recycle* rc) {
  rc->k = 0;
  if (k < 1) return LB_OK;
  const int64_t N = c->N;
  Gm G;
  LB_CHECK(gm_work(c, max_iter, &G));  // the first solve's layout
  const size_t need = (size_t)(2 * k + 1) * N + (size_t)k * (max_iter + 3) + (size_t)(k + 1) * k + 8;
  LB_CHECK(lb_ensure(c, c->ws_rec, need * sizeof(double)));
  rc->V = (double*)c->ws_rec.p;
  rc->C = rc->V + (size_t)(k + 1) * N;
  rc->sm = rc->C + (size_t)k * N;
  double* Qd = rc->sm + (size_t)k * (max_iter + 3);
  LB_CUDA(c, cudaMemcpyAsync(rc->V, G.V, (size_t)(k + 1) * N * sizeof(double), cudaMemcpyDeviceToDevice, c->stream));
  std::vector<double> Hm((size_t)G.ldh * k), cs(k), sn(k);
  LB_CUDA(c, cudaMemcpyAsync(Hm.data(), G.Hm, Hm.size() * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  LB_CUDA(c, cudaMemcpyAsync(cs.data(), G.cs, k * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  LB_CUDA(c, cudaMemcpyAsync(sn.data(), G.sn, k * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  LB_CUDA(c, cudaStreamSynchronize(c->stream));
  rc->R.assign((size_t)k * k, 0.0);
  for (int l = 0; l < k; ++l)
    for (int i = 0; i <= l; ++i) rc->R[(size_t)l * k + i] = Hm[(size_t)l * G.ldh + i];
  for (int i = 0; i < k; ++i)
    if (!(std::fabs(rc->R[(size_t)i * k + i]) > 0)) return LB_OK;  // breakdown: no recycling
  // Q = Omega_1^T ... Omega_k^T [I_k; 0], column-major (k + 1) x k
  std::vector<double> Q((size_t)(k + 1) * k, 0.0);
  for (int l = 0; l < k; ++l) Q[(size_t)l * (k + 1) + l] = 1.0;
  for (int j = k - 1; j >= 0; --j)
    for (int l = 0; l < k; ++l) {
      double* q = &Q[(size_t)l * (k + 1)];
      const double a = q[j], b = q[j + 1];
      q[j] = cs[j] * a - sn[j] * b;
      q[j + 1] = sn[j] * a + cs[j] * b;
    }
  LB_CUDA(c, cudaMemcpyAsync(Qd, Q.data(), Q.size() * sizeof(double), cudaMemcpyHostToDevice, c->stream));
  const unsigned nb = vec_blocks(c);
  for (int l = 0; l < k; ++l) {
    k_combine<<<nb, 256, 0, c->stream>>>(N, k + 1, rc->V, N, Qd + (size_t)l * (k + 1), rc->C + (size_t)l * N, 0);
    LB_LAUNCH(c);
  }
  LB_CUDA(c, cudaStreamSynchronize(c->stream));  // Q (host) is released on return
  rc->k = k;
  return LB_OK;
}

// GMRES for A32 x = b over span(U) + the projected Krylov space (above);
// *res relative to |b|
static int gmres_recycled(lb_ctx* c, const double* b, double* x, double tol, int max_iter, const Recycle& rc,
                          int* iters, double* res) {
  const int64_t N = c->N;
  const int k = rc.k;
  const unsigned nb = vec_blocks(c);
  Gm G;
  LB_CHECK(gm_work(c, max_iter, &G));
  double* alpha = rc.sm;
  double* Bm = alpha + k;                          // column j at Bm + j k
  double* t1 = Bm + (size_t)k * max_iter;          // second projection pass
  *iters = 0;
  *res = 0;
  double bb = 0;
  LB_CHECK(dots(c, G, 1, b, b, G.scal + 2, 0));
  LB_CHECK(read_scalar(c, G.scal + 2, &bb));
  const double bnorm = std::sqrt(bb);
  if (!std::isfinite(bnorm)) return lb_fail(c, LB_EINVAL, "non-finite right-hand side");
  if (!(bnorm > 0)) {
    LB_CUDA(c, cudaMemsetAsync(x, 0, N * sizeof(double), c->stream));
    return LB_OK;
  }
  // alpha = C^T b, r' = b - C alpha (two passes)
  LB_CUDA(c, cudaMemcpyAsync(G.w, b, N * sizeof(double), cudaMemcpyDeviceToDevice, c->stream));
  LB_CHECK(dots(c, G, k, rc.C, G.w, alpha, 0));
  k_axpy_multi<<<nb, 256, 0, c->stream>>>(N, k, rc.C, N, alpha, G.w);
  LB_LAUNCH(c);
  LB_CHECK(dots(c, G, k, rc.C, G.w, t1, 0));
  k_axpy_multi<<<nb, 256, 0, c->stream>>>(N, k, rc.C, N, t1, G.w);
  LB_LAUNCH(c);
  k_add_small<<<lb_div_up(k, 128), 128, 0, c->stream>>>(k, t1, alpha);
  LB_LAUNCH(c);
  double rr2 = 0;
  LB_CHECK(dots(c, G, 1, G.w, G.w, G.scal + 2, 0));
  LB_CHECK(read_scalar(c, G.scal + 2, &rr2));
  const double beta = std::sqrt(rr2);
  int kk = 0;
  double r = beta / bnorm;
  if (beta > 0 && r >= tol) {
    LB_CUDA(c, cudaMemsetAsync(G.g, 0, (G.m + 2) * sizeof(double), c->stream));
    c->host_pinned[8] = beta;
    LB_CUDA(c, cudaMemcpyAsync(G.g, c->host_pinned + 8, sizeof(double), cudaMemcpyHostToDevice, c->stream));
    k_sqrt_to<<<1, 32, 0, c->stream>>>(G.scal + 2, G.scal + 3);
    LB_LAUNCH(c);
    k_scale_by<<<nb, 256, 0, c->stream>>>(N, G.w, G.scal + 3, G.V);
    LB_LAUNCH(c);
    for (int j = 0; j < max_iter; ++j) {
      const double* vj = G.V + (int64_t)j * G.ldv;
      LB_CHECK(lb_apply_op(c, c->params.formulation, LB_FP32, vj, G.w));
      double* bj = Bm + (size_t)j * k;
      LB_CHECK(dots(c, G, k, rc.C, G.w, bj, 0));
      k_axpy_multi<<<nb, 256, 0, c->stream>>>(N, k, rc.C, N, bj, G.w);
      LB_LAUNCH(c);
      LB_CHECK(dots(c, G, k, rc.C, G.w, t1, 0));
      k_axpy_multi<<<nb, 256, 0, c->stream>>>(N, k, rc.C, N, t1, G.w);
      LB_LAUNCH(c);
      k_add_small<<<lb_div_up(k, 128), 128, 0, c->stream>>>(k, t1, bj);
      LB_LAUNCH(c);
      LB_CHECK(arnoldi_step(c, G, j, beta));
      double rj = 0;
      LB_CHECK(read_scalar(c, G.scal, &rj));
      kk = j + 1;
      r = rj * beta / bnorm;
      if (!std::isfinite(r)) return lb_fail(c, LB_EINVAL, "GMRES breakdown: non-finite residual");
      if (r < tol || rj == 0.0) break;
    }
    k_backsolve<<<1, 32, 0, c->stream>>>(kk, G.ldh, G.Hm, G.g, G.y);
    LB_LAUNCH(c);
  }
  // z = alpha - B y, coefficients of V_k: R^-1 z
  std::vector<double> al(k), Bh((size_t)k * std::max(kk, 1)), yh(std::max(kk, 1)), cu(k);
  LB_CUDA(c, cudaMemcpyAsync(al.data(), alpha, k * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  if (kk > 0) {
    LB_CUDA(c, cudaMemcpyAsync(Bh.data(), Bm, (size_t)k * kk * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    LB_CUDA(c, cudaMemcpyAsync(yh.data(), G.y, kk * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  }
  LB_CUDA(c, cudaStreamSynchronize(c->stream));
  for (int i = 0; i < k; ++i) {
    double z = al[i];
    for (int j = 0; j < kk; ++j) z -= Bh[(size_t)j * k + i] * yh[j];
    cu[i] = z;
  }
  for (int i = k - 1; i >= 0; --i) {
    double s = cu[i];
    for (int l = i + 1; l < k; ++l) s -= rc.R[(size_t)l * k + i] * cu[l];
    cu[i] = s / rc.R[(size_t)i * k + i];
  }
  LB_CUDA(c, cudaMemcpyAsync(t1, cu.data(), k * sizeof(double), cudaMemcpyHostToDevice, c->stream));
  k_combine<<<nb, 256, 0, c->stream>>>(N, k, rc.V, N, t1, x, 0);
  LB_LAUNCH(c);
  if (kk > 0) {
    k_combine<<<nb, 256, 0, c->stream>>>(N, kk, G.V, G.ldv, G.y, x, 1);
    LB_LAUNCH(c);
  }
  LB_CUDA(c, cudaStreamSynchronize(c->stream));  // host vectors are released on return
  *iters = kk;
  *res = r;
  return LB_OK;
}

// one right-hand side: b (device) -> sigma (device).  In the refined mode the
// solution potential u is produced here too (u_out), otherwise by the caller.
//
// Refinement (LB_FP32_REFINED), standard iterative refinement with the
// residual in higher precision where it matters:
//   x1 = GMRES32(b); r1 = b - A_df x1 (the one double-float apply; its second
//   pass also yields S^2 x1 for A3, its first S x1 for A2);
//   then x_{k+1} = x_k + GMRES32(r_k), r_{k+1} = r_k - A32 delta: delta is
//   about inner_tol |x|, so float32 pairs (relative 1e-7) keep this update
//   accurate to about 1e-7 inner_tol |b|;
//   u = (S^2 x1 or S x1) + the float32 potentials of the corrections, for
//   the same reason; each update apply A32 delta computes the potential of
//   delta on the way (S^2 delta in A3's second pass, S delta in the first
//   pass of A2 and A1), and x - x1 is the sum of the deltas.
static int solve_one(lb_ctx* c, const double* b, double* sigma, double* scratch, lb_solve_info* info, int first,
                     double* u_out) {
  const int64_t N = c->N;
  const lb_params& p = c->params;
  std::vector<double> hist;
  int it = 0;
  double res = 0;
  const unsigned nb = vec_blocks(c);
  if (p.precision != LB_FP32_REFINED) {
    LB_CHECK(gmres(c, p.precision, b, sigma, p.tol, p.max_iter, &it, &res, first ? &hist : nullptr));
    if (info) {
      info->iterations += it;
      info->converged = info->converged && (res < p.tol);
      info->rel_residual = std::max(info->rel_residual, res);
    }
  } else {
    double* r = scratch;
    double* delta = scratch + N;
    double* Ax = scratch + 2 * N;
    double* x1 = scratch + 3 * N;
    double* ux1 = scratch + 4 * N;
    double* uacc = scratch + 5 * N;  // float32 solution potential of x - x1
    double nbv = 0, rn = 0;
    LB_CHECK(norm2(c, b, &nbv));
    LB_CUDA(c, cudaMemsetAsync(sigma, 0, N * sizeof(double), c->stream));
    LB_CUDA(c, cudaMemsetAsync(x1, 0, N * sizeof(double), c->stream));
    LB_CUDA(c, cudaMemsetAsync(ux1, 0, N * sizeof(double), c->stream));
    LB_CUDA(c, cudaMemsetAsync(uacc, 0, N * sizeof(double), c->stream));
    LB_CUDA(c, cudaMemcpyAsync(r, b, N * sizeof(double), cudaMemcpyDeviceToDevice, c->stream));
    bool ok = nbv == 0.0;
    int steps = 0;
    double rel = nbv == 0.0 ? 0.0 : 1.0;
    Recycle rec;
    if (first) hist.push_back(1.0);
    for (int s = 0; s < p.max_refine && !ok; ++s) {
      int its = 0;
      double ires = 0;
      // once the residual r_s is known (rel = |r_s| / |b|), the inner solve
      // need only take it to half the target: tol |b| / 2
      const double itol = s == 0 ? p.inner_tol : std::max(p.inner_tol, std::min(0.5, 0.5 * p.tol / rel));
      if (s > 0 && rec.k > 0)
        LB_CHECK(gmres_recycled(c, r, delta, itol, p.max_iter, rec, &its, &ires));
      else
        LB_CHECK(gmres(c, LB_FP32, r, delta, itol, p.max_iter, &its, &ires, nullptr));
      if (s == 0) LB_CHECK(recycle_capture(c, its, p.max_iter, &rec));
      it += its;
      k_axpby<<<nb, 256, 0, c->stream>>>(N, 1.0, delta, 1.0, sigma);
      LB_LAUNCH(c);
      if (s == 0) {
        // r = b - A x1 in double-float; keep x1 and its solution potential
        LB_CHECK(lb_apply_op(c, p.formulation, LB_DF64, sigma, Ax));
        const double* pot = (const double*)c->ws_pot.p;  // [4][N] of the last apply
        LB_CUDA(c, cudaMemcpyAsync(ux1, p.formulation == LB_A3 ? pot + N : pot, N * sizeof(double),
                                   cudaMemcpyDeviceToDevice, c->stream));
        LB_CUDA(c, cudaMemcpyAsync(x1, sigma, N * sizeof(double), cudaMemcpyDeviceToDevice, c->stream));
        LB_CUDA(c, cudaMemcpyAsync(r, b, N * sizeof(double), cudaMemcpyDeviceToDevice, c->stream));
        k_axpby<<<nb, 256, 0, c->stream>>>(N, -1.0, Ax, 1.0, r);
        LB_LAUNCH(c);
      } else {
        // r -= A32 delta; the apply's passes also hold the solution potential
        // of delta (S[S[delta]] for A3, S[delta] otherwise), accumulated for u
        LB_CHECK(lb_apply_op(c, p.formulation, LB_FP32, delta, Ax));
        k_axpby<<<nb, 256, 0, c->stream>>>(N, -1.0, Ax, 1.0, r);
        LB_LAUNCH(c);
        const double* pot = (const double*)c->ws_pot.p;
        k_axpby<<<nb, 256, 0, c->stream>>>(N, 1.0, p.formulation == LB_A3 ? pot + N : pot, 1.0, uacc);
        LB_LAUNCH(c);
      }
      LB_CHECK(norm2(c, r, &rn));
      rel = rn / nbv;
      ++steps;
      if (first) hist.push_back(rel);
      if (rel < p.tol) ok = true;
    }
    res = rel;
    if (info) {
      info->iterations += it;
      info->refinements += steps;
      info->converged = info->converged && ok;
      info->rel_residual = std::max(info->rel_residual, rel);
    }
    if (u_out) {  // u = u(x1) + the float32 potentials of the later corrections (x - x1 = their sum)
      LB_CUDA(c, cudaMemcpyAsync(u_out, ux1, N * sizeof(double), cudaMemcpyDeviceToDevice, c->stream));
      k_axpby<<<nb, 256, 0, c->stream>>>(N, 1.0, uacc, 1.0, u_out);
      LB_LAUNCH(c);
    }
  }
  if (info && first) {
    info->history_len = (int32_t)std::min<size_t>(hist.size(), 128);
    for (int i = 0; i < info->history_len; ++i) info->history[i] = hist[i];
  }
  return LB_OK;
}

// ---------------------------------------------------------------------------
// Lockstep solves of R right-hand sides (A3, float32 or double-float pairs).
//
// The R systems advance together: each GMRES iteration applies A3 once to
// the current basis vectors of all systems still iterating (one batched
// far-field pass per A3 pass, several densities per pair evaluation), then
// runs the Arnoldi step of those systems in kernels that cover all of them
// at once (blockIdx.y = system).  A system stops when its own residual
// estimate is below tol, exactly as it would alone.
//
// The iteration index j lives on the device and the active systems travel
// as a kernel argument, so one iteration is a fixed sequence of launches:
// captured once as a CUDA graph per active set and replayed (parameter
// `graphs`), or launched directly; both
// run the same kernels on the same data and give identical results.
//
// Workspace: V [m+1][R][N] (the j-th vectors of all systems adjacent), the
// gathered apply input and its output [R][N], split partials of the
// multi-dots, and per system a small block: h, the Hessenberg columns, the
// rotations, g, y and scalars (residual, squared norms, beta).
struct LkAct {
  int n;
  int r[LB_BATCH_MAX];
};

struct LkDev {
  int64_t N;
  int R, m, ldh;
  int64_t SM;          // doubles per system's small block
  double* V;           // [m+1][R][N]
  double* small;       // [R][SM]
  double* partial;     // [R][m+2][GM_RB]
  int* jdev;           // iteration index
  double* resbuf;      // [R] residual estimates of the active systems, in act order
  // recycled first-stage spaces (refinement; null when off): for system r,
  // ck[r] vectors C at C + coff[r] (stride N), B = C^T A V2 columns at
  // Bm + r * bld + j * kmax, a second-pass scratch at Bm + r * bld + m * kmax
  const double* C = nullptr;
  const int64_t* coff = nullptr;
  const int* ck = nullptr;
  double* Bm = nullptr;
  int64_t bld = 0;
  int kmax = 0;
};

// offsets inside a system's small block
#define LK_H(d) 0
#define LK_HM(d) ((d).m + 2)
#define LK_CS(d) (LK_HM(d) + (int64_t)(d).ldh * (d).m)
#define LK_SN(d) (LK_CS(d) + (d).m + 2)
#define LK_G(d) (LK_SN(d) + (d).m + 2)
#define LK_Y(d) (LK_G(d) + (d).m + 2)
#define LK_SC(d) (LK_Y(d) + (d).m + 2)  // [0] residual, [1] r, [2] |w|^2, [4] |b|^2, [5] beta
#define LK_SMALL(m) ((int64_t)((m) + 2) * 5 + (int64_t)((m) + 1) * (m) + 8)

// in[a] = V[j][act[a]]
__global__ void k_lk_gather(LkDev d, LkAct act, double* __restrict__ in) {
  const int a = blockIdx.y, r = act.r[a];
  const double* src = d.V + ((int64_t)(*d.jdev) * d.R + r) * d.N;
  double* dst = in + (int64_t)a * d.N;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < d.N; i += (int64_t)gridDim.x * blockDim.x)
    dst[i] = src[i];
}

// per-block partial dot products of w_a with V_r[0..j] (self = 0) or with
// itself (self = 1): partial[a][v][blk]
__global__ void k_lk_dots(LkDev d, LkAct act, const double* __restrict__ W, int self) {
  __shared__ double sh[256];
  const int a = blockIdx.y, r = act.r[a];
  const double* w = W + (int64_t)a * d.N;
  const int nvec = self ? 1 : *d.jdev + 1;
  for (int v = 0; v < nvec; ++v) {
    const double* x = self ? w : d.V + ((int64_t)v * d.R + r) * d.N;
    double s = 0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < d.N; i += (int64_t)gridDim.x * blockDim.x)
      s += x[i] * w[i];
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int k = blockDim.x / 2; k > 0; k >>= 1) {
      if (threadIdx.x < k) sh[threadIdx.x] += sh[threadIdx.x + k];
      __syncthreads();
    }
    if (threadIdx.x == 0) d.partial[((int64_t)a * (d.m + 2) + v) * gridDim.x + blockIdx.x] = sh[0];
    __syncthreads();
  }
}

// small_r[off + v] = ordered sum of the partials of vector v
__global__ void k_lk_reduce(LkDev d, LkAct act, int self, int64_t off, int nblk) {
  const int a = blockIdx.y, r = act.r[a];
  const int v = blockIdx.x * blockDim.x + threadIdx.x;
  const int nvec = self ? 1 : *d.jdev + 1;
  if (v >= nvec) return;
  double s = 0;
  for (int b = 0; b < nblk; ++b) s += d.partial[((int64_t)a * (d.m + 2) + v) * nblk + b];
  d.small[(int64_t)r * d.SM + off + v] = s;
}

// w_a -= sum_{v <= j} small_r[off + v] V_r[v]
__global__ void k_lk_axpy(LkDev d, LkAct act, double* __restrict__ W, int64_t off) {
  const int a = blockIdx.y, r = act.r[a];
  const int nvec = *d.jdev + 1;
  const double* c = d.small + (int64_t)r * d.SM + off;
  double* w = W + (int64_t)a * d.N;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < d.N; i += (int64_t)gridDim.x * blockDim.x) {
    double s = w[i];
    for (int v = 0; v < nvec; ++v) s -= c[v] * d.V[((int64_t)v * d.R + r) * d.N + i];
    w[i] = s;
  }
}

// h += y (the second Gram-Schmidt pass's coefficients)
__global__ void k_lk_addsmall(LkDev d, LkAct act) {
  const int a = blockIdx.y, r = act.r[a];
  const int v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v > *d.jdev) return;
  double* sm = d.small + (int64_t)r * d.SM;
  sm[LK_H(d) + v] += sm[LK_Y(d) + v];
}

// partial dot products of w_a with system r's recycled vectors C_r
__global__ void k_lk_cdots(LkDev d, LkAct act, const double* __restrict__ W) {
  __shared__ double sh[256];
  const int a = blockIdx.y, r = act.r[a];
  const double* w = W + (int64_t)a * d.N;
  const int nvec = d.ck[r];
  for (int v = 0; v < nvec; ++v) {
    const double* x = d.C + d.coff[r] + (int64_t)v * d.N;
    double s = 0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < d.N; i += (int64_t)gridDim.x * blockDim.x)
      s += x[i] * w[i];
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int k = blockDim.x / 2; k > 0; k >>= 1) {
      if (threadIdx.x < k) sh[threadIdx.x] += sh[threadIdx.x + k];
      __syncthreads();
    }
    if (threadIdx.x == 0) d.partial[((int64_t)a * (d.m + 2) + v) * gridDim.x + blockIdx.x] = sh[0];
    __syncthreads();
  }
}

// column `slot` of system r's coefficient block (slot < 0: the current
// iteration's B column j; m: a scratch column; m + 1: alpha = C^T b)
__device__ __forceinline__ double* lk_ccol(const LkDev& d, int r, int slot) {
  return d.Bm + (int64_t)r * d.bld + (int64_t)(slot < 0 ? *d.jdev : slot) * d.kmax;
}

// column `slot` = ordered sums of the partials of k_lk_cdots
__global__ void k_lk_creduce(LkDev d, LkAct act, int slot, int nblk) {
  const int a = blockIdx.y, r = act.r[a];
  const int v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= d.ck[r]) return;
  double s = 0;
  for (int b = 0; b < nblk; ++b) s += d.partial[((int64_t)a * (d.m + 2) + v) * nblk + b];
  lk_ccol(d, r, slot)[v] = s;
}

// w_a -= C_r (column `slot`)
__global__ void k_lk_caxpy(LkDev d, LkAct act, double* __restrict__ W, int slot) {
  const int a = blockIdx.y, r = act.r[a];
  const int nvec = d.ck[r];
  const double* coef = lk_ccol(d, r, slot);
  double* w = W + (int64_t)a * d.N;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < d.N; i += (int64_t)gridDim.x * blockDim.x) {
    double s2 = w[i];
    for (int v = 0; v < nvec; ++v) s2 -= coef[v] * d.C[d.coff[r] + (int64_t)v * d.N + i];
    w[i] = s2;
  }
}

// column `dst` += column `src`
__global__ void k_lk_cadd(LkDev d, LkAct act, int dst, int src) {
  const int a = blockIdx.y, r = act.r[a];
  const int v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= d.ck[r]) return;
  lk_ccol(d, r, dst)[v] += lk_ccol(d, r, src)[v];
}

// W_a -= C_r (C_r^T W_a) in two passes, the coefficients summed into
// column `slot` of system r's block
static int lk_project(lb_ctx* c, const LkDev& d, const LkAct& act, double* W, int slot) {
  const unsigned nb = vec_blocks(c);
  const dim3 gv(nb, act.n), gd(GM_RB, act.n), gc(lb_div_up(d.kmax, 64), act.n);
  for (int pass = 0; pass < 2; ++pass) {
    const int dst = pass == 0 ? slot : d.m;
    k_lk_cdots<<<gd, 256, 0, c->stream>>>(d, act, W);
    LB_LAUNCH(c);
    k_lk_creduce<<<gc, 64, 0, c->stream>>>(d, act, dst, GM_RB);
    LB_LAUNCH(c);
    k_lk_caxpy<<<gv, 256, 0, c->stream>>>(d, act, W, dst);
    LB_LAUNCH(c);
  }
  k_lk_cadd<<<gc, 64, 0, c->stream>>>(d, act, slot, d.m);
  LB_LAUNCH(c);
  return LB_OK;
}

// h_{j+1} = |w|, V_r[j+1] = w / |w| (zero when |w| = 0)
__global__ void k_lk_normalize(LkDev d, LkAct act, const double* __restrict__ W) {
  const int a = blockIdx.y, r = act.r[a];
  const int j = *d.jdev;
  double* sm = d.small + (int64_t)r * d.SM;
  const double hn = sqrt(sm[LK_SC(d) + 2]);
  if (blockIdx.x == 0 && threadIdx.x == 0) sm[LK_H(d) + j + 1] = hn;
  const double inv = hn != 0.0 ? 1.0 / hn : 0.0;
  const double* w = W + (int64_t)a * d.N;
  double* vn = d.V + ((int64_t)(j + 1) * d.R + r) * d.N;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < d.N; i += (int64_t)gridDim.x * blockDim.x)
    vn[i] = w[i] * inv;
}

// Givens update of column j for each active system; residual estimate
// |g_{j+1}| / beta into its scalars and into resbuf[a]
__global__ void k_lk_givens(LkDev d, LkAct act) {
  const int a = blockIdx.x * blockDim.x + threadIdx.x;
  if (a >= act.n) return;
  const int r = act.r[a];
  const int j = *d.jdev;
  double* sm = d.small + (int64_t)r * d.SM;
  const double* h = sm + LK_H(d);
  double* col = sm + LK_HM(d) + (int64_t)j * d.ldh;
  double* cs = sm + LK_CS(d);
  double* sn = sm + LK_SN(d);
  double* g = sm + LK_G(d);
  double* sc = sm + LK_SC(d);
  for (int i = 0; i <= j + 1; ++i) col[i] = h[i];
  for (int i = 0; i < j; ++i) {
    const double t = cs[i] * col[i] + sn[i] * col[i + 1];
    col[i + 1] = -sn[i] * col[i] + cs[i] * col[i + 1];
    col[i] = t;
  }
  const double x = col[j], y = col[j + 1];
  const double rr = hypot(x, y);
  const double cc = rr > 0 ? x / rr : 1.0, ss = rr > 0 ? y / rr : 0.0;
  cs[j] = cc;
  sn[j] = ss;
  col[j] = rr;
  col[j + 1] = 0.0;
  g[j + 1] = -ss * g[j];
  g[j] = cc * g[j];
  sc[0] = fabs(g[j + 1]) / sc[5];
  sc[1] = rr;
  d.resbuf[a] = sc[0];
}

__global__ void k_lk_advance(LkDev d) {
  if (threadIdx.x == 0 && blockIdx.x == 0) ++*d.jdev;
}

// start: beta_r = |b_r|, g_r = (beta_r, 0, ...), V_r[0] = b_r / beta_r
__global__ void k_lk_start(LkDev d, LkAct act, const double* __restrict__ b) {
  const int a = blockIdx.y, r = act.r[a];
  double* sm = d.small + (int64_t)r * d.SM;
  const double beta = sqrt(sm[LK_SC(d) + 4]);
  if (blockIdx.x == 0 && threadIdx.x == 0) sm[LK_SC(d) + 5] = beta;
  const double inv = beta != 0.0 ? 1.0 / beta : 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < d.N; i += (int64_t)gridDim.x * blockDim.x)
    d.V[(int64_t)r * d.N + i] = b[(int64_t)r * d.N + i] * inv;
  if (blockIdx.x == 0)
    for (int v = threadIdx.x; v < d.m + 2; v += blockDim.x) sm[LK_G(d) + v] = v == 0 ? beta : 0.0;
}

// back substitution and x_r = V_r y_r for system r with k_r iterations
__global__ void k_lk_backsolve(LkDev d, int r, int k) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double* sm = d.small + (int64_t)r * d.SM;
  const double* Hm = sm + LK_HM(d);
  const double* g = sm + LK_G(d);
  double* y = sm + LK_Y(d);
  for (int i = k - 1; i >= 0; --i) {
    double s = g[i];
    for (int l = i + 1; l < k; ++l) s -= Hm[(int64_t)l * d.ldh + i] * y[l];
    const double dd = Hm[(int64_t)i * d.ldh + i];
    y[i] = dd != 0.0 ? s / dd : 0.0;
  }
}

struct Lockstep {
  int R = 0, m = 0;
  LkDev d{};
  double* in = nullptr;   // [R][N] gathered apply input
  double* out = nullptr;  // [R][N] apply output
};

static int lockstep_work(lb_ctx* c, int R, int m, Lockstep* L) {
  const int64_t N = c->N;
  const int64_t SM = LK_SMALL(m);
  const size_t need = (size_t)(m + 1) * R * N + 2 * (size_t)R * N + (size_t)R * (m + 2) * GM_RB +
                      (size_t)R * SM + (size_t)R + 8;
  LB_CHECK(lb_ensure(c, c->ws_bgm, need * sizeof(double)));
  double* p = (double*)c->ws_bgm.p;
  L->R = R;
  L->m = m;
  LkDev& d = L->d;
  d.N = N;
  d.R = R;
  d.m = m;
  d.ldh = m + 1;
  d.SM = SM;
  d.V = p; p += (size_t)(m + 1) * R * N;
  L->in = p; p += (size_t)R * N;
  L->out = p; p += (size_t)R * N;
  d.partial = p; p += (size_t)R * (m + 2) * GM_RB;
  d.small = p; p += (size_t)R * SM;
  d.resbuf = p; p += R;
  d.jdev = (int*)p;
  return LB_OK;
}

static LkAct make_act(const std::vector<int>& sys) {
  LkAct a{};
  a.n = (int)sys.size();
  for (int k = 0; k < a.n; ++k) a.r[k] = sys[k];
  return a;
}

// squared norms |v_r|^2 of the listed systems into their scalars [4];
// returns the norms on the host
static int lk_norms(lb_ctx* c, Lockstep& L, const double* v, const std::vector<int>& sys, std::vector<double>* out) {
  if (sys.empty()) { out->clear(); return LB_OK; }
  const LkAct act = make_act(sys);
  LkDev d = L.d;
  k_lk_dots<<<dim3(GM_RB, act.n), 256, 0, c->stream>>>(d, act, v, 1);
  LB_LAUNCH(c);
  k_lk_reduce<<<dim3(1, act.n), 64, 0, c->stream>>>(d, act, 1, LK_SC(d) + 4, GM_RB);
  LB_LAUNCH(c);
  for (int a = 0; a < act.n; ++a)
    LB_CUDA(c, cudaMemcpyAsync(c->host_pinned + a, d.small + (int64_t)act.r[a] * d.SM + LK_SC(d) + 4, sizeof(double),
                               cudaMemcpyDeviceToHost, c->stream));
  LB_CUDA(c, cudaStreamSynchronize(c->stream));
  out->resize(act.n);
  for (int a = 0; a < act.n; ++a) (*out)[a] = sqrt(c->host_pinned[a]);
  return LB_OK;
}

// the norms_of helper of the refinement: v [R][N], listed systems
static int norms_of(lb_ctx* c, Lockstep& L, const double* v, const std::vector<int>& sys, std::vector<double>* out) {
  // lk_norms reads row a of its input for system act[a]: gather the rows
  // into L.in first when they are not already in system order
  bool ident = true;
  for (size_t a = 0; a < sys.size(); ++a) ident = ident && sys[a] == (int)a;
  if (ident) return lk_norms(c, L, v, sys, out);
  for (size_t a = 0; a < sys.size(); ++a)
    LB_CUDA(c, cudaMemcpyAsync(L.in + (int64_t)a * c->N, v + (int64_t)sys[a] * c->N, c->N * sizeof(double),
                               cudaMemcpyDeviceToDevice, c->stream));
  return lk_norms(c, L, L.in, sys, out);
}

// dst[a] = src[sys[a]] (rows of N doubles)
static int gather_rows(lb_ctx* c, const double* src, const std::vector<int>& sys, double* dst) {
  for (size_t a = 0; a < sys.size(); ++a)
    LB_CUDA(c, cudaMemcpyAsync(dst + (int64_t)a * c->N, src + (int64_t)sys[a] * c->N, c->N * sizeof(double),
                               cudaMemcpyDeviceToDevice, c->stream));
  return LB_OK;
}

// one lockstep iteration for the active set, enqueued on the context stream
// (direct launches or stream capture); ends with the residual estimates of
// the active systems copied to host_pinned[0..n)
static int lk_iteration(lb_ctx* c, Lockstep& L, int prec, const LkAct& act) {
  const LkDev d = L.d;
  const unsigned nb = vec_blocks(c);
  const dim3 gv(nb, act.n), gd(GM_RB, act.n), gs(lb_div_up(d.m + 2, 64), act.n);
  k_lk_gather<<<gv, 256, 0, c->stream>>>(d, act, L.in);
  LB_LAUNCH(c);
  LB_CHECK(lb_apply_a3_batch(c, prec, act.n, L.in, L.out, nullptr));
  if (d.C) LB_CHECK(lk_project(c, d, act, L.out, -1));  // recycled spaces: B column j = C^T w
  // classical Gram-Schmidt, twice: h = V^T w, w -= V h, y = V^T w, w -= V y, h += y
  k_lk_dots<<<gd, 256, 0, c->stream>>>(d, act, L.out, 0);
  LB_LAUNCH(c);
  k_lk_reduce<<<gs, 64, 0, c->stream>>>(d, act, 0, LK_H(d), GM_RB);
  LB_LAUNCH(c);
  k_lk_axpy<<<gv, 256, 0, c->stream>>>(d, act, L.out, LK_H(d));
  LB_LAUNCH(c);
  k_lk_dots<<<gd, 256, 0, c->stream>>>(d, act, L.out, 0);
  LB_LAUNCH(c);
  k_lk_reduce<<<gs, 64, 0, c->stream>>>(d, act, 0, LK_Y(d), GM_RB);
  LB_LAUNCH(c);
  k_lk_axpy<<<gv, 256, 0, c->stream>>>(d, act, L.out, LK_Y(d));
  LB_LAUNCH(c);
  k_lk_addsmall<<<gs, 64, 0, c->stream>>>(d, act);
  LB_LAUNCH(c);
  k_lk_dots<<<gd, 256, 0, c->stream>>>(d, act, L.out, 1);
  LB_LAUNCH(c);
  k_lk_reduce<<<dim3(1, act.n), 64, 0, c->stream>>>(d, act, 1, LK_SC(d) + 2, GM_RB);
  LB_LAUNCH(c);
  k_lk_normalize<<<gv, 256, 0, c->stream>>>(d, act, L.out);
  LB_LAUNCH(c);
  k_lk_givens<<<lb_div_up(act.n, 64), 64, 0, c->stream>>>(d, act);
  LB_LAUNCH(c);
  k_lk_advance<<<1, 32, 0, c->stream>>>(d);
  LB_LAUNCH(c);
  LB_CUDA(c, cudaMemcpyAsync(c->host_pinned, d.resbuf, act.n * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  return LB_OK;
}

// A captured iteration, the counters it advances per replay, and the
// profiling events recorded inside it (timed again at every replay).
struct LkGraph {
  lb_ctx* c = nullptr;
  cudaGraphExec_t exec = nullptr;
  int64_t launches = 0, pairs = 0;
  int a32 = 0, a64 = 0;
  std::vector<ProfPending> prof;
  void clear() {
    if (exec) cudaGraphExecDestroy(exec);
    exec = nullptr;
    for (auto& p : prof) { c->ev_pool.push_back(p.a); c->ev_pool.push_back(p.b); }
    prof.clear();
  }
  ~LkGraph() { if (c) clear(); }
};

static int lk_capture(lb_ctx* c, Lockstep& L, int prec, const LkAct& act, LkGraph* g) {
  g->c = c;
  g->clear();
  const int64_t l0 = c->launches, p0 = lb_pair_counter;
  const int a32 = lb_apply32_counter, a64 = lb_apply64_counter;
  // capture on the context's private stream (the caller's stream may be the
  // legacy default stream, which cannot capture); the graph is replayed on
  // the caller's stream, in order with its other work
  if (!c->cap_stream) LB_CUDA(c, cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking));
  cudaStream_t user = c->stream;
  LB_CUDA(c, cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeThreadLocal));
  c->stream = c->cap_stream;
  c->capture_prof = &g->prof;
  c->capturing = true;
  const int rc = lk_iteration(c, L, prec, act);
  c->capturing = false;
  c->capture_prof = nullptr;
  c->stream = user;
  cudaGraph_t graph = nullptr;
  const cudaError_t e = cudaStreamEndCapture(c->cap_stream, &graph);
  // the capture enqueued nothing: its counter increments belong to each replay
  g->launches = c->launches - l0;
  g->pairs = lb_pair_counter - p0;
  g->a32 = lb_apply32_counter - a32;
  g->a64 = lb_apply64_counter - a64;
  c->launches = l0;
  lb_pair_counter = p0;
  lb_apply32_counter = a32;
  lb_apply64_counter = a64;
  if (rc != LB_OK || e != cudaSuccess) {
    if (graph) cudaGraphDestroy(graph);
    return rc != LB_OK ? rc : lb_fail(c, LB_ECUDA, "stream capture of the GMRES iteration failed: %s",
                                      cudaGetErrorString(e));
  }
  const cudaError_t ei = cudaGraphInstantiate(&g->exec, graph, 0);
  cudaGraphDestroy(graph);
  if (ei != cudaSuccess) {
    g->exec = nullptr;
    return lb_fail(c, LB_ECUDA, "graph instantiation failed: %s", cudaGetErrorString(ei));
  }
  return LB_OK;
}

static int lk_replay(lb_ctx* c, LkGraph& g) {
  LB_CUDA(c, cudaGraphLaunch(g.exec, c->stream));
  c->launches += g.launches;
  lb_pair_counter += g.pairs;
  lb_apply32_counter += g.a32;
  lb_apply64_counter += g.a64;
  ++lb_graph_counter;
  return LB_OK;
}

// after a replay has completed: add the times of its profiled launches
static void lk_replay_profile(lb_ctx* c, const LkGraph& g) {
  for (const auto& p : g.prof) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, p.a, p.b) == cudaSuccess && p.cat >= 0 && p.cat < LB_PROF_NCAT) {
      c->prof_ms[p.cat] += ms;
      c->prof_calls[p.cat] += 1;
      c->prof_pairs[p.cat] += p.pairs;
    }
  }
}

// GMRES on R systems at once: b, x [R][N]; systems with b = 0 get x = 0
static int gmres_lockstep(lb_ctx* c, Lockstep& L, int prec, const double* b, double* x, double tol, int max_iter,
                          std::vector<int>* its, std::vector<double>* res, std::vector<double>* hist0,
                          const std::vector<double>* tolscale = nullptr) {
  const int64_t N = c->N;
  const int R = L.R;
  const LkDev d = L.d;
  const unsigned nb = vec_blocks(c);
  its->assign(R, 0);
  res->assign(R, 0.0);
  std::vector<int> all(R);
  for (int r = 0; r < R; ++r) all[r] = r;
  std::vector<double> beta;
  LB_CHECK(lk_norms(c, L, b, all, &beta));
  std::vector<int> act;
  for (int r = 0; r < R; ++r) {
    if (!std::isfinite(beta[r])) return lb_fail(c, LB_EINVAL, "non-finite right-hand side");
    if (beta[r] > 0) act.push_back(r);
    else LB_CUDA(c, cudaMemsetAsync(x + (int64_t)r * N, 0, N * sizeof(double), c->stream));
  }
  if (!act.empty()) {
    const LkAct a0 = make_act(act);
    k_lk_start<<<dim3(nb, a0.n), 256, 0, c->stream>>>(d, a0, b);
    LB_LAUNCH(c);
  }
  LB_CUDA(c, cudaMemsetAsync(d.jdev, 0, sizeof(int), c->stream));
  if (hist0 && R > 0 && beta[0] > 0) hist0->push_back(1.0);
  // graphs replay from the second iteration on: the first, launched
  // directly, sizes every workspace the apply needs
  bool use_graphs = c->params.graphs != 0;
  LkGraph graph;
  std::vector<int> captured;
  for (int j = 0; j < max_iter && !act.empty(); ++j) {
    const LkAct a = make_act(act);
    bool done = false;
    if (use_graphs && j > 0) {
      if (captured != act) {
        if (lk_capture(c, L, prec, a, &graph) == LB_OK) {
          captured = act;
        } else {  // capture refused: plain launches from here on
          cudaGetLastError();
          use_graphs = false;
        }
      }
      if (use_graphs) {
        LB_CHECK(lk_replay(c, graph));
        done = true;
      }
    }
    if (!done) LB_CHECK(lk_iteration(c, L, prec, a));
    LB_CUDA(c, cudaStreamSynchronize(c->stream));
    if (done) lk_replay_profile(c, graph);
    std::vector<int> next;
    for (int k = 0; k < a.n; ++k) {
      const int r = act[k];
      const double rr = c->host_pinned[k];
      if (!std::isfinite(rr)) return lb_fail(c, LB_EINVAL, "GMRES breakdown: non-finite residual");
      (*its)[r] = j + 1;
      (*res)[r] = rr;
      if (hist0 && r == 0) hist0->push_back(rr);
      if (!(rr < tol * (tolscale ? (*tolscale)[r] : 1.0) || rr == 0.0)) next.push_back(r);
    }
    act.swap(next);
  }
  for (int r = 0; r < R; ++r) {
    if (!(beta[r] > 0)) continue;
    k_lk_backsolve<<<1, 32, 0, c->stream>>>(d, r, (*its)[r]);
    LB_LAUNCH(c);
    k_combine<<<nb, 256, 0, c->stream>>>(N, (*its)[r], d.V + (int64_t)r * N, (int64_t)R * N,
                                         d.small + (int64_t)r * d.SM + LK_Y(d), x + (int64_t)r * N, 0);
    LB_LAUNCH(c);
  }
  return LB_OK;
}

// The lockstep refinement recycles each system's first inner Krylov space
// as the single solve does (recycle_capture, gmres_recycled): per original
// system its basis V (k + 1 vectors), C = V Q (k vectors) and R, kept in
// ws_rec for the later stages, whose batched iterations project every new
// vector against C (lk_project) and record B = C^T A V2.
struct LkRecycle {
  int R = 0, m = 0, kmax = 0;
  std::vector<int> k;          // per original system, 0: nothing recycled
  std::vector<int64_t> voff;   // offsets of V and C in ws_rec
  std::vector<int64_t> coff;
  std::vector<std::vector<double>> Rm;  // k x k upper triangles, column-major
  double* base = nullptr;
  int64_t* dcoff = nullptr;    // device: per stage-2 system
  int* dck = nullptr;
  double* Bm = nullptr;        // device: per stage-2 system (m + 2) kmax coefficients
  double* coef = nullptr;      // device: kmax closing coefficients
};

// after the first lockstep stage of the systems act (stage index a ~ act[a])
static int lk_recycle_capture(lb_ctx* c, Lockstep& La, const std::vector<int>& act, const std::vector<int>& its,
                              int R, int m, LkRecycle* rc) {
  const int64_t N = c->N;
  const int Ra = (int)act.size();
  rc->R = R;
  rc->m = m;
  rc->k.assign(R, 0);
  rc->voff.assign(R, 0);
  rc->coff.assign(R, 0);
  rc->Rm.assign(R, {});
  int64_t tot = 0;
  int kmax = 1;
  for (int a = 0; a < Ra; ++a) {
    tot += (int64_t)(2 * its[a] + 1) * N;
    kmax = std::max(kmax, its[a]);
  }
  rc->kmax = kmax;
  // layout (doubles): V and C of every system [tot], Q [qn], the closing
  // coefficients [kmax], the stage blocks [R (m + 2) kmax], then R int64
  // offsets and R ints
  const int64_t qn = (int64_t)(kmax + 1) * kmax;
  const size_t need = (size_t)tot + (size_t)qn + (size_t)kmax + (size_t)R * (m + 2) * kmax + (size_t)R * 2 + 16;
  LB_CHECK(lb_ensure(c, c->ws_rec, need * sizeof(double)));
  double* p = (double*)c->ws_rec.p;
  rc->base = p;
  double* Qd = p + tot;
  rc->coef = Qd + qn;
  rc->Bm = rc->coef + kmax;
  rc->dcoff = (int64_t*)(rc->Bm + (size_t)R * (m + 2) * kmax);
  rc->dck = (int*)(rc->dcoff + R);
  const LkDev& d = La.d;
  const unsigned nb = vec_blocks(c);
  int64_t off = 0;
  std::vector<double> small(d.SM);
  for (int a = 0; a < Ra; ++a) {
    const int k = its[a], r = act[a];
    if (k < 1) continue;
    LB_CUDA(c, cudaMemcpyAsync(small.data(), d.small + (int64_t)a * d.SM, d.SM * sizeof(double),
                               cudaMemcpyDeviceToHost, c->stream));
    LB_CUDA(c, cudaStreamSynchronize(c->stream));
    const double* Hm = small.data() + LK_HM(d);
    const double* cs = small.data() + LK_CS(d);
    const double* sn = small.data() + LK_SN(d);
    std::vector<double> Rk((size_t)k * k, 0.0);
    bool ok = true;
    for (int l = 0; l < k; ++l)
      for (int i = 0; i <= l; ++i) Rk[(size_t)l * k + i] = Hm[(size_t)l * d.ldh + i];
    for (int i = 0; i < k; ++i) ok = ok && std::fabs(Rk[(size_t)i * k + i]) > 0;
    if (!ok) continue;  // breakdown: this system restarts plainly
    std::vector<double> Q((size_t)(k + 1) * k, 0.0);
    for (int l = 0; l < k; ++l) Q[(size_t)l * (k + 1) + l] = 1.0;
    for (int j = k - 1; j >= 0; --j)
      for (int l = 0; l < k; ++l) {
        double* q = &Q[(size_t)l * (k + 1)];
        const double x0 = q[j], x1 = q[j + 1];
        q[j] = cs[j] * x0 - sn[j] * x1;
        q[j + 1] = sn[j] * x0 + cs[j] * x1;
      }
    double* V = p + off;
    double* C = V + (int64_t)(k + 1) * N;
    for (int v = 0; v <= k; ++v)
      LB_CUDA(c, cudaMemcpyAsync(V + (int64_t)v * N, d.V + ((int64_t)v * d.R + a) * N, N * sizeof(double),
                                 cudaMemcpyDeviceToDevice, c->stream));
    LB_CUDA(c, cudaMemcpyAsync(Qd, Q.data(), Q.size() * sizeof(double), cudaMemcpyHostToDevice, c->stream));
    for (int l = 0; l < k; ++l) {
      k_combine<<<nb, 256, 0, c->stream>>>(N, k + 1, V, N, Qd + (size_t)l * (k + 1), C + (int64_t)l * N, 0);
      LB_LAUNCH(c);
    }
    LB_CUDA(c, cudaStreamSynchronize(c->stream));  // Q (host) is reused for the next system
    rc->k[r] = k;
    rc->voff[r] = off;
    rc->coff[r] = off + (int64_t)(k + 1) * N;
    rc->Rm[r] = std::move(Rk);
    off += (int64_t)(2 * k + 1) * N;
  }
  return LB_OK;
}

// attach the recycled spaces of the systems act to a stage's lockstep; false
// when one of them has none (that stage then restarts plainly)
static int lk_recycle_attach(lb_ctx* c, const LkRecycle& rc, const std::vector<int>& act, Lockstep& La, bool* on) {
  *on = false;
  if (rc.k.empty()) return LB_OK;
  for (int r : act)
    if (rc.k[r] < 1) return LB_OK;
  const int Ra = (int)act.size();
  std::vector<int64_t> co(Ra);
  std::vector<int> ck(Ra);
  for (int a = 0; a < Ra; ++a) {
    co[a] = rc.coff[act[a]];
    ck[a] = rc.k[act[a]];
  }
  LB_CUDA(c, cudaMemcpyAsync(rc.dcoff, co.data(), Ra * sizeof(int64_t), cudaMemcpyHostToDevice, c->stream));
  LB_CUDA(c, cudaMemcpyAsync(rc.dck, ck.data(), Ra * sizeof(int), cudaMemcpyHostToDevice, c->stream));
  LB_CUDA(c, cudaStreamSynchronize(c->stream));
  LkDev& d = La.d;
  d.C = rc.base;
  d.coff = rc.dcoff;
  d.ck = rc.dck;
  d.Bm = rc.Bm;
  d.kmax = rc.kmax;
  d.bld = (int64_t)(d.m + 2) * rc.kmax;
  *on = true;
  return LB_OK;
}

// x_a += V_a R_a^-1 (alpha_a - B_a y_a) for every system of a recycled stage
static int lk_recycle_close(lb_ctx* c, const LkRecycle& rc, const std::vector<int>& act, Lockstep& La,
                            const std::vector<int>& its, double* x) {
  const int64_t N = c->N;
  const LkDev& d = La.d;
  const unsigned nb = vec_blocks(c);
  double* coef = rc.coef;
  for (size_t a = 0; a < act.size(); ++a) {
    const int r = act[a], k = rc.k[r], kk = its[a];
    std::vector<double> blk((size_t)d.bld), y(std::max(kk, 1)), cu(k);
    LB_CUDA(c, cudaMemcpyAsync(blk.data(), rc.Bm + (int64_t)a * d.bld, d.bld * sizeof(double),
                               cudaMemcpyDeviceToHost, c->stream));
    if (kk > 0)
      LB_CUDA(c, cudaMemcpyAsync(y.data(), d.small + (int64_t)a * d.SM + LK_Y(d), kk * sizeof(double),
                                 cudaMemcpyDeviceToHost, c->stream));
    LB_CUDA(c, cudaStreamSynchronize(c->stream));
    const double* alpha = blk.data() + (size_t)(d.m + 1) * d.kmax;
    for (int i = 0; i < k; ++i) {
      double z = alpha[i];
      for (int j = 0; j < kk; ++j) z -= blk[(size_t)j * d.kmax + i] * y[j];
      cu[i] = z;
    }
    const std::vector<double>& Rk = rc.Rm[r];
    for (int i = k - 1; i >= 0; --i) {
      double sum = cu[i];
      for (int l = i + 1; l < k; ++l) sum -= Rk[(size_t)l * k + i] * cu[l];
      cu[i] = sum / Rk[(size_t)i * k + i];
    }
    LB_CUDA(c, cudaMemcpyAsync(coef, cu.data(), k * sizeof(double), cudaMemcpyHostToDevice, c->stream));
    k_combine<<<nb, 256, 0, c->stream>>>(N, k, rc.base + rc.voff[r], N, coef, x + (int64_t)a * N, 1);
    LB_LAUNCH(c);
    LB_CUDA(c, cudaStreamSynchronize(c->stream));  // cu (host) is reused
  }
  return LB_OK;
}

// R mean-zero right-hand sides b [R][N] -> densities sigma and potentials u
// (A3, u = S[S[sigma]]), precision LB_FP32, LB_DF64 or LB_FP32_REFINED.
static int solve_lockstep(lb_ctx* c, int R, const double* b, double* sigma, double* u, lb_solve_info* info,
                          bool first) {
  const int64_t N = c->N;
  const lb_params& p = c->params;
  const unsigned nb = vec_blocks(c);
  const int64_t RN = (int64_t)R * N;
  Lockstep L;
  LB_CHECK(lockstep_work(c, R, p.max_iter, &L));
  LB_CHECK(lb_ensure(c, c->ws_bvec, (size_t)(8 * RN) * sizeof(double)));
  double* r = (double*)c->ws_bvec.p;  // residuals [R][N]
  double* delta = r + RN;             // corrections (gathered) [Ra][N]
  double* Ax = delta + RN;            // apply output (gathered)
  double* x1 = Ax + RN;               // first iterates
  double* ux1 = x1 + RN;              // their double-float potentials S[S[x1]]
  double* tmp = ux1 + RN;
  double* rin = tmp + RN;             // gathered residuals
  double* uacc = rin + RN;            // float32 solution potentials of x - x1
  std::vector<double> hist;
  std::vector<int> its;
  std::vector<double> res;
  if (p.precision != LB_FP32_REFINED) {
    LB_CHECK(gmres_lockstep(c, L, p.precision, b, sigma, p.tol, p.max_iter, &its, &res, &hist));
    for (int k = 0; k < R; ++k) {
      info->iterations += its[k];
      info->converged = info->converged && (res[k] < p.tol);
      info->rel_residual = std::max(info->rel_residual, res[k]);
    }
    // u = S[S[sigma]] in the solve's own pair arithmetic
    LB_CHECK(lb_apply_s_batch(c, p.precision, R, sigma, tmp));
    LB_CHECK(lb_apply_s_batch(c, p.precision, R, tmp, u));
  } else {
    std::vector<int> all(R);
    for (int k = 0; k < R; ++k) all[k] = k;
    std::vector<double> nbv;
    LB_CHECK(norms_of(c, L, b, all, &nbv));
    LB_CUDA(c, cudaMemsetAsync(sigma, 0, RN * sizeof(double), c->stream));
    LB_CUDA(c, cudaMemsetAsync(x1, 0, RN * sizeof(double), c->stream));
    LB_CUDA(c, cudaMemsetAsync(ux1, 0, RN * sizeof(double), c->stream));
    LB_CUDA(c, cudaMemsetAsync(uacc, 0, RN * sizeof(double), c->stream));
    LB_CUDA(c, cudaMemcpyAsync(r, b, RN * sizeof(double), cudaMemcpyDeviceToDevice, c->stream));
    std::vector<int> act;
    std::vector<double> rel(R, 0.0);
    std::vector<int> steps(R, 0), itsum(R, 0);
    for (int k = 0; k < R; ++k) {
      if (nbv[k] != 0.0) { act.push_back(k); rel[k] = 1.0; }
    }
    if (R > 0 && nbv[0] != 0.0) hist.push_back(1.0);
    LkRecycle rec;
    for (int s = 0; s < p.max_refine && !act.empty(); ++s) {
      const int Ra = (int)act.size();
      LB_CHECK(gather_rows(c, r, act, rin));
      Lockstep La;
      LB_CHECK(lockstep_work(c, Ra, p.max_iter, &La));
      bool recycled = false;
      if (s > 0) LB_CHECK(lk_recycle_attach(c, rec, act, La, &recycled));
      if (recycled) {
        // project the residuals off C (alpha = C^T r into slot m + 1); the
        // inner tolerance stays relative to the unprojected |r|
        std::vector<int> idx(Ra);
        for (int a = 0; a < Ra; ++a) idx[a] = a;
        std::vector<double> before, after;
        LB_CHECK(lk_norms(c, La, rin, idx, &before));
        LB_CHECK(lk_project(c, La.d, make_act(idx), rin, La.d.m + 1));
        LB_CHECK(lk_norms(c, La, rin, idx, &after));
        std::vector<double> scale(Ra, 1.0);
        for (int a = 0; a < Ra; ++a) scale[a] = after[a] > 0 ? before[a] / after[a] : 1.0;
        LB_CHECK(gmres_lockstep(c, La, LB_FP32, rin, delta, p.inner_tol, p.max_iter, &its, &res, nullptr, &scale));
        LB_CHECK(lk_recycle_close(c, rec, act, La, its, delta));
      } else {
        LB_CHECK(gmres_lockstep(c, La, LB_FP32, rin, delta, p.inner_tol, p.max_iter, &its, &res, nullptr));
      }
      if (s == 0) LB_CHECK(lk_recycle_capture(c, La, act, its, R, p.max_iter, &rec));
      for (int a = 0; a < Ra; ++a) {
        itsum[act[a]] += its[a];
        k_axpby<<<nb, 256, 0, c->stream>>>(N, 1.0, delta + (int64_t)a * N, 1.0, sigma + (int64_t)act[a] * N);
        LB_LAUNCH(c);
      }
      if (s == 0) {
        // r = b - A x1 in double-float; keep x1 and S[S[x1]]
        LB_CHECK(gather_rows(c, sigma, act, rin));
        LB_CHECK(lb_apply_a3_batch(c, LB_DF64, Ra, rin, Ax, tmp));
        for (int a = 0; a < Ra; ++a) {
          const int64_t o = (int64_t)act[a] * N;
          LB_CUDA(c, cudaMemcpyAsync(ux1 + o, tmp + (int64_t)a * N, N * sizeof(double), cudaMemcpyDeviceToDevice,
                                     c->stream));
          LB_CUDA(c, cudaMemcpyAsync(x1 + o, sigma + o, N * sizeof(double), cudaMemcpyDeviceToDevice, c->stream));
          LB_CUDA(c, cudaMemcpyAsync(r + o, b + o, N * sizeof(double), cudaMemcpyDeviceToDevice, c->stream));
          k_axpby<<<nb, 256, 0, c->stream>>>(N, -1.0, Ax + (int64_t)a * N, 1.0, r + o);
          LB_LAUNCH(c);
        }
      } else {
        // r -= A32 delta: delta is about inner_tol |x|, so float32 pairs keep
        // this update accurate to about 1e-7 inner_tol |b|
        // (the apply also yields S[S[delta]], accumulated for u)
        LB_CHECK(lb_apply_a3_batch(c, LB_FP32, Ra, delta, Ax, tmp));
        for (int a = 0; a < Ra; ++a) {
          k_axpby<<<nb, 256, 0, c->stream>>>(N, -1.0, Ax + (int64_t)a * N, 1.0, r + (int64_t)act[a] * N);
          LB_LAUNCH(c);
          k_axpby<<<nb, 256, 0, c->stream>>>(N, 1.0, tmp + (int64_t)a * N, 1.0, uacc + (int64_t)act[a] * N);
          LB_LAUNCH(c);
        }
      }
      std::vector<double> rn;
      LB_CHECK(norms_of(c, L, r, act, &rn));
      std::vector<int> next;
      for (int a = 0; a < Ra; ++a) {
        const int k = act[a];
        rel[k] = rn[a] / nbv[k];
        ++steps[k];
        if (k == 0) hist.push_back(rel[k]);
        if (!(rel[k] < p.tol)) next.push_back(k);
      }
      act.swap(next);
    }
    for (int k = 0; k < R; ++k) {
      info->iterations += itsum[k];
      info->refinements += steps[k];
      info->converged = info->converged && (rel[k] < p.tol);
      info->rel_residual = std::max(info->rel_residual, rel[k]);
    }
    // u = S[S[x1]] (double-float) + the float32 potentials of the corrections
    LB_CUDA(c, cudaMemcpyAsync(u, ux1, RN * sizeof(double), cudaMemcpyDeviceToDevice, c->stream));
    k_axpby<<<nb, 256, 0, c->stream>>>(RN, 1.0, uacc, 1.0, u);
    LB_LAUNCH(c);
  }
  if (first) {
    info->history_len = (int32_t)std::min<size_t>(hist.size(), 128);
    for (int i = 0; i < info->history_len; ++i) info->history[i] = hist[i];
  }
  return LB_OK;
}

static int solve_batch(lb_ctx* c, int nrhs, const double* f, double* u, lb_solve_info* info) {
  const int64_t N = c->N;
  const lb_params& p = c->params;
  LB_CHECK(lb_ensure(c, c->ws_quad, (size_t)(9 * N) * sizeof(double)));
  double* fb = (double*)c->ws_quad.p;    // projected f, then b
  double* sig = fb + N;
  double* scratch = fb + 2 * N;          // 6 N for refinement
  double* tmp = fb + 8 * N;
  // solution potentials of the plain modes in their own pair arithmetic
  const int post = p.precision == LB_FP32 ? LB_FP32 : (p.precision == LB_FP64 ? LB_FP64 : LB_DF64);
  // the finite-check flag lives in ws_red, which later applies may grow:
  // its address is taken afresh before every use
  auto bad_flag = [&](int** d) {
    LB_CHECK(lb_ensure(c, c->ws_red, 8192));
    *d = (int*)((char*)c->ws_red.p + 8192 - 64);
    return LB_OK;
  };
  int* dbad = nullptr;
  if (p.formulation == LB_A3 && p.precision != LB_FP64 && nrhs >= 2 && !c->far_order) {
    // several right-hand sides in lockstep, in groups of LB_BATCH_MAX
    lb_solve_info local{};
    if (!info) { local.converged = 1; info = &local; }
    for (int r0 = 0; r0 < nrhs; r0 += LB_BATCH_MAX) {
      const int R = std::min(LB_BATCH_MAX, nrhs - r0);
      LB_CHECK(lb_ensure(c, c->ws_quad, (size_t)(2 * R * N) * sizeof(double)));
      double* bg = (double*)c->ws_quad.p;
      double* sg = bg + (int64_t)R * N;
      for (int k = 0; k < R; ++k) {
        const double* fr = f + (int64_t)(r0 + k) * N;
        LB_CHECK(bad_flag(&dbad));
        LB_CUDA(c, cudaMemsetAsync(dbad, 0, sizeof(int), c->stream));
        k_check_finite<<<vec_blocks(c), 256, 0, c->stream>>>(N, fr, dbad);
        LB_LAUNCH(c);
        int bad = 0;
        LB_CUDA(c, cudaMemcpyAsync(&bad, dbad, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
        LB_CUDA(c, cudaStreamSynchronize(c->stream));
        if (bad) return lb_fail(c, LB_EINVAL, "right-hand side %d has non-finite entries", r0 + k);
        double removed = 0;
        LB_CHECK(project_mean_zero(c, fr, bg + (int64_t)k * N, &removed));
        if (r0 + k == 0) info->removed_mean = removed;
      }
      LB_CHECK(solve_lockstep(c, R, bg, sg, u + (int64_t)r0 * N, info, r0 == 0));
    }
    return LB_OK;
  }
  for (int r = 0; r < nrhs; ++r) {
    const double* fr = f + (int64_t)r * N;
    LB_CHECK(bad_flag(&dbad));
    LB_CUDA(c, cudaMemsetAsync(dbad, 0, sizeof(int), c->stream));
    k_check_finite<<<vec_blocks(c), 256, 0, c->stream>>>(N, fr, dbad);
    LB_LAUNCH(c);
    int bad = 0;
    LB_CUDA(c, cudaMemcpyAsync(&bad, dbad, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    LB_CUDA(c, cudaStreamSynchronize(c->stream));
    if (bad) return lb_fail(c, LB_EINVAL, "right-hand side %d has non-finite entries", r);
    double removed = 0;
    LB_CHECK(project_mean_zero(c, fr, fb, &removed));
    if (info && r == 0) info->removed_mean = removed;
    if (p.formulation != LB_A3) {  // A1, A2: b = S[f]
      LB_CHECK(apply_S_dev(c, post, fb, tmp));
      LB_CUDA(c, cudaMemcpyAsync(fb, tmp, N * sizeof(double), cudaMemcpyDeviceToDevice, c->stream));
    }
    double* ur = u + (int64_t)r * N;
    LB_CHECK(solve_one(c, fb, sig, scratch, info, r == 0, ur));
    if (p.precision == LB_FP32_REFINED) continue;  // u produced by the refinement
    if (p.formulation == LB_A3) {  // u = S[S[sigma]]
      LB_CHECK(apply_S_dev(c, post, sig, tmp));
      LB_CHECK(apply_S_dev(c, post, tmp, ur));
    } else {
      LB_CHECK(apply_S_dev(c, post, sig, ur));
    }
  }
  return LB_OK;
}

extern "C" int lb_solve_lb(lb_ctx* c, int nrhs, const double* f, double* u, lb_solve_info* info) {
  LB_CHECK(lb_require_corr(c));
  if (nrhs < 1) return lb_fail(c, LB_EINVAL, "nrhs must be >= 1");
  LB_CUDA(c, cudaSetDevice(c->device));
  const int64_t N = c->N;
  if (info) {
    *info = lb_solve_info{};
    info->converged = 1;
    info->nrhs = nrhs;
  }
  lb_pair_counter = 0;
  lb_apply64_counter = lb_apply32_counter = 0;
  lb_graph_counter = 0;
  const double* din;
  double* dout;
  LB_CHECK(lb_stage_in(c, f, nrhs * N * sizeof(double), c->ws_stage_in, (const void**)&din));
  LB_CHECK(lb_stage_out(c, u, nrhs * N * sizeof(double), c->ws_stage_out, (void**)&dout));
  LB_CHECK(solve_batch(c, nrhs, din, dout, info));
  LB_CHECK(lb_stage_out_finish(c, u, dout, nrhs * N * sizeof(double)));
  if (info) {
    info->pairs = lb_pair_counter;
    info->applies_fp64 = lb_apply64_counter;
    info->applies_fp32 = lb_apply32_counter;
    info->graph_iterations = lb_graph_counter;
    LB_CUDA(c, cudaStreamSynchronize(c->stream));
    if (!info->converged) return lb_fail(c, LB_ENOTCONVERGED, "GMRES did not reach tol %.3g (residual %.3g)",
                                         c->params.tol, info->rel_residual);
  }
  return LB_OK;
}

// ---------------------------------------------------------------------------
// surface gradient and divergence by nodal differentiation (Section 2)

__global__ void k_surf_grad(int64_t N, int np, const double* __restrict__ f, const double* __restrict__ Du,
                            const double* __restrict__ Dv, const double* __restrict__ ginv,
                            const double* __restrict__ Xu, const double* __restrict__ Xv,
                            const double* __restrict__ add_n, const double* __restrict__ nrm,
                            double* __restrict__ out) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= N) return;
  const int64_t P = i / np;
  const int q = (int)(i - P * np);
  double fu = 0, fv = 0;
  for (int b = 0; b < np; ++b) {
    const double x = f[P * np + b];
    fu += Du[q * np + b] * x;
    fv += Dv[q * np + b] * x;
  }
  const double a = ginv[3 * i] * fu + ginv[3 * i + 1] * fv;
  const double bb = ginv[3 * i + 1] * fu + ginv[3 * i + 2] * fv;
  for (int k = 0; k < 3; ++k) {
    double g = a * Xu[3 * i + k] + bb * Xv[3 * i + k];
    if (add_n) g += add_n[i] * nrm[3 * i + k];
    out[3 * i + k] = g;
  }
}

// P1 = J F^1, P2 = J F^2 with F^a = g^ab (F . X_b); cross_n: use n x F instead of F
__global__ void k_div_prep(int64_t N, const double* __restrict__ F, int cross_n, const double* __restrict__ nrm,
                           const double* __restrict__ ginv, const double* __restrict__ Xu,
                           const double* __restrict__ Xv, const double* __restrict__ J, double* __restrict__ P) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= N) return;
  double v[3] = {F[3 * i], F[3 * i + 1], F[3 * i + 2]};
  if (cross_n) {
    const double* n = nrm + 3 * i;
    const double c0 = n[1] * v[2] - n[2] * v[1], c1 = n[2] * v[0] - n[0] * v[2], c2 = n[0] * v[1] - n[1] * v[0];
    v[0] = c0; v[1] = c1; v[2] = c2;
  }
  const double a = v[0] * Xu[3 * i] + v[1] * Xu[3 * i + 1] + v[2] * Xu[3 * i + 2];
  const double b = v[0] * Xv[3 * i] + v[1] * Xv[3 * i + 1] + v[2] * Xv[3 * i + 2];
  P[i] = J[i] * (ginv[3 * i] * a + ginv[3 * i + 1] * b);
  P[N + i] = J[i] * (ginv[3 * i + 1] * a + ginv[3 * i + 2] * b);
}

__global__ void k_div_finish(int64_t N, int np, const double* __restrict__ P, const double* __restrict__ Du,
                             const double* __restrict__ Dv, const double* __restrict__ J, double scale,
                             double* __restrict__ out) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= N) return;
  const int64_t p = i / np;
  const int q = (int)(i - p * np);
  double s = 0;
  for (int b = 0; b < np; ++b) s += Du[q * np + b] * P[p * np + b] + Dv[q * np + b] * P[N + p * np + b];
  out[i] = scale * s / J[i];
}

static int surface_div_dev(lb_ctx* c, const double* F, int cross_n, double scale, double* out) {
  LB_CHECK(lb_ensure(c, c->ws_vec, (size_t)(4 * c->N) * sizeof(double)));
  double* P = (double*)c->ws_vec.p;
  k_div_prep<<<lb_div_up(c->N, 128), 128, 0, c->stream>>>(c->N, F, cross_n, c->nrm, c->ginv, c->Xu, c->Xv, c->J, P);
  LB_LAUNCH(c);
  k_div_finish<<<lb_div_up(c->N, 128), 128, 0, c->stream>>>(c->N, c->np, P, c->dDu, c->dDv, c->J, scale, out);
  LB_LAUNCH(c);
  return LB_OK;
}

extern "C" int lb_surface_div(lb_ctx* c, int nrhs, const double* F, double* out) {
  if (!c) return lb_fail(nullptr, LB_EINVAL, "null context");
  if (!c->have_geom) return lb_fail(c, LB_ESTATE, "no geometry uploaded");
  if (nrhs < 1) return lb_fail(c, LB_EINVAL, "nrhs must be >= 1");
  LB_CUDA(c, cudaSetDevice(c->device));
  const int64_t N = c->N;
  const double* din;
  double* dout;
  LB_CHECK(lb_stage_in(c, F, nrhs * 3 * N * sizeof(double), c->ws_stage_in, (const void**)&din));
  LB_CHECK(lb_stage_out(c, out, nrhs * N * sizeof(double), c->ws_stage_out, (void**)&dout));
  for (int r = 0; r < nrhs; ++r) LB_CHECK(surface_div_dev(c, din + (int64_t)r * 3 * N, 0, 1.0, dout + r * N));
  return lb_stage_out_finish(c, out, dout, nrhs * N * sizeof(double));
}

extern "C" int lb_apply_gradS(lb_ctx* c, int nrhs, const double* sigma, double* out) {
  LB_CHECK(lb_require_corr(c));
  if (nrhs < 1) return lb_fail(c, LB_EINVAL, "nrhs must be >= 1");
  LB_CUDA(c, cudaSetDevice(c->device));
  const int64_t N = c->N;
  const double* din;
  double* dout;
  LB_CHECK(lb_stage_in(c, sigma, nrhs * N * sizeof(double), c->ws_stage_in, (const void**)&din));
  LB_CHECK(lb_stage_out(c, out, nrhs * 3 * N * sizeof(double), c->ws_stage_out, (void**)&dout));
  LB_CHECK(lb_ensure(c, c->ws_quad, (size_t)(4 * N) * sizeof(double)));
  double* pot = (double*)c->ws_quad.p;
  const int pp = c->params.precision;
  const int prec = (pp == LB_FP64 || pp == LB_DF64) ? pp : LB_FP32;
  for (int r = 0; r < nrhs; ++r) {
    LB_CHECK(lb_potentials(c, prec, din + r * N, pot, (1u << LB_K_S) | (1u << LB_K_SP)));
    k_surf_grad<<<lb_div_up(N, 128), 128, 0, c->stream>>>(N, c->np, pot, c->dDu, c->dDv, c->ginv, c->Xu, c->Xv,
                                                            pot + 2 * N, c->nrm, dout + (int64_t)r * 3 * N);
    LB_LAUNCH(c);
  }
  return lb_stage_out_finish(c, out, dout, nrhs * 3 * N * sizeof(double));
}

// ---------------------------------------------------------------------------
// A1 = div S grad_Gamma S + S W S (Section 4.1, eq. ie-dis0), applied right
// to left: s = S[tau]; mu = grad_Gamma s by nodal differentiation; the vector
// single layer of mu and its divergence sum_l d_l S[mu_l], each d_l S[sigma]
// the principal-value gradient n_l S'[sigma] + (grad_Gamma S[sigma])_l; plus
// W[s] S[1], with S[1] computed once per pair precision.

// g [N][3] -> out [3][N]
__global__ void k_vec_split(int64_t N, const double* __restrict__ g, double* __restrict__ out) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x)
    for (int k = 0; k < 3; ++k) out[k * N + i] = g[3 * i + k];
}

// div (+)= component l of the gradient g [N][3]
__global__ void k_a1_acc(int64_t N, int l, const double* __restrict__ g, double* __restrict__ div) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x)
    div[i] = (l == 0 ? 0.0 : div[i]) + g[3 * i + l];
}

// out = div + (sum of the w s partials / area) S[1]
__global__ void k_a1_final(int64_t N, const double* __restrict__ div, const double* __restrict__ phi0,
                           const double* __restrict__ partial, int npart, double area, double* __restrict__ out) {
  __shared__ double eta;
  if (threadIdx.x == 0) {
    double s = 0;
    for (int k = 0; k < npart; ++k) s += partial[k];
    eta = s / area;
  }
  __syncthreads();
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = div[i] + eta * phi0[i];
}

__global__ void k_fill(int64_t N, double v, double* __restrict__ x) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x)
    x[i] = v;
}

int lb_apply_a1(lb_ctx* c, int prec, const double* tau, double* out) {
  const int64_t N = c->N;
  const unsigned nb = vec_blocks(c), gb = lb_div_up(N, 128);
  LB_CHECK(lb_ensure(c, c->ws_pot, (size_t)(8 * N) * sizeof(double)));
  LB_CHECK(lb_ensure(c, c->ws_a1, (size_t)(15 * N + GM_RB) * sizeof(double)));
  double* pot = (double*)c->ws_pot.p;      // [4][N]: S[tau] at K_S
  double* a = (double*)c->ws_a1.p;
  double* mu = a;                          // [N][3]
  double* mus = mu + 3 * N;                // [3][N]
  double* potl = mus + 3 * N;              // [4][N]
  double* grad = potl + 4 * N;             // [N][3]
  double* div = grad + 3 * N;              // [N]
  double* tmp = div + N;                   // [N]
  double* partial = tmp + N;               // [GM_RB]
  if (!c->phi0 || c->phi0_prec != prec) {  // S[1]
    LB_CHECK(lb_alloc(c, &c->phi0, (size_t)N));
    k_fill<<<nb, 256, 0, c->stream>>>(N, 1.0, tmp);
    LB_LAUNCH(c);
    LB_CHECK(lb_potentials(c, prec, tmp, potl, 1u << LB_K_S));
    LB_CUDA(c, cudaMemcpyAsync(c->phi0, potl + LB_K_S * N, N * sizeof(double), cudaMemcpyDeviceToDevice,
                               c->stream));
    c->phi0_prec = prec;
  }
  LB_CHECK(lb_potentials(c, prec, tau, pot, 1u << LB_K_S));
  const double* s = pot + LB_K_S * N;
  k_surf_grad<<<gb, 128, 0, c->stream>>>(N, c->np, s, c->dDu, c->dDv, c->ginv, c->Xu, c->Xv, nullptr, c->nrm, mu);
  LB_LAUNCH(c);
  k_vec_split<<<nb, 256, 0, c->stream>>>(N, mu, mus);
  LB_LAUNCH(c);
  for (int l = 0; l < 3; ++l) {
    LB_CHECK(lb_potentials(c, prec, mus + l * N, potl, (1u << LB_K_S) | (1u << LB_K_SP)));
    k_surf_grad<<<gb, 128, 0, c->stream>>>(N, c->np, potl + LB_K_S * N, c->dDu, c->dDv, c->ginv, c->Xu, c->Xv,
                                            potl + LB_K_SP * N, c->nrm, grad);
    LB_LAUNCH(c);
    k_a1_acc<<<nb, 256, 0, c->stream>>>(N, l, grad, div);
    LB_LAUNCH(c);
  }
  k_multidot<<<GM_RB, 256, 0, c->stream>>>(N, 1, s, N, c->w, partial);
  LB_LAUNCH(c);
  k_a1_final<<<nb, 256, 0, c->stream>>>(N, div, c->phi0, partial, GM_RB, c->area, out);
  LB_LAUNCH(c);
  if (prec == LB_FP32) ++lb_apply32_counter; else ++lb_apply64_counter;
  return LB_OK;
}

// H = F - grad a - n x grad b, and n x H
__global__ void k_hodge(int64_t N, const double* __restrict__ F, const double* __restrict__ ga,
                        const double* __restrict__ gb, const double* __restrict__ nrm, double* __restrict__ H,
                        double* __restrict__ nH) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= N) return;
  const double* n = nrm + 3 * i;
  const double* b = gb + 3 * i;
  const double nb0 = n[1] * b[2] - n[2] * b[1], nb1 = n[2] * b[0] - n[0] * b[2], nb2 = n[0] * b[1] - n[1] * b[0];
  const double h0 = F[3 * i] - ga[3 * i] - nb0;
  const double h1 = F[3 * i + 1] - ga[3 * i + 1] - nb1;
  const double h2 = F[3 * i + 2] - ga[3 * i + 2] - nb2;
  H[3 * i] = h0; H[3 * i + 1] = h1; H[3 * i + 2] = h2;
  nH[3 * i] = n[1] * h2 - n[2] * h1;
  nH[3 * i + 1] = n[2] * h0 - n[0] * h2;
  nH[3 * i + 2] = n[0] * h1 - n[1] * h0;
}

extern "C" int lb_harmonic_fields(lb_ctx* c, int nF, const double* F, double* H, lb_solve_info* info) {
  LB_CHECK(lb_require_corr(c));
  if (nF < 1) return lb_fail(c, LB_EINVAL, "nF must be >= 1");
  LB_CUDA(c, cudaSetDevice(c->device));
  const int64_t N = c->N;
  const double* dF;
  double* dH;
  LB_CHECK(lb_stage_in(c, F, nF * 3 * N * sizeof(double), c->ws_stage_in, (const void**)&dF));
  LB_CHECK(lb_stage_out(c, H, 2 * nF * 3 * N * sizeof(double), c->ws_stage_out, (void**)&dH));
  // per field: rhs (2N), potentials (2N), gradients (6N)
  size_t need = (size_t)(2 * N * nF + 2 * N * nF + 6 * N) * sizeof(double);
  void* mem = nullptr;
  if (lb_alloc_fails_now(c) || cudaMalloc(&mem, need) != cudaSuccess) {
    cudaGetLastError();
    return lb_fail(c, LB_ENOMEM, "harmonic-field workspace");
  }
  double* rhs = (double*)mem;                 // [2 nF][N]
  double* pots = rhs + 2 * N * nF;            // [2 nF][N]
  double* grads = pots + 2 * N * nF;          // [2][N][3]
  int rc = LB_OK;
  for (int k = 0; k < nF && rc == LB_OK; ++k) {
    rc = surface_div_dev(c, dF + (int64_t)k * 3 * N, 0, 1.0, rhs + (int64_t)(2 * k) * N);
    if (rc == LB_OK) rc = surface_div_dev(c, dF + (int64_t)k * 3 * N, 1, -1.0, rhs + (int64_t)(2 * k + 1) * N);
  }
  lb_solve_info local{};
  if (rc == LB_OK) {
    if (info) { *info = lb_solve_info{}; info->converged = 1; info->nrhs = 2 * nF; }
    lb_pair_counter = 0;
    lb_apply64_counter = lb_apply32_counter = 0;
    rc = solve_batch(c, 2 * nF, rhs, pots, info ? info : &local);
    if (info) { info->pairs = lb_pair_counter; info->applies_fp64 = lb_apply64_counter; info->applies_fp32 = lb_apply32_counter; }
  }
  for (int k = 0; k < nF && rc == LB_OK; ++k) {
    for (int s = 0; s < 2; ++s) {
      k_surf_grad<<<lb_div_up(N, 128), 128, 0, c->stream>>>(N, c->np, pots + (int64_t)(2 * k + s) * N, c->dDu,
                                                              c->dDv, c->ginv, c->Xu, c->Xv, nullptr, c->nrm,
                                                              grads + (int64_t)s * 3 * N);
      ++c->launches;
    }
    k_hodge<<<lb_div_up(N, 128), 128, 0, c->stream>>>(N, dF + (int64_t)k * 3 * N, grads, grads + 3 * N, c->nrm,
                                                        dH + (int64_t)(2 * k) * 3 * N, dH + (int64_t)(2 * k + 1) * 3 * N);
    ++c->launches;
    if (cudaGetLastError() != cudaSuccess) rc = lb_fail(c, LB_ECUDA, "harmonic-field kernel launch failed");
  }
  cudaStreamSynchronize(c->stream);
  cudaFree(mem);
  if (rc != LB_OK) return rc;
  LB_CHECK(lb_stage_out_finish(c, H, dH, 2 * nF * 3 * N * sizeof(double)));
  if (info && !info->converged) return lb_fail(c, LB_ENOTCONVERGED, "GMRES did not converge for a Hodge solve");
  return LB_OK;
}

// ---------------------------------------------------------------------------
// Adjoint of the solve (density gradient): the solve is the linear map
// u = S S A3^-1 P f with P = I - 1 w^T / |Gamma| the weighted mean
// projection, so a gradient g_u of u gives g_f = P^T A3^-T S^T S^T g_u, with
// P^T z = z - w sum(z) / |Gamma|.  Float64 transposed applies and GMRES on A3^T.

// per-block sums of z (fixed order)
__global__ void k_sum_plain(int64_t N, const double* __restrict__ z, double* __restrict__ partial) {
  __shared__ double sh[256];
  double s = 0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x)
    s += z[i];
  sh[threadIdx.x] = s;
  __syncthreads();
  for (int k = blockDim.x / 2; k > 0; k >>= 1) {
    if (threadIdx.x < k) sh[threadIdx.x] += sh[threadIdx.x + k];
    __syncthreads();
  }
  if (threadIdx.x == 0) partial[blockIdx.x] = sh[0];
}

__global__ void k_proj_t(int64_t N, const double* __restrict__ z, const double* __restrict__ w,
                         const double* __restrict__ partial, int npart, double area, double* __restrict__ out) {
  __shared__ double eta;
  if (threadIdx.x == 0) {
    double s = 0;
    for (int k = 0; k < npart; ++k) s += partial[k];
    eta = s / area;
  }
  __syncthreads();
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = z[i] - w[i] * eta;
}

extern "C" int lb_solve_lb_adjoint(lb_ctx* c, int nrhs, const double* gu, double* gf, lb_solve_info* info) {
  LB_CHECK(lb_require_corr(c));
  if (c->far_order) return lb_fail(c, LB_EINVAL, "the adjoint solve uses the node rule: clear the far rule");
  const bool a2 = c->params.formulation == LB_A2;
  if (c->params.formulation != LB_A3 && !a2)
    return lb_fail(c, LB_EINVAL, "the adjoint solve takes the A3 or A2 formulation");
  if (nrhs < 1) return lb_fail(c, LB_EINVAL, "nrhs must be >= 1");
  LB_CUDA(c, cudaSetDevice(c->device));
  const int64_t N = c->N;
  if (info) {
    *info = lb_solve_info{};
    info->converged = 1;
    info->nrhs = nrhs;
  }
  lb_pair_counter = 0;
  lb_apply64_counter = lb_apply32_counter = 0;
  const double* din;
  double* dout;
  LB_CHECK(lb_stage_in(c, gu, nrhs * N * sizeof(double), c->ws_stage_in, (const void**)&din));
  LB_CHECK(lb_stage_out(c, gf, nrhs * N * sizeof(double), c->ws_stage_out, (void**)&dout));
  LB_CHECK(lb_ensure(c, c->ws_quad, (size_t)(3 * N + GM_RB) * sizeof(double)));
  double* t1 = (double*)c->ws_quad.p;
  double* t2 = t1 + N;
  double* z = t2 + N;
  double* partial = z + N;
  const unsigned nb = vec_blocks(c);
  for (int r = 0; r < nrhs; ++r) {
    // A3: solve A3^T z = S^T S^T g_u, g_f = P^T z;
    // A2: solve A2^T z = S^T g_u,     g_f = P^T S^T z
    LB_CHECK(lb_apply_st_dev(c, din + (int64_t)r * N, t1));
    if (a2) LB_CUDA(c, cudaMemcpyAsync(t2, t1, N * sizeof(double), cudaMemcpyDeviceToDevice, c->stream));
    else LB_CHECK(lb_apply_st_dev(c, t1, t2));
    int it = 0;
    double res = 0;
    std::vector<double> hist;
    c->adjoint = true;
    const int rc = gmres(c, LB_FP64, t2, z, c->params.tol, c->params.max_iter, &it, &res, r == 0 ? &hist : nullptr);
    c->adjoint = false;
    LB_CHECK(rc);
    if (a2) {
      LB_CHECK(lb_apply_st_dev(c, z, t1));
      LB_CUDA(c, cudaMemcpyAsync(z, t1, N * sizeof(double), cudaMemcpyDeviceToDevice, c->stream));
    }
    k_sum_plain<<<GM_RB, 256, 0, c->stream>>>(N, z, partial);
    LB_LAUNCH(c);
    k_proj_t<<<nb, 256, 0, c->stream>>>(N, z, c->w, partial, GM_RB, c->area, dout + (int64_t)r * N);
    LB_LAUNCH(c);
    if (info) {
      info->iterations += it;
      info->converged = info->converged && (res < c->params.tol);
      info->rel_residual = std::max(info->rel_residual, res);
      if (r == 0) {
        info->history_len = (int32_t)std::min<size_t>(hist.size(), 128);
        for (int i = 0; i < info->history_len; ++i) info->history[i] = hist[i];
      }
    }
  }
  LB_CHECK(lb_stage_out_finish(c, gf, dout, nrhs * N * sizeof(double)));
  if (info) {
    info->pairs = lb_pair_counter;
    info->applies_fp64 = lb_apply64_counter;
    LB_CUDA(c, cudaStreamSynchronize(c->stream));
    if (!info->converged) return lb_fail(c, LB_ENOTCONVERGED, "adjoint GMRES did not reach tol %.3g (residual %.3g)",
                                         c->params.tol, info->rel_residual);
  }
  return LB_OK;
}

// Geometry gradients of a loss of the A3 solve: sigma from A3 sigma = P f,
// z from A3^T z = S^T S^T g_u (both float64 GMRES), then the gradient pair
// sums of the adjoint module: node positions (grad) and/or tangents (gXu,
// gXv); any output may be null.
static int geometry_gradient(lb_ctx* c, int nrhs, const double* f, const double* gu, double* grad, double* gXu,
                             double* gXv, lb_solve_info* info) {
  LB_CHECK(lb_require_corr(c));
  if (c->far_order) return lb_fail(c, LB_EINVAL, "the geometry gradients use the node rule: clear the far rule");
  if (c->params.formulation != LB_A3) return lb_fail(c, LB_EINVAL, "the geometry gradients take the A3 formulation");
  if (nrhs < 1) return lb_fail(c, LB_EINVAL, "nrhs must be >= 1");
  if (!gu || !f) return lb_fail(c, LB_EINVAL, "null input pointer");
  if (!grad && !gXu && !gXv) return lb_fail(c, LB_EINVAL, "no output requested");
  if ((gXu == nullptr) != (gXv == nullptr)) return lb_fail(c, LB_EINVAL, "gXu and gXv come together");
  LB_CUDA(c, cudaSetDevice(c->device));
  const int64_t N = c->N;
  if (info) {
    *info = lb_solve_info{};
    info->converged = 1;
    info->nrhs = nrhs;
  }
  lb_pair_counter = 0;
  lb_apply64_counter = lb_apply32_counter = 0;
  const double* df;
  double* dgrad = nullptr;
  LB_CHECK(lb_stage_in(c, f, nrhs * N * sizeof(double), c->ws_stage_in, (const void**)&df));
  if (grad) LB_CHECK(lb_stage_out(c, grad, 3 * nrhs * N * sizeof(double), c->ws_stage_out, (void**)&dgrad));
  // tangent outputs: the caller's device buffers, or a staging area in ws_bvec
  double *dgu = nullptr, *dgv = nullptr;
  const bool tan_host = gXu && (!lb_is_device_ptr(gXu) || !lb_is_device_ptr(gXv));
  if (gXu) {
    if (tan_host) {
      LB_CHECK(lb_ensure(c, c->ws_bvec, (size_t)(6 * nrhs * N) * sizeof(double)));
      dgu = (double*)c->ws_bvec.p;
      dgv = dgu + 3 * nrhs * N;
    } else {
      dgu = gXu;
      dgv = gXv;
    }
  }
  const bool gu_dev = lb_is_device_ptr(gu);
  // b, sigma, potentials [4], q1, t2, z, staged g_u
  LB_CHECK(lb_ensure(c, c->ws_shape, (size_t)(11 * N) * sizeof(double)));
  double* b = (double*)c->ws_shape.p;
  double* sg = b + N;
  double* pot = sg + N;
  double* q1 = pot + 4 * N;
  double* t2 = q1 + N;
  double* z = t2 + N;
  double* gus = z + N;
  const double* mu2 = pot + (int64_t)LB_K_S * N;
  const double* mu1 = pot + (int64_t)LB_K_SP * N;
  for (int r = 0; r < nrhs; ++r) {
    const double* gr = gu + (int64_t)r * N;
    if (!gu_dev) {
      LB_CUDA(c, cudaMemcpyAsync(gus, gr, N * sizeof(double), cudaMemcpyHostToDevice, c->stream));
      gr = gus;
    }
    double removed = 0;
    LB_CHECK(project_mean_zero(c, df + (int64_t)r * N, b, &removed));
    if (info && r == 0) info->removed_mean = removed;
    int it1 = 0, it2 = 0;
    double res1 = 0, res2 = 0;
    std::vector<double> hist;
    LB_CHECK(gmres(c, LB_FP64, b, sg, c->params.tol, c->params.max_iter, &it1, &res1, r == 0 ? &hist : nullptr));
    LB_CHECK(lb_potentials(c, LB_FP64, sg, pot, (1u << LB_K_S) | (1u << LB_K_SP)));
    LB_CHECK(lb_apply_st_dev(c, gr, q1));
    LB_CHECK(lb_apply_st_dev(c, q1, t2));
    c->adjoint = true;
    const int rc = gmres(c, LB_FP64, t2, z, c->params.tol, c->params.max_iter, &it2, &res2, nullptr);
    c->adjoint = false;
    LB_CHECK(rc);
    if (dgrad) LB_CHECK(lb_shape_grad_pairs(c, gr, sg, mu1, mu2, q1, z, dgrad + (int64_t)r * 3 * N));
    if (dgu)
      LB_CHECK(lb_tangent_grad_pairs(c, gr, b, sg, mu1, mu2, q1, z, dgu + (int64_t)r * 3 * N,
                                     dgv + (int64_t)r * 3 * N));
    if (info) {
      info->iterations += it1 + it2;
      const double res = std::max(res1, res2);
      info->converged = info->converged && (res < c->params.tol);
      info->rel_residual = std::max(info->rel_residual, res);
      if (r == 0) {
        info->history_len = (int32_t)std::min<size_t>(hist.size(), 128);
        for (int i = 0; i < info->history_len; ++i) info->history[i] = hist[i];
      }
    }
  }
  if (dgrad) LB_CHECK(lb_stage_out_finish(c, grad, dgrad, 3 * nrhs * N * sizeof(double)));
  if (tan_host) {
    LB_CUDA(c, cudaMemcpyAsync(gXu, dgu, 3 * nrhs * N * sizeof(double), cudaMemcpyDefault, c->stream));
    LB_CUDA(c, cudaMemcpyAsync(gXv, dgv, 3 * nrhs * N * sizeof(double), cudaMemcpyDefault, c->stream));
    LB_CUDA(c, cudaStreamSynchronize(c->stream));
  }
  if (info) {
    info->pairs = lb_pair_counter;
    info->applies_fp64 = lb_apply64_counter;
    LB_CUDA(c, cudaStreamSynchronize(c->stream));
    if (!info->converged)
      return lb_fail(c, LB_ENOTCONVERGED, "a GMRES of the gradient did not reach tol %.3g (residual %.3g)",
                     c->params.tol, info->rel_residual);
  }
  return LB_OK;
}

extern "C" int lb_shape_gradient(lb_ctx* c, int nrhs, const double* f, const double* gu, double* grad,
                                 lb_solve_info* info) {
  if (!grad) return lb_fail(c, LB_EINVAL, "null output pointer");
  return geometry_gradient(c, nrhs, f, gu, grad, nullptr, nullptr, info);
}

extern "C" int lb_geometry_gradient(lb_ctx* c, int nrhs, const double* f, const double* gu, double* gX,
                                    double* gXu, double* gXv, lb_solve_info* info) {
  return geometry_gradient(c, nrhs, f, gu, gX, gXu, gXv, info);
}
