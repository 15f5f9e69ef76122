// Context management, argument staging, surface upload and near lists.
//
// Geometry (Sections 2 and 4): from the chart samples X, Xu, Xv at the node
// rule of every patch, one thread per node computes the unit normal
// n = Xu x Xv / |Xu x Xv|, the smooth weight w = w_ref |Xu x Xv|, the inverse
// metric, and the mean curvature H = -1/2 tr(g^-1 L) with L_ab = X_ab . n,
// where the second derivatives come from nodal differentiation of the
// sampled tangents within the patch (X_uu = D_u Xu, X_vv = D_v Xv,
// X_uv = (D_v Xu + D_u Xv)/2).  Near lists (Section 4, Near/Far split):
// Near(i) = {P : |x_i - c_P| < eta R_P}, c_P the mean of the patch's nodes
// and R_P the largest node distance from it.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>

#include "internal.cuh"

thread_local int64_t lb_pair_counter = 0;
thread_local int lb_apply64_counter = 0, lb_apply32_counter = 0;
thread_local int lb_graph_counter = 0;

static char g_static_err[512] = "no error";

int lb_fail(lb_ctx* c, int code, const char* fmt, ...) {
  char buf[1024];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  if (c) c->err = buf;
  else snprintf(g_static_err, sizeof g_static_err, "%s", buf);
  return code;
}

int lb_ensure(lb_ctx* c, DevBuf& b, size_t bytes) {
  if (bytes <= b.bytes && b.p) return LB_OK;
  if (b.p) {
    cudaStreamSynchronize(c->stream);  // buffer may still be in use by queued work
    cudaFree(b.p);
  }
  b.p = nullptr;
  b.bytes = 0;
  size_t want = std::max<size_t>(bytes, 256);
  if (lb_alloc_fails_now(c))
    return lb_fail(c, LB_ENOMEM, "workspace cudaMalloc(%zu) failed: simulated by lb_debug_fail_alloc", want);
  cudaError_t e = cudaMalloc(&b.p, want);
  if (e != cudaSuccess) {
    b.p = nullptr;
    return lb_fail(c, LB_ENOMEM, "workspace cudaMalloc(%zu) failed: %s", want, cudaGetErrorString(e));
  }
  b.bytes = want;
  return LB_OK;
}

int lb_is_device_ptr(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

int lb_stage_in(lb_ctx* c, const void* src, size_t bytes, DevBuf& tmp, const void** dev) {
  if (!src) return lb_fail(c, LB_EINVAL, "null input pointer");
  if (lb_is_device_ptr(src)) {
    *dev = src;
    return LB_OK;
  }
  LB_CHECK(lb_ensure(c, tmp, bytes));
  LB_CUDA(c, cudaMemcpyAsync(tmp.p, src, bytes, cudaMemcpyHostToDevice, c->stream));
  *dev = tmp.p;
  return LB_OK;
}

int lb_stage_out(lb_ctx* c, void* dst, size_t bytes, DevBuf& tmp, void** dev) {
  if (!dst) return lb_fail(c, LB_EINVAL, "null output pointer");
  if (lb_is_device_ptr(dst)) {
    *dev = dst;
    return LB_OK;
  }
  LB_CHECK(lb_ensure(c, tmp, bytes));
  *dev = tmp.p;
  return LB_OK;
}

int lb_stage_out_finish(lb_ctx* c, void* dst, const void* dev, size_t bytes) {
  if (dst == dev) return LB_OK;
  LB_CUDA(c, cudaMemcpyAsync(dst, dev, bytes, cudaMemcpyDeviceToHost, c->stream));
  LB_CUDA(c, cudaStreamSynchronize(c->stream));
  return LB_OK;
}

// ---------------------------------------------------------------------------
// ---------------------------------------------------------------------------
// profiling
ProfScope::ProfScope(lb_ctx* ctx, int category, int64_t npairs) : c(ctx), cat(category), pairs(npairs) {
  if (!c || !c->prof_on) return;
  if (c->ev_pool.empty()) {
    cudaEvent_t e;
    if (cudaEventCreate(&e) != cudaSuccess) return;
    c->ev_pool.push_back(e);
  }
  a = c->ev_pool.back();
  c->ev_pool.pop_back();
  // inside a stream capture the record becomes a node of the graph, timed
  // again at every replay
  if (c->capture_prof) cudaEventRecordWithFlags(a, c->stream, cudaEventRecordExternal);
  else cudaEventRecord(a, c->stream);
}

ProfScope::~ProfScope() {
  if (!a) return;
  cudaEvent_t b;
  if (c->ev_pool.empty()) {
    if (cudaEventCreate(&b) != cudaSuccess) { c->ev_pool.push_back(a); return; }
  } else {
    b = c->ev_pool.back();
    c->ev_pool.pop_back();
  }
  if (c->capture_prof) {
    cudaEventRecordWithFlags(b, c->stream, cudaEventRecordExternal);
    c->capture_prof->push_back({cat, a, b, pairs});
  } else {
    cudaEventRecord(b, c->stream);
    c->prof_pending.push_back({cat, a, b, pairs});
  }
}

static int prof_resolve(lb_ctx* c) {
  if (c->prof_pending.empty()) return LB_OK;
  LB_CUDA(c, cudaStreamSynchronize(c->stream));
  for (auto& p : c->prof_pending) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, p.a, p.b) == cudaSuccess && p.cat >= 0 && p.cat < LB_PROF_NCAT) {
      c->prof_ms[p.cat] += ms;
      c->prof_calls[p.cat] += 1;
      c->prof_pairs[p.cat] += p.pairs;
    }
    c->ev_pool.push_back(p.a);
    c->ev_pool.push_back(p.b);
  }
  c->prof_pending.clear();
  return LB_OK;
}

extern "C" int lb_set_profiling(lb_ctx* c, int on) {
  if (!c) return lb_fail(nullptr, LB_EINVAL, "null context");
  LB_CUDA(c, cudaSetDevice(c->device));
  LB_CHECK(prof_resolve(c));
  for (int k = 0; k < LB_PROF_NCAT; ++k) { c->prof_ms[k] = 0; c->prof_calls[k] = 0; c->prof_pairs[k] = 0; }
  c->launches = 0;
  c->prof_on = on ? 1 : 0;
  return LB_OK;
}

extern "C" int lb_get_profile(lb_ctx* c, lb_profile* out) {
  if (!c || !out) return lb_fail(c, LB_EINVAL, "null argument");
  LB_CUDA(c, cudaSetDevice(c->device));
  LB_CHECK(prof_resolve(c));
  for (int k = 0; k < LB_PROF_NCAT; ++k) {
    out->ms[k] = c->prof_ms[k];
    out->calls[k] = c->prof_calls[k];
    out->pairs[k] = c->prof_pairs[k];
  }
  out->launches = c->launches;
  return LB_OK;
}

extern "C" int lb_default_params(lb_params* p) {
  if (!p) return lb_fail(nullptr, LB_EINVAL, "null params");
  p->eps_quad = 1e-12;
  p->near_factor = 2.0;
  p->precision = LB_FP64;
  p->formulation = LB_A3;
  p->max_iter = 100;
  p->tol = 1e-10;
  p->inner_tol = 1e-5;
  p->max_refine = 6;
  p->graphs = 1;
  return LB_OK;
}

static int check_params(lb_ctx* c, const lb_params* p) {
  if (!(p->eps_quad > 0 && p->eps_quad < 1)) return lb_fail(c, LB_EINVAL, "eps_quad must be in (0,1)");
  if (!(p->near_factor > 1.0 && p->near_factor < 1e3))
    return lb_fail(c, LB_EINVAL, "near_factor must be in (1, 1000): the own patch must be near");
  if (p->precision < LB_FP64 || p->precision > LB_DF64) return lb_fail(c, LB_EINVAL, "bad precision");
  if (p->formulation != LB_A1 && p->formulation != LB_A2 && p->formulation != LB_A3)
    return lb_fail(c, LB_EINVAL, "bad formulation");
  if (p->max_iter < 1 || p->max_iter > 1000) return lb_fail(c, LB_EINVAL, "max_iter must be in [1,1000]");
  if (!(p->tol > 0 && p->tol < 1)) return lb_fail(c, LB_EINVAL, "tol must be in (0,1)");
  if (!(p->inner_tol > 0 && p->inner_tol < 1)) return lb_fail(c, LB_EINVAL, "inner_tol must be in (0,1)");
  if (p->max_refine < 1 || p->max_refine > 100) return lb_fail(c, LB_EINVAL, "max_refine must be in [1,100]");
  if (p->graphs != 0 && p->graphs != 1) return lb_fail(c, LB_EINVAL, "graphs must be 0 or 1");
  return LB_OK;
}

extern "C" int lb_create(lb_ctx** out, int device, const lb_params* p) {
  if (!out) return lb_fail(nullptr, LB_EINVAL, "null output pointer");
  *out = nullptr;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
    cudaGetLastError();
    return lb_fail(nullptr, LB_ECUDA, "no CUDA device available");
  }
  if (device < 0 || device >= ndev) return lb_fail(nullptr, LB_EINVAL, "device %d out of range", device);
  lb_ctx* c = new (std::nothrow) lb_ctx();
  if (!c) return lb_fail(nullptr, LB_ENOMEM, "host allocation failed");
  c->device = device;
  if (p) c->params = *p;
  else lb_default_params(&c->params);
  int rc = check_params(c, &c->params);
  if (rc != LB_OK) {
    snprintf(g_static_err, sizeof g_static_err, "%s", c->err.c_str());
    delete c;
    return rc;
  }
  if (cudaSetDevice(device) != cudaSuccess) {
    delete c;
    return lb_fail(nullptr, LB_ECUDA, "cudaSetDevice failed");
  }
  cudaDeviceGetAttribute(&c->sm_count, cudaDevAttrMultiProcessorCount, device);
  if (cudaMallocHost((void**)&c->host_pinned, LB_PINNED_DOUBLES * sizeof(double)) != cudaSuccess) {
    delete c;
    return lb_fail(nullptr, LB_ENOMEM, "pinned host allocation failed");
  }
  *out = c;
  return LB_OK;
}

static void free_geometry(lb_ctx* c) {
  lb_free(&c->X); lb_free(&c->Xu); lb_free(&c->Xv); lb_free(&c->nrm); lb_free(&c->inrm);
  lb_free(&c->w); lb_free(&c->H); lb_free(&c->ginv); lb_free(&c->J); lb_free(&c->cen);
  lb_free(&c->rad); lb_free(&c->area_p); lb_free(&c->dVinv); lb_free(&c->dDu); lb_free(&c->dDv);
  lb_free(&c->dref); lb_free(&c->pos32); lb_free(&c->nrm32); lb_free(&c->pos64); lb_free(&c->nrm64);
  lb_free_far_rule(c);
  c->have_geom = false;
}

void lb_free_transpose(lb_ctx* c) {
  lb_free(&c->tptr); lb_free(&c->trow); lb_free(&c->tblk); lb_free(&c->tmask); lb_free(&c->tflag);
  lb_free(&c->v0);
  lb_free(&c->v1);
  c->have_trans = false;
}

static void free_near(lb_ctx* c) {
  lb_free_transpose(c);
  lb_free(&c->row_ptr); lb_free(&c->near_patch); lb_free(&c->vals);
  lb_free(&c->vals_hi); lb_free(&c->vals_lo);
  lb_free(&c->phi0);
  c->phi0_prec = -1;
  for (auto& m : c->masks) lb_free(&m.flags);
  c->masks.clear();
  c->have_near = c->have_corr = false;
  c->nnzb = 0;
}

extern "C" int lb_destroy(lb_ctx* c) {
  if (!c) return LB_OK;
  cudaSetDevice(c->device);
  if (c->stream) cudaStreamSynchronize(c->stream);
  free_geometry(c);
  free_near(c);
  for (DevBuf* b : {&c->ws_part, &c->ws_pot, &c->ws_src, &c->ws_vec, &c->ws_red, &c->ws_stage_in,
                    &c->ws_stage_out, &c->ws_gm, &c->ws_quad, &c->ws_bpot, &c->ws_bgm, &c->ws_bvec, &c->ws_dlow, &c->ws_a1,
                    &c->ws_adj, &c->ws_shape, &c->ws_grad, &c->ws_fden, &c->ws_rec})
    if (b->p) cudaFree(b->p);
  if (c->host_pinned) cudaFreeHost(c->host_pinned);
  if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
  for (auto& p : c->prof_pending) { cudaEventDestroy(p.a); cudaEventDestroy(p.b); }
  for (auto e : c->ev_pool) cudaEventDestroy(e);
  delete c;
  return LB_OK;
}

extern "C" const char* lb_last_error(const lb_ctx* c) { return c ? c->err.c_str() : g_static_err; }

extern "C" int lb_set_params(lb_ctx* c, const lb_params* p) {
  if (!c || !p) return lb_fail(c, LB_EINVAL, "null argument");
  LB_CHECK(check_params(c, p));
  bool drop = p->eps_quad != c->params.eps_quad || p->near_factor != c->params.near_factor;
  c->params = *p;
  if (drop) {
    cudaSetDevice(c->device);
    free_near(c);
  }
  return LB_OK;
}

extern "C" int lb_get_params(const lb_ctx* c, lb_params* p) {
  if (!c || !p) return lb_fail(nullptr, LB_EINVAL, "null argument");
  *p = c->params;
  return LB_OK;
}

extern "C" int lb_set_stream(lb_ctx* c, void* stream) {
  if (!c) return lb_fail(nullptr, LB_EINVAL, "null context");
  c->stream = (cudaStream_t)stream;
  return LB_OK;
}

// ---------------------------------------------------------------------------
// geometry kernels

__global__ void k_geometry(int64_t N, int np, const double* __restrict__ X, const double* __restrict__ Xu,
                           const double* __restrict__ Xv, const double* __restrict__ ref,
                           const double* __restrict__ Du, const double* __restrict__ Dv,
                           double* __restrict__ nrm, double* __restrict__ inrm, double* __restrict__ w,
                           double* __restrict__ H, double* __restrict__ ginv, double* __restrict__ J,
                           int* __restrict__ bad) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= N) return;
  int64_t P = i / np;
  int q = (int)(i - P * np);
  const double* xu = Xu + 3 * i;
  const double* xv = Xv + 3 * i;
  double c0 = xu[1] * xv[2] - xu[2] * xv[1];
  double c1 = xu[2] * xv[0] - xu[0] * xv[2];
  double c2 = xu[0] * xv[1] - xu[1] * xv[0];
  double jn = sqrt(c0 * c0 + c1 * c1 + c2 * c2);
  if (!(jn > 0.0)) {
    atomicExch(bad, 1);
    jn = 1.0;
  }
  double n0 = c0 / jn, n1 = c1 / jn, n2 = c2 / jn;
  nrm[3 * i] = n0; nrm[3 * i + 1] = n1; nrm[3 * i + 2] = n2;
  J[i] = jn;
  w[i] = ref[3 * q + 2] * jn;
  double g11 = xu[0] * xu[0] + xu[1] * xu[1] + xu[2] * xu[2];
  double g12 = xu[0] * xv[0] + xu[1] * xv[1] + xu[2] * xv[2];
  double g22 = xv[0] * xv[0] + xv[1] * xv[1] + xv[2] * xv[2];
  double det = g11 * g22 - g12 * g12;
  double a11 = g22 / det, a12 = -g12 / det, a22 = g11 / det;
  ginv[3 * i] = a11; ginv[3 * i + 1] = a12; ginv[3 * i + 2] = a22;
  // second derivatives and interpolant tangents by nodal differentiation
  double xuu[3] = {0, 0, 0}, xvv[3] = {0, 0, 0}, xuv[3] = {0, 0, 0}, yu[3] = {0, 0, 0}, yv[3] = {0, 0, 0};
  const int64_t base = P * np;
  for (int b = 0; b < np; ++b) {
    double du = Du[q * np + b], dv = Dv[q * np + b];
    const double* pu = Xu + 3 * (base + b);
    const double* pv = Xv + 3 * (base + b);
    const double* px = X + 3 * (base + b);
    for (int k = 0; k < 3; ++k) {
      xuu[k] += du * pu[k];
      xvv[k] += dv * pv[k];
      xuv[k] += 0.5 * (dv * pu[k] + du * pv[k]);
      yu[k] += du * px[k];
      yv[k] += dv * px[k];
    }
  }
  double L11 = xuu[0] * n0 + xuu[1] * n1 + xuu[2] * n2;
  double L12 = xuv[0] * n0 + xuv[1] * n1 + xuv[2] * n2;
  double L22 = xvv[0] * n0 + xvv[1] * n1 + xvv[2] * n2;
  H[i] = -0.5 * (a11 * L11 + 2.0 * a12 * L12 + a22 * L22);
  double m0 = yu[1] * yv[2] - yu[2] * yv[1];
  double m1 = yu[2] * yv[0] - yu[0] * yv[2];
  double m2 = yu[0] * yv[1] - yu[1] * yv[0];
  double mn = sqrt(m0 * m0 + m1 * m1 + m2 * m2);
  if (!(mn > 0.0)) {
    atomicExch(bad, 1);
    mn = 1.0;
  }
  inrm[3 * i] = m0 / mn; inrm[3 * i + 1] = m1 / mn; inrm[3 * i + 2] = m2 / mn;
}

__global__ void k_patches(int64_t npatch, int np, const double* __restrict__ X, const double* __restrict__ w,
                          double* __restrict__ cen, double* __restrict__ rad, double* __restrict__ area) {
  int64_t P = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (P >= npatch) return;
  const double* x = X + 3 * P * np;
  double c[3] = {0, 0, 0}, a = 0;
  for (int q = 0; q < np; ++q) {
    for (int k = 0; k < 3; ++k) c[k] += x[3 * q + k];
    a += w[P * np + q];
  }
  for (int k = 0; k < 3; ++k) c[k] /= np;
  double r2 = 0;
  for (int q = 0; q < np; ++q) {
    double d0 = x[3 * q] - c[0], d1 = x[3 * q + 1] - c[1], d2 = x[3 * q + 2] - c[2];
    r2 = fmax(r2, d0 * d0 + d1 * d1 + d2 * d2);
  }
  cen[3 * P] = c[0]; cen[3 * P + 1] = c[1]; cen[3 * P + 2] = c[2];
  rad[P] = sqrt(r2);
  area[P] = a;
}

__global__ void k_pack_sources(int64_t N, int64_t Npad, const double* __restrict__ X, const double* __restrict__ nrm,
                               double cx, double cy, double cz, float4* __restrict__ p32,
                               float4* __restrict__ n32, double4_32a* __restrict__ p64, double4_32a* __restrict__ n64) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= Npad) return;
  if (i < N) {
    double x = X[3 * i], y = X[3 * i + 1], z = X[3 * i + 2];
    p32[i] = make_float4((float)(x - cx), (float)(y - cy), (float)(z - cz), 0.f);
    n32[i] = make_float4((float)nrm[3 * i], (float)nrm[3 * i + 1], (float)nrm[3 * i + 2], 0.f);
    p64[i] = make_double4_32a(x - cx, y - cy, z - cz, 0.0);
    n64[i] = make_double4_32a(nrm[3 * i], nrm[3 * i + 1], nrm[3 * i + 2], 0.0);
  } else {  // padding: far away, zero normal (its density is always zero)
    p32[i] = make_float4(1e15f, 1e15f, 1e15f, 0.f);
    n32[i] = make_float4(0.f, 0.f, 0.f, 0.f);
    p64[i] = make_double4_32a(1e15, 1e15, 1e15, 0.0);
    n64[i] = make_double4_32a(0.0, 0.0, 0.0, 0.0);
  }
}

static const int64_t kPad = 1024;  // node arrays padded to a multiple of the largest source tile

extern "C" int lb_upload_geometry(lb_ctx* c, int64_t npatch, int order, const double* ref_uv,
                                  const double* ref_w, const double* X, const double* Xu,
                                  const double* Xv) {
  if (!c) return lb_fail(nullptr, LB_EINVAL, "null context");
  if (npatch < 1 || order < 1 || order > 10)
    return lb_fail(c, LB_EINVAL, "need npatch >= 1 and order in [1, 10]");
  if (!ref_uv || !ref_w || !X || !Xu || !Xv) return lb_fail(c, LB_EINVAL, "null geometry pointer");
  LB_CUDA(c, cudaSetDevice(c->device));
  const int np = (order + 1) * (order + 2) / 2;
  const int64_t N = npatch * np;
  if (N > (int64_t)1 << 31) return lb_fail(c, LB_EINVAL, "too many nodes");
  // node rule to host
  std::vector<double> uv(2 * np), rw(np);
  if (lb_is_device_ptr(ref_uv)) LB_CUDA(c, cudaMemcpy(uv.data(), ref_uv, 2 * np * sizeof(double), cudaMemcpyDeviceToHost));
  else memcpy(uv.data(), ref_uv, 2 * np * sizeof(double));
  if (lb_is_device_ptr(ref_w)) LB_CUDA(c, cudaMemcpy(rw.data(), ref_w, np * sizeof(double), cudaMemcpyDeviceToHost));
  else memcpy(rw.data(), ref_w, np * sizeof(double));
  double sw = 0;
  for (int q = 0; q < np; ++q) {
    sw += rw[q];
    if (!(uv[2 * q] >= 0 && uv[2 * q + 1] >= 0 && uv[2 * q] + uv[2 * q + 1] <= 1))
      return lb_fail(c, LB_EINVAL, "reference node %d outside T0", q);
  }
  if (!(std::fabs(sw - 0.5) < 1e-12)) return lb_fail(c, LB_EINVAL, "reference weights sum to %.17g, not 1/2", sw);
  free_near(c);
  free_geometry(c);
  c->N = N;
  c->npatch = npatch;
  c->np = np;
  c->order = order;
  c->ref_uv = uv;
  c->ref_w = rw;
  LB_CHECK(lb_host_basis_matrices(c));
  c->Npad = ((N + kPad - 1) / kPad) * kPad;
  LB_CHECK(lb_alloc(c, &c->X, 3 * N)); LB_CHECK(lb_alloc(c, &c->Xu, 3 * N)); LB_CHECK(lb_alloc(c, &c->Xv, 3 * N));
  LB_CHECK(lb_alloc(c, &c->nrm, 3 * N)); LB_CHECK(lb_alloc(c, &c->inrm, 3 * N));
  LB_CHECK(lb_alloc(c, &c->w, N)); LB_CHECK(lb_alloc(c, &c->H, N)); LB_CHECK(lb_alloc(c, &c->ginv, 3 * N));
  LB_CHECK(lb_alloc(c, &c->J, N)); LB_CHECK(lb_alloc(c, &c->cen, 3 * npatch)); LB_CHECK(lb_alloc(c, &c->rad, npatch));
  LB_CHECK(lb_alloc(c, &c->area_p, npatch));
  LB_CHECK(lb_alloc(c, &c->dVinv, np * np)); LB_CHECK(lb_alloc(c, &c->dDu, np * np)); LB_CHECK(lb_alloc(c, &c->dDv, np * np));
  LB_CHECK(lb_alloc(c, &c->dref, 3 * np));
  LB_CHECK(lb_alloc(c, &c->pos32, c->Npad)); LB_CHECK(lb_alloc(c, &c->nrm32, c->Npad));
  LB_CHECK(lb_alloc(c, &c->pos64, c->Npad)); LB_CHECK(lb_alloc(c, &c->nrm64, c->Npad));
  const size_t vb = 3 * N * sizeof(double);
  for (auto pr : {std::make_pair(c->X, X), std::make_pair(c->Xu, Xu), std::make_pair(c->Xv, Xv)})
    LB_CUDA(c, cudaMemcpyAsync(pr.first, pr.second, vb, cudaMemcpyDefault, c->stream));
  std::vector<double> ref3(3 * np);
  for (int q = 0; q < np; ++q) { ref3[3 * q] = uv[2 * q]; ref3[3 * q + 1] = uv[2 * q + 1]; ref3[3 * q + 2] = rw[q]; }
  LB_CUDA(c, cudaMemcpyAsync(c->dref, ref3.data(), 3 * np * sizeof(double), cudaMemcpyHostToDevice, c->stream));
  LB_CUDA(c, cudaMemcpyAsync(c->dVinv, c->Vinv.data(), np * np * sizeof(double), cudaMemcpyHostToDevice, c->stream));
  LB_CUDA(c, cudaMemcpyAsync(c->dDu, c->Du.data(), np * np * sizeof(double), cudaMemcpyHostToDevice, c->stream));
  LB_CUDA(c, cudaMemcpyAsync(c->dDv, c->Dv.data(), np * np * sizeof(double), cudaMemcpyHostToDevice, c->stream));
  LB_CHECK(lb_ensure(c, c->ws_red, 1 << 20));
  int* dbad = (int*)c->ws_red.p;
  LB_CUDA(c, cudaMemsetAsync(dbad, 0, sizeof(int), c->stream));
  k_geometry<<<lb_div_up(N, 128), 128, 0, c->stream>>>(N, np, c->X, c->Xu, c->Xv, c->dref, c->dDu, c->dDv,
                                                         c->nrm, c->inrm, c->w, c->H, c->ginv, c->J, dbad);
  LB_LAUNCH(c);
  k_patches<<<lb_div_up(npatch, 128), 128, 0, c->stream>>>(npatch, np, c->X, c->w, c->cen, c->rad, c->area_p);
  LB_LAUNCH(c);
  int bad = 0;
  LB_CUDA(c, cudaMemcpyAsync(&bad, dbad, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  // centre and area on the host from the patch sums (npatch doubles)
  std::vector<double> cen(3 * npatch), ar(npatch);
  LB_CUDA(c, cudaMemcpyAsync(cen.data(), c->cen, 3 * npatch * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  LB_CUDA(c, cudaMemcpyAsync(ar.data(), c->area_p, npatch * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  LB_CUDA(c, cudaStreamSynchronize(c->stream));
  if (bad) return lb_fail(c, LB_EGEOM, "degenerate chart: |Xu x Xv| = 0 at some node");
  double cc[3] = {0, 0, 0}, a = 0;
  for (int64_t P = 0; P < npatch; ++P) {
    for (int k = 0; k < 3; ++k) cc[k] += cen[3 * P + k];
    a += ar[P];
  }
  for (int k = 0; k < 3; ++k) c->center[k] = cc[k] / npatch;
  c->area = a;
  // double-float grid: 2^e bounds every recentred coordinate, h = 2^(e-23), so
  // that differences of grid values (at most 2^(e+1) = 2^24 h) are exact floats
  double ext = 0;
  {
    std::vector<double> rad(npatch);
    LB_CUDA(c, cudaMemcpy(rad.data(), c->rad, npatch * sizeof(double), cudaMemcpyDeviceToHost));
    for (int64_t P = 0; P < npatch; ++P)
      for (int k = 0; k < 3; ++k) ext = std::max(ext, std::fabs(cen[3 * P + k] - c->center[k]) + rad[P]);
  }
  c->df_grid = std::ldexp(1.0, (int)std::ceil(std::log2(std::max(ext, 1e-300))) - 23);
  k_pack_sources<<<lb_div_up(c->Npad, 256), 256, 0, c->stream>>>(N, c->Npad, c->X, c->nrm, c->center[0],
                                                                   c->center[1], c->center[2], c->pos32,
                                                                   c->nrm32, c->pos64, c->nrm64);
  LB_LAUNCH(c);
  c->have_geom = true;
  return LB_OK;
}

extern "C" int lb_get_geometry(lb_ctx* c, double* n, double* w, double* H) {
  if (!c) return lb_fail(nullptr, LB_EINVAL, "null context");
  if (!c->have_geom) return lb_fail(c, LB_ESTATE, "no geometry uploaded");
  LB_CUDA(c, cudaSetDevice(c->device));
  if (n) LB_CUDA(c, cudaMemcpyAsync(n, c->nrm, 3 * c->N * sizeof(double), cudaMemcpyDefault, c->stream));
  if (w) LB_CUDA(c, cudaMemcpyAsync(w, c->w, c->N * sizeof(double), cudaMemcpyDefault, c->stream));
  if (H) LB_CUDA(c, cudaMemcpyAsync(H, c->H, c->N * sizeof(double), cudaMemcpyDefault, c->stream));
  LB_CUDA(c, cudaStreamSynchronize(c->stream));
  return LB_OK;
}

extern "C" int lb_geometry_info(lb_ctx* c, lb_geom_info* info) {
  if (!c || !info) return lb_fail(c, LB_EINVAL, "null argument");
  info->N = c->N;
  info->npatch = c->npatch;
  info->np = c->np;
  info->order = c->order;
  info->nnzb = c->nnzb;
  info->area = c->area;
  info->sm_count = c->sm_count;
  info->corrections = c->have_corr ? 1 : 0;
  return LB_OK;
}

// ---------------------------------------------------------------------------
// near lists

__global__ void k_near_count(int64_t N, int64_t npatch, const double* __restrict__ X,
                             const double* __restrict__ cen, const double* __restrict__ rad, double eta,
                             int64_t* __restrict__ cnt) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= N) return;
  double x0 = X[3 * i], x1 = X[3 * i + 1], x2 = X[3 * i + 2];
  int64_t c = 0;
  for (int64_t P = 0; P < npatch; ++P) {
    double d0 = x0 - cen[3 * P], d1 = x1 - cen[3 * P + 1], d2 = x2 - cen[3 * P + 2];
    c += sqrt(d0 * d0 + d1 * d1 + d2 * d2) < eta * rad[P];
  }
  cnt[i] = c;
}

__global__ void k_near_fill(int64_t N, int64_t npatch, const double* __restrict__ X,
                            const double* __restrict__ cen, const double* __restrict__ rad, double eta,
                            const int64_t* __restrict__ ptr, int32_t* __restrict__ patch) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= N) return;
  double x0 = X[3 * i], x1 = X[3 * i + 1], x2 = X[3 * i + 2];
  int64_t o = ptr[i];
  for (int64_t P = 0; P < npatch; ++P) {
    double d0 = x0 - cen[3 * P], d1 = x1 - cen[3 * P + 1], d2 = x2 - cen[3 * P + 2];
    if (sqrt(d0 * d0 + d1 * d1 + d2 * d2) < eta * rad[P]) patch[o++] = (int32_t)P;
  }
}

// exclusive scan of cnt[0..n) into ptr[0..n] by one block (setup only)
__global__ void k_scan_single(int64_t n, const int64_t* __restrict__ cnt, int64_t* __restrict__ ptr) {
  __shared__ int64_t part[1024];
  int t = threadIdx.x;
  int64_t chunk = (n + blockDim.x - 1) / blockDim.x;
  int64_t b = t * chunk, e = min(n, b + chunk);
  int64_t s = 0;
  for (int64_t i = b; i < e; ++i) s += cnt[i];
  part[t] = s;
  __syncthreads();
  if (t == 0) {
    int64_t run = 0;
    for (int k = 0; k < (int)blockDim.x; ++k) {
      int64_t v = part[k];
      part[k] = run;
      run += v;
    }
    ptr[n] = run;
  }
  __syncthreads();
  s = part[t];
  for (int64_t i = b; i < e; ++i) {
    ptr[i] = s;
    s += cnt[i];
  }
}

extern "C" int lb_build_near(lb_ctx* c) {
  if (!c) return lb_fail(nullptr, LB_EINVAL, "null context");
  if (!c->have_geom) return lb_fail(c, LB_ESTATE, "no geometry uploaded");
  LB_CUDA(c, cudaSetDevice(c->device));
  free_near(c);
  const int64_t N = c->N;
  LB_CHECK(lb_alloc(c, &c->row_ptr, N + 1));
  LB_CHECK(lb_ensure(c, c->ws_red, (N + 1) * sizeof(int64_t)));
  int64_t* cnt = (int64_t*)c->ws_red.p;
  const double eta = c->params.near_factor;
  k_near_count<<<lb_div_up(N, 128), 128, 0, c->stream>>>(N, c->npatch, c->X, c->cen, c->rad, eta, cnt);
  LB_LAUNCH(c);
  k_scan_single<<<1, 1024, 0, c->stream>>>(N, cnt, c->row_ptr);
  LB_LAUNCH(c);
  int64_t nnzb = 0;
  LB_CUDA(c, cudaMemcpyAsync(&nnzb, c->row_ptr + N, sizeof(int64_t), cudaMemcpyDeviceToHost, c->stream));
  LB_CUDA(c, cudaStreamSynchronize(c->stream));
  if (nnzb < N) return lb_fail(c, LB_EGEOM, "near lists miss the own patch (nnzb=%lld)", (long long)nnzb);
  LB_CHECK(lb_alloc(c, &c->near_patch, nnzb));
  k_near_fill<<<lb_div_up(N, 128), 128, 0, c->stream>>>(N, c->npatch, c->X, c->cen, c->rad, eta, c->row_ptr,
                                                          c->near_patch);
  LB_LAUNCH(c);
  c->nnzb = nnzb;
  c->have_near = true;
  return LB_OK;
}

// Structure check of loaded near lists (bit 0: row_ptr not nondecreasing or
// outside [0, nnzb]; bit 1: a patch index outside [0, npatch); bit 2: patches
// of a row not strictly ascending).  Every read stays inside row_ptr [N+1] and
// patch [nnzb]: a row's patches are read only after its bounds passed.
__global__ void k_check_csr(int64_t N, int64_t nnzb, int64_t npatch, const int64_t* __restrict__ row_ptr,
                            const int32_t* __restrict__ patch, int* __restrict__ bad) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t a = row_ptr[i], b = row_ptr[i + 1];
    if (a < 0 || b < a || b > nnzb) {
      atomicOr(bad, 1);
      continue;
    }
    int prev = -1;
    for (int64_t k = a; k < b; ++k) {
      const int p = patch[k];
      if (p < 0 || p >= npatch) atomicOr(bad, 2);
      else if (p <= prev) atomicOr(bad, 4);
      prev = p;
    }
  }
}

extern "C" int lb_load_corrections(lb_ctx* c, int64_t nnzb, const int64_t* row_ptr, const int32_t* patch,
                                   const double* vals) {
  if (!c) return lb_fail(nullptr, LB_EINVAL, "null context");
  if (!c->have_geom) return lb_fail(c, LB_ESTATE, "no geometry uploaded");
  if (nnzb < c->N || !row_ptr || !patch || !vals) return lb_fail(c, LB_EINVAL, "bad correction arrays");
  LB_CUDA(c, cudaSetDevice(c->device));
  free_near(c);
  const int64_t N = c->N;
  LB_CHECK(lb_alloc(c, &c->row_ptr, N + 1));
  LB_CHECK(lb_alloc(c, &c->near_patch, nnzb));
  lb_free(&c->vals_hi);
  lb_free(&c->vals_lo);
  lb_free(&c->phi0);
  c->phi0_prec = -1;
  lb_free_transpose(c);
  LB_CHECK(lb_alloc(c, &c->vals, nnzb * LB_NKERNELS * c->np));
  LB_CUDA(c, cudaMemcpyAsync(c->row_ptr, row_ptr, (N + 1) * sizeof(int64_t), cudaMemcpyDefault, c->stream));
  LB_CUDA(c, cudaMemcpyAsync(c->near_patch, patch, nnzb * sizeof(int32_t), cudaMemcpyDefault, c->stream));
  LB_CUDA(c, cudaMemcpyAsync(c->vals, vals, nnzb * LB_NKERNELS * c->np * sizeof(double), cudaMemcpyDefault,
                             c->stream));
  // the first and last row pointer, then the structure of every row, before
  // any kernel indexes with them
  LB_CHECK(lb_ensure(c, c->ws_red, 64));
  int* dbad = (int*)c->ws_red.p;
  LB_CUDA(c, cudaMemsetAsync(dbad, 0, sizeof(int), c->stream));
  k_check_csr<<<lb_div_up(N, 256) < 1024u ? lb_div_up(N, 256) : 1024u, 256, 0, c->stream>>>(
      N, nnzb, c->npatch, c->row_ptr, c->near_patch, dbad);
  LB_LAUNCH(c);
  int64_t ends[2];
  int bad = 0;
  LB_CUDA(c, cudaMemcpyAsync(&ends[0], c->row_ptr, sizeof(int64_t), cudaMemcpyDeviceToHost, c->stream));
  LB_CUDA(c, cudaMemcpyAsync(&ends[1], c->row_ptr + N, sizeof(int64_t), cudaMemcpyDeviceToHost, c->stream));
  LB_CUDA(c, cudaMemcpyAsync(&bad, dbad, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  LB_CUDA(c, cudaStreamSynchronize(c->stream));
  if (ends[0] != 0 || ends[1] != nnzb || bad) {
    free_near(c);
    if (ends[0] != 0 || ends[1] != nnzb) return lb_fail(c, LB_EINVAL, "row_ptr must start at 0 and end at nnzb");
    if (bad & 1) return lb_fail(c, LB_EINVAL, "row_ptr must be nondecreasing");
    if (bad & 2) return lb_fail(c, LB_EINVAL, "a near patch index lies outside [0, npatch)");
    return lb_fail(c, LB_EINVAL, "near patches of a row must be strictly ascending");
  }
  c->nnzb = nnzb;
  c->have_near = c->have_corr = true;
  return LB_OK;
}

extern "C" int lb_get_corrections(lb_ctx* c, int64_t* row_ptr, int32_t* patch, double* vals) {
  if (!c) return lb_fail(nullptr, LB_EINVAL, "null context");
  if (!c->have_near) return lb_fail(c, LB_ESTATE, "no near lists");
  LB_CUDA(c, cudaSetDevice(c->device));
  if (row_ptr) LB_CUDA(c, cudaMemcpyAsync(row_ptr, c->row_ptr, (c->N + 1) * sizeof(int64_t), cudaMemcpyDefault, c->stream));
  if (patch) LB_CUDA(c, cudaMemcpyAsync(patch, c->near_patch, c->nnzb * sizeof(int32_t), cudaMemcpyDefault, c->stream));
  if (vals) {
    if (!c->have_corr) return lb_fail(c, LB_ESTATE, "no corrections built");
    LB_CUDA(c, cudaMemcpyAsync(vals, c->vals, c->nnzb * LB_NKERNELS * c->np * sizeof(double), cudaMemcpyDefault,
                               c->stream));
  }
  LB_CUDA(c, cudaStreamSynchronize(c->stream));
  return LB_OK;
}

int lb_require_corr(lb_ctx* c) {
  if (!c) return lb_fail(nullptr, LB_EINVAL, "null context");
  if (!c->have_geom) return lb_fail(c, LB_ESTATE, "no geometry uploaded");
  if (!c->have_corr) return lb_fail(c, LB_ESTATE, "no corrections: call lb_build_corrections or lb_load_corrections");
  return LB_OK;
}

extern "C" int lb_debug_fail_alloc(lb_ctx* c, int64_t after) {
  if (!c) return lb_fail(nullptr, LB_EINVAL, "null context");
  c->fail_alloc_in = after < 0 ? -1 : after;
  return LB_OK;
}
