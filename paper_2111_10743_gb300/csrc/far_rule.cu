// Oversampled far-field rule (Section 4).
//
// The paper evaluates the smooth far-field quadrature on an oversampled
// rule: on every patch the density, positions and tangents are interpolated
// from the node rule to a finer rule on T0, and the far sums run over those
// points,
//   K[sigma]_i (far) = sum_{P not in Near(i)} sum_o w~_{P,o} K(x_i, y_{P,o}) sigma~_{P,o},
//   y_{P,o} = sum_q l_q(u_o) X_{P,q},   sigma~_{P,o} = sum_q l_q(u_o) sigma_{P,q},
// with the normal and area element of the interpolated tangents,
//   n = X~_u x X~_v / |X~_u x X~_v|,  w~ = w_o |X~_u x X~_v|.
// l_q are the Lagrange polynomials of the node rule (degree <= order).  The
// near corrections do not change: they integrate every near patch in full.
//
// lb_set_far_rule builds the source points once per surface; every
// single-density pass (lb_far_sums, the potentials, the A1/A2/A3 applies and
// the solves built on them) then packs the upsampled densities of its
// charges (k_far_upsample) with these points instead of the nodes.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <vector>

#include "basis.cuh"
#include "internal.cuh"

// source geometry: one thread per (patch, far-rule node)
__global__ void k_far_geometry(int64_t npatch, int np, int nps, const double* __restrict__ fI,
                               const double* __restrict__ X, const double* __restrict__ Xu,
                               const double* __restrict__ Xv, const double* __restrict__ wo, double* __restrict__ Y,
                               double* __restrict__ nY, double* __restrict__ wY) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= npatch * nps) return;
  const int64_t P = t / nps;
  const int o = (int)(t - P * nps);
  double y[3] = {0, 0, 0}, yu[3] = {0, 0, 0}, yv[3] = {0, 0, 0};
  for (int q = 0; q < np; ++q) {
    const double l = fI[o * np + q];
    const int64_t j = 3 * (P * np + q);
    for (int k = 0; k < 3; ++k) {
      y[k] = fma(l, X[j + k], y[k]);
      yu[k] = fma(l, Xu[j + k], yu[k]);
      yv[k] = fma(l, Xv[j + k], yv[k]);
    }
  }
  const double m0 = yu[1] * yv[2] - yu[2] * yv[1];
  const double m1 = yu[2] * yv[0] - yu[0] * yv[2];
  const double m2 = yu[0] * yv[1] - yu[1] * yv[0];
  const double J = sqrt(m0 * m0 + m1 * m1 + m2 * m2);
  for (int k = 0; k < 3; ++k) Y[3 * t + k] = y[k];
  nY[3 * t] = m0 / J;
  nY[3 * t + 1] = m1 / J;
  nY[3 * t + 2] = m2 / J;
  wY[t] = wo[o] * J;
}

// sigma~[P][o] = sum_q fI[o][q] sigma[P][q]
__global__ void k_far_upsample(int64_t npatch, int np, int nps, const double* __restrict__ fI,
                               const double* __restrict__ d, double* __restrict__ out) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= npatch * nps) return;
  const int64_t P = t / nps;
  const int o = (int)(t - P * nps);
  double s = 0.0;
  for (int q = 0; q < np; ++q) s = fma(fI[o * np + q], d[P * np + q], s);
  out[t] = s;
}

// recentred float / double source arrays, padding far away with zero charge
__global__ void k_far_points(int64_t n, int64_t npad, const double* __restrict__ Y, const double* __restrict__ nY,
                             double cx, double cy, double cz, float4* __restrict__ p32, float4* __restrict__ n32,
                             double4_32a* __restrict__ p64, double4_32a* __restrict__ n64) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= npad) return;
  if (i < n) {
    const double x = Y[3 * i] - cx, y = Y[3 * i + 1] - cy, z = Y[3 * i + 2] - cz;
    p32[i] = make_float4((float)x, (float)y, (float)z, 0.f);
    n32[i] = make_float4((float)nY[3 * i], (float)nY[3 * i + 1], (float)nY[3 * i + 2], 0.f);
    p64[i] = make_double4_32a(x, y, z, 0.0);
    n64[i] = make_double4_32a(nY[3 * i], nY[3 * i + 1], nY[3 * i + 2], 0.0);
  } else {
    p32[i] = make_float4(1e15f, 1e15f, 1e15f, 0.f);
    n32[i] = make_float4(0.f, 0.f, 0.f, 0.f);
    p64[i] = make_double4_32a(1e15, 1e15, 1e15, 0.0);
    n64[i] = make_double4_32a(0.0, 0.0, 0.0, 0.0);
  }
}

// A = (position, w~ d1~), B = (normal, w~ d2~)
template <typename R, typename V4>
__global__ void k_far_charges(int64_t n, int64_t npad, const V4* __restrict__ pos, const V4* __restrict__ nrm,
                              const double* __restrict__ w, const double* __restrict__ d1,
                              const double* __restrict__ d2, V4* __restrict__ A, V4* __restrict__ B) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= npad) return;
  V4 p = pos[i], q = nrm[i];
  p.w = i < n ? (R)(w[i] * d1[i]) : R(0);
  q.w = (i < n && d2) ? (R)(w[i] * d2[i]) : R(0);
  A[i] = p;
  B[i] = q;
}

void lb_free_far_rule(lb_ctx* c) {
  lb_free(&c->fI); lb_free(&c->fY); lb_free(&c->fn); lb_free(&c->fw);
  lb_free(&c->fpos32); lb_free(&c->fnrm32); lb_free(&c->fpos64); lb_free(&c->fnrm64);
  c->far_order = 0;
  c->nps = 0;
  c->Ns = c->Nspad = 0;
  c->far_uv.clear();
  c->far_w.clear();
}

extern "C" int lb_set_far_rule(lb_ctx* c, int order, const double* uv, const double* w) {
  if (!c) return lb_fail(nullptr, LB_EINVAL, "null context");
  if (!c->have_geom) return lb_fail(c, LB_ESTATE, "no geometry uploaded");
  LB_CUDA(c, cudaSetDevice(c->device));
  if (order == 0) {
    lb_free_far_rule(c);
    return LB_OK;
  }
  if (order < 1 || order > 20 || !uv || !w) return lb_fail(c, LB_EINVAL, "far rule: need order in [1, 20] and nodes");
  const int nps = (order + 1) * (order + 2) / 2;
  std::vector<double> hu(2 * nps), hw(nps);
  LB_CUDA(c, cudaMemcpy(hu.data(), uv, 2 * nps * sizeof(double), cudaMemcpyDefault));
  LB_CUDA(c, cudaMemcpy(hw.data(), w, nps * sizeof(double), cudaMemcpyDefault));
  double sw = 0;
  for (int o = 0; o < nps; ++o) {
    sw += hw[o];
    if (!(hu[2 * o] >= 0 && hu[2 * o + 1] >= 0 && hu[2 * o] + hu[2 * o + 1] <= 1))
      return lb_fail(c, LB_EINVAL, "far rule node %d outside T0", o);
  }
  if (!(std::fabs(sw - 0.5) < 1e-12)) return lb_fail(c, LB_EINVAL, "far rule weights sum to %.17g, not 1/2", sw);
  lb_free_far_rule(c);
  const int np = c->np;
  // Lagrange basis of the node rule at the far-rule nodes: l_q = sum_b phi_b Vinv[b][q]
  std::vector<double> I((size_t)nps * np), ph(np);
  for (int o = 0; o < nps; ++o) {
    lb_basis_eval(c->order, hu[2 * o], hu[2 * o + 1], [&](int b, double f, double, double) { ph[b] = f; });
    for (int q = 0; q < np; ++q) {
      double l = 0.0;
      for (int b = 0; b < np; ++b) l += ph[b] * c->Vinv[(size_t)b * np + q];
      I[(size_t)o * np + q] = l;
    }
  }
  const int64_t Ns = c->npatch * nps;
  const int64_t Nspad = ((Ns + 1023) / 1024) * 1024;
  double* dwo = nullptr;
  LB_CHECK(lb_alloc(c, &c->fI, (size_t)nps * np));
  LB_CHECK(lb_alloc(c, &c->fY, 3 * Ns));
  LB_CHECK(lb_alloc(c, &c->fn, 3 * Ns));
  LB_CHECK(lb_alloc(c, &c->fw, Ns));
  LB_CHECK(lb_alloc(c, &c->fpos32, Nspad));
  LB_CHECK(lb_alloc(c, &c->fnrm32, Nspad));
  LB_CHECK(lb_alloc(c, &c->fpos64, Nspad));
  LB_CHECK(lb_alloc(c, &c->fnrm64, Nspad));
  LB_CHECK(lb_ensure(c, c->ws_fden, (size_t)nps * sizeof(double)));
  dwo = (double*)c->ws_fden.p;
  LB_CUDA(c, cudaMemcpyAsync(c->fI, I.data(), I.size() * sizeof(double), cudaMemcpyHostToDevice, c->stream));
  LB_CUDA(c, cudaMemcpyAsync(dwo, hw.data(), nps * sizeof(double), cudaMemcpyHostToDevice, c->stream));
  k_far_geometry<<<lb_div_up(Ns, 128), 128, 0, c->stream>>>(c->npatch, np, nps, c->fI, c->X, c->Xu, c->Xv, dwo,
                                                              c->fY, c->fn, c->fw);
  LB_LAUNCH(c);
  k_far_points<<<lb_div_up(Nspad, 256), 256, 0, c->stream>>>(Ns, Nspad, c->fY, c->fn, c->center[0], c->center[1],
                                                               c->center[2], c->fpos32, c->fnrm32, c->fpos64,
                                                               c->fnrm64);
  LB_LAUNCH(c);
  // the double-float position grid must bound these points too
  std::vector<double> hY(3 * Ns);
  LB_CUDA(c, cudaMemcpyAsync(hY.data(), c->fY, 3 * Ns * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  LB_CUDA(c, cudaStreamSynchronize(c->stream));
  double ext = 0;
  for (int64_t s = 0; s < Ns; ++s)
    for (int k = 0; k < 3; ++k) {
      const double v = hY[3 * s + k];
      if (!std::isfinite(v)) return lb_fail(c, LB_EGEOM, "far rule: non-finite interpolated position");
      ext = std::max(ext, std::fabs(v - c->center[k]));
    }
  const double h = std::ldexp(1.0, (int)std::ceil(std::log2(std::max(ext, 1e-300))) - 23);
  c->df_grid = std::max(c->df_grid, h);
  c->far_order = order;
  c->nps = nps;
  c->Ns = Ns;
  c->Nspad = Nspad;
  c->far_uv = hu;
  c->far_w = hw;
  return LB_OK;
}

int lb_far_rule_pack(lb_ctx* c, int prec, const double* d1, const double* d2, void** A, void** B) {
  const int64_t Ns = c->Ns, Nspad = c->Nspad;
  // upsampled densities, then the packed sources
  LB_CHECK(lb_ensure(c, c->ws_fden, (size_t)(2 * Ns) * sizeof(double)));
  double* u1 = (double*)c->ws_fden.p;
  double* u2 = u1 + Ns;
  k_far_upsample<<<lb_div_up(Ns, 256), 256, 0, c->stream>>>(c->npatch, c->np, c->nps, c->fI, d1, u1);
  LB_LAUNCH(c);
  if (d2) {
    k_far_upsample<<<lb_div_up(Ns, 256), 256, 0, c->stream>>>(c->npatch, c->np, c->nps, c->fI, d2, u2);
    LB_LAUNCH(c);
  }
  if (prec == LB_DF64) {
    // sources: four planes of Nspad; then the nodes as targets: four planes of Npad
    LB_CHECK(lb_ensure(c, c->ws_src, (size_t)(4 * Nspad + 4 * c->Npad) * sizeof(float4)));
    float4* S = (float4*)c->ws_src.p;
    LB_CHECK(lb_pack_df_points(c, Ns, Nspad, c->fY, c->fn, c->fw, u1, d2 ? u2 : nullptr, S));
    LB_CHECK(lb_pack_df_points(c, c->N, c->Npad, c->X, c->nrm, c->w, c->w, nullptr, S + 4 * Nspad));
    *A = S;
    *B = nullptr;
    return LB_OK;
  }
  const size_t v4 = prec == LB_FP64 ? sizeof(double4_32a) : sizeof(float4);
  LB_CHECK(lb_ensure(c, c->ws_src, 2 * Nspad * v4));
  *A = c->ws_src.p;
  *B = (char*)c->ws_src.p + Nspad * v4;
  if (prec == LB_FP64)
    k_far_charges<double, double4_32a><<<lb_div_up(Nspad, 256), 256, 0, c->stream>>>(
        Ns, Nspad, c->fpos64, c->fnrm64, c->fw, u1, d2 ? u2 : nullptr, (double4_32a*)*A, (double4_32a*)*B);
  else
    k_far_charges<float, float4><<<lb_div_up(Nspad, 256), 256, 0, c->stream>>>(
        Ns, Nspad, c->fpos32, c->fnrm32, c->fw, u1, d2 ? u2 : nullptr, (float4*)*A, (float4*)*B);
  LB_LAUNCH(c);
  return LB_OK;
}
