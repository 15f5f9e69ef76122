// Near-field correction blocks by adaptive quadrature on the device.
//
// For every row i and patch P in Near(i) (Section 4, the locally corrected
// scheme: self patch by singular quadrature, close patches by adaptive
// integration), and every kernel K in {S, D, S', S''+D'}:
//   W^K_{i,P}[q] = int_{Gamma_P} K(x_i, y) l_q(y) da(y),
// l_q the Lagrange polynomial of node q on P (the density's implicit
// interpolation).  The integral is accumulated in the orthonormal basis,
//   I_K[b] = int K phi_b da,   W^K[q] = sum_b I_K[b] Vinv[b][q].
//
// Cells and rules:
//   * a cell is a triangle (a, b, c) of T0 and a rectangle [s0,s1]x[t0,t1]
//     of the Duffy square; its points are a + s (b - a) + s t (c - b) with
//     Jacobian s |det(b - a, c - b)|, tensor Gauss-Legendre (m = 8) in (s, t);
//   * self patch: three root triangles with apex at the target's reference
//     node (Duffy 1982: the Jacobian s cancels the 1/r singularity), refined
//     by splitting the rectangle in four;
//   * other near patches: root T0, refined by midpoint 1 -> 4 splitting of the
//     triangle.
//   A cell is integrated, then its four children; the children's sum is
//   accepted when, mapped to the Lagrange weights (the entries of W), it
//   differs from the cell's value by at most max(tol, floor) in every entry,
//   else the children are pushed on the warp's stack.
//   tol = eps_quad A_P / (4 pi R_P); floor = 64 eps_mach Lambda times the
//   cell sum of omega J rho, Lambda the Lebesgue constant of the node set,
//   bounds the rounding of the numerators n.d as it reaches the weights;
//   below it refinement cannot improve the estimate.  On other patches
//   d = x - y carries eps (|x| + 2 R_P) rounding, rho = (|x| + 2 R_P) /
//   (4 pi r^3); on the self patch d = y(a) - y(p) is summed from the basis
//   differences phi_b(p) - phi_b(a) (carried through the recurrences), which
//   keeps full relative accuracy next to the target, and rho = 1/(4 pi r^2).  A cell whose children sum is below tol in every weight is
//   accepted too (its whole contribution is within the tolerance; this ends
//   the refinement of the vanishing cells next to the Duffy apex).
//
// Points lie on the polynomial chart y = sum_b cX_b phi_b; tangents, normal
// and area element are those of this polynomial, and the target normal is
// the normal of the position interpolant of the target's patch at its node.
// (The sampled tangents are not the derivatives of the position interpolant;
// using them would leave an odd 1/r^2 term on the self patch whose
// Duffy-split integral does not converge.)
//
// One warp per (row, patch) block; lanes take one quadrature point each in
// two rounds of 32, write basis values to shared memory, and then own basis
// coefficients b = lane + 32 s for the accumulation (deterministic order).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <vector>

#include "basis.cuh"
#include "internal.cuh"

#define QM 8           // Gauss-Legendre points per direction
#define QSTACK 100     // cells per warp stack
#define QMAXDEPTH 30
#define QWARPS 4
#define QMAXCELLS 40000  // per block; exceeding it sets the error flag

__constant__ double c_gx[QM], c_gw[QM];

// Gauss-Legendre nodes/weights on [0,1] by Newton iteration on P_m (host).
static void gauss_legendre01(int m, double* x, double* w) {
  for (int i = 0; i < m; ++i) {
    double z = cos(LB_PI * (i + 0.75) / (m + 0.5));
    double dp = 1;
    for (int it = 0; it < 100; ++it) {
      double p0 = 1, p1 = z;
      for (int k = 2; k <= m; ++k) {
        const double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
        p0 = p1;
        p1 = p2;
      }
      dp = m * (z * p1 - p0) / (z * z - 1.0);
      const double dz = p1 / dp;
      z -= dz;
      if (fabs(dz) < 1e-16) break;
    }
    x[i] = 0.5 * (1.0 - z);
    w[i] = 1.0 / ((1.0 - z * z) * dp * dp);
  }
}

__global__ void k_chart_coeffs(int64_t npatch, int np, const double* __restrict__ X, const double* __restrict__ Vinv,
                               double* __restrict__ cX) {
  int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= npatch * np) return;
  const int64_t P = t / np;
  const int b = (int)(t - P * np);
  double s[3] = {0, 0, 0};
  for (int q = 0; q < np; ++q) {
    const double v = Vinv[b * np + q];
    for (int k = 0; k < 3; ++k) s[k] += v * X[3 * (P * np + q) + k];
  }
  for (int k = 0; k < 3; ++k) cX[3 * t + k] = s[k];
}

struct QCell {
  double a0, a1, b0, b1, c0, c1, s0, s1, t0, t1;
  int depth;
};

// integrate one cell: I[k][s] for basis b = lane + 32 s, plus the rounding sum.
// offset (self patch): d = y(a) - y(p) from basis differences at the apex a.
__device__ void q_cell(const QCell& cl, int k, int np, const double* __restrict__ cX, double x0, double x1,
                       double x2, double n0, double n1, double n2, double xs, bool offset, double* phi,
                       double* fv, double I[4][3], double* rnd) {
  const int lane = threadIdx.x & 31;
  for (int kk = 0; kk < 4; ++kk)
    for (int s = 0; s < 3; ++s) I[kk][s] = 0.0;
  double rs = 0.0;
  const double e10 = cl.b0 - cl.a0, e11 = cl.b1 - cl.a1, e20 = cl.c0 - cl.b0, e21 = cl.c1 - cl.b1;
  const double det = fabs(e10 * e21 - e11 * e20);
  for (int round = 0; round < (QM * QM) / 32; ++round) {
    const int p = round * 32 + lane;
    const int is = p / QM, it = p - (p / QM) * QM;
    const double s = cl.s0 + (cl.s1 - cl.s0) * c_gx[is];
    const double t = cl.t0 + (cl.t1 - cl.t0) * c_gx[it];
    const double om = (cl.s1 - cl.s0) * c_gw[is] * (cl.t1 - cl.t0) * c_gw[it] * s * det;
    const double du = s * e10 + s * t * e20;
    const double dv = s * e11 + s * t * e21;
    double y[3] = {0, 0, 0}, yu[3] = {0, 0, 0}, yv[3] = {0, 0, 0};
    double* ph = phi + lane * np;
    if (offset) {  // y holds y(p) - y(a)
      lb_basis_eval_diff(k, cl.a0, cl.a1, du, dv, [&](int b, double f, double fu, double fvv, double df) {
        const double* cb = cX + 3 * b;
        for (int d = 0; d < 3; ++d) {
          y[d] = fma(df, cb[d], y[d]);
          yu[d] = fma(fu, cb[d], yu[d]);
          yv[d] = fma(fvv, cb[d], yv[d]);
        }
        ph[b] = f;
      });
    } else {
      lb_basis_eval(k, cl.a0 + du, cl.a1 + dv, [&](int b, double f, double fu, double fvv) {
        const double* cb = cX + 3 * b;
        for (int d = 0; d < 3; ++d) {
          y[d] = fma(f, cb[d], y[d]);
          yu[d] = fma(fu, cb[d], yu[d]);
          yv[d] = fma(fvv, cb[d], yv[d]);
        }
        ph[b] = f;
      });
    }
    const double m0 = yu[1] * yv[2] - yu[2] * yv[1];
    const double m1 = yu[2] * yv[0] - yu[0] * yv[2];
    const double m2 = yu[0] * yv[1] - yu[1] * yv[0];
    const double J = sqrt(m0 * m0 + m1 * m1 + m2 * m2);
    const double ny0 = m0 / J, ny1 = m1 / J, ny2 = m2 / J;
    const double d0 = offset ? -y[0] : x0 - y[0];
    const double d1 = offset ? -y[1] : x1 - y[1];
    const double d2 = offset ? -y[2] : x2 - y[2];
    const double r2 = d0 * d0 + d1 * d1 + d2 * d2;
    const double r = sqrt(r2);
    const double g = 1.0 / (4.0 * LB_PI * r);
    const double g3 = g / r2;
    const double nxd = n0 * d0 + n1 * d1 + n2 * d2;
    const double nyd = ny0 * d0 + ny1 * d1 + ny2 * d2;
    const double e0 = n0 - ny0, e1 = n1 - ny1, e2 = n2 - ny2;
    const double wJ = om * J;
    fv[lane * 4 + 0] = wJ * g;
    fv[lane * 4 + 1] = wJ * nyd * g3;
    fv[lane * 4 + 2] = -wJ * nxd * g3;
    fv[lane * 4 + 3] = wJ * (3.0 * nxd * (nxd - nyd) / r2 - 0.5 * (e0 * e0 + e1 * e1 + e2 * e2)) * g3;
    // rounding of the numerators: eps |d| r on the self patch, eps (|x| + 2R) elsewhere
    rs += offset ? wJ * g / r : wJ * g3 * xs;
    __syncwarp();
    for (int s2 = 0; s2 < 3; ++s2) {
      const int b = lane + 32 * s2;
      if (b >= np) break;
      double a0 = I[0][s2], a1 = I[1][s2], a2 = I[2][s2], a3 = I[3][s2];
      for (int pp = 0; pp < 32; ++pp) {
        const double f = phi[pp * np + b];
        a0 = fma(fv[pp * 4 + 0], f, a0);
        a1 = fma(fv[pp * 4 + 1], f, a1);
        a2 = fma(fv[pp * 4 + 2], f, a2);
        a3 = fma(fv[pp * 4 + 3], f, a3);
      }
      I[0][s2] = a0; I[1][s2] = a1; I[2][s2] = a2; I[3][s2] = a3;
    }
    __syncwarp();
  }
  for (int off = 16; off > 0; off >>= 1) rs += __shfl_xor_sync(0xffffffffu, rs, off);
  *rnd = rs;
}

__device__ __forceinline__ void q_child(const QCell& p, int which, bool tri, QCell& c) {
  c = p;
  c.depth = p.depth + 1;
  if (tri) {
    const double ab0 = 0.5 * (p.a0 + p.b0), ab1 = 0.5 * (p.a1 + p.b1);
    const double bc0 = 0.5 * (p.b0 + p.c0), bc1 = 0.5 * (p.b1 + p.c1);
    const double ca0 = 0.5 * (p.c0 + p.a0), ca1 = 0.5 * (p.c1 + p.a1);
    switch (which) {
      case 0: c.b0 = ab0; c.b1 = ab1; c.c0 = ca0; c.c1 = ca1; break;
      case 1: c.a0 = ab0; c.a1 = ab1; c.c0 = bc0; c.c1 = bc1; break;
      case 2: c.a0 = ca0; c.a1 = ca1; c.b0 = bc0; c.b1 = bc1; break;
      default: c.a0 = ab0; c.a1 = ab1; c.b0 = bc0; c.b1 = bc1; c.c0 = ca0; c.c1 = ca1; break;
    }
  } else {
    const double sm = 0.5 * (p.s0 + p.s1), tm = 0.5 * (p.t0 + p.t1);
    if (which & 1) c.s0 = sm; else c.s1 = sm;
    if (which & 2) c.t0 = tm; else c.t1 = tm;
  }
}

__global__ void __launch_bounds__(32 * QWARPS) k_near_quad(
    int64_t N, int np, int k, const int64_t* __restrict__ row_ptr, const int32_t* __restrict__ near_patch,
    int64_t nnzb, const double* __restrict__ X, const double* __restrict__ inrm, const double* __restrict__ ref,
    const double* __restrict__ cXall, const double* __restrict__ Vinv, const double* __restrict__ area,
    const double* __restrict__ rad, double eps_q, double lebesgue, double* __restrict__ vals,
    int* __restrict__ status) {
  extern __shared__ double smem[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int per_warp = 32 * np + 32 * 4 + 4 * np;
  double* phi = smem + warp * per_warp;
  double* fv = phi + 32 * np;
  double* acc = fv + 32 * 4;
  __shared__ QCell stack[QWARPS][QSTACK];
  const double eps = 2.220446049250313e-16;

  for (int64_t blk = (int64_t)blockIdx.x * QWARPS + warp; blk < nnzb; blk += (int64_t)gridDim.x * QWARPS) {
    // row of this block: binary search in row_ptr
    int64_t lo = 0, hi = N;
    while (hi - lo > 1) {
      const int64_t mid = (lo + hi) >> 1;
      if (row_ptr[mid] <= blk) lo = mid; else hi = mid;
    }
    const int64_t i = lo;
    const int64_t P = near_patch[blk];
    const double x0 = X[3 * i], x1 = X[3 * i + 1], x2 = X[3 * i + 2];
    const double n0 = inrm[3 * i], n1 = inrm[3 * i + 1], n2 = inrm[3 * i + 2];
    const double* cX = cXall + 3 * P * np;
    const double tol = eps_q * area[P] / (4.0 * LB_PI * rad[P]);
    const double xs = sqrt(x0 * x0 + x1 * x1 + x2 * x2) + 2.0 * rad[P];
    const double fscale = 64.0 * eps * lebesgue;
    const bool self = (i / np) == P;
    double tot[4][3];
    for (int kk = 0; kk < 4; ++kk)
      for (int s = 0; s < 3; ++s) tot[kk][s] = 0.0;
    int sp = 0;
    if (lane == 0) {
      if (self) {
        const int q = (int)(i - P * np);
        const double au = ref[3 * q], av = ref[3 * q + 1];
        const double vx[3] = {0.0, 1.0, 0.0}, vy[3] = {0.0, 0.0, 1.0};
        for (int j = 0; j < 3; ++j) {
          QCell c{au, av, vx[j], vy[j], vx[(j + 1) % 3], vy[(j + 1) % 3], 0.0, 1.0, 0.0, 1.0, 0};
          stack[warp][j] = c;
        }
      } else {
        QCell c{0.0, 0.0, 1.0, 0.0, 0.0, 1.0, 0.0, 1.0, 0.0, 1.0, 0};
        stack[warp][0] = c;
      }
    }
    sp = self ? 3 : 1;
    __syncwarp();
    int ncells = 0;
    bool overflow = false;
    while (sp > 0) {
      const QCell cell = stack[warp][sp - 1];
      --sp;
      __syncwarp();
      double Ip[4][3], Ik[4][3], It[4][3], rp, rk = 0.0, rt;
      q_cell(cell, k, np, cX, x0, x1, x2, n0, n1, n2, xs, self, phi, fv, Ip, &rp);
      for (int kk = 0; kk < 4; ++kk)
        for (int s = 0; s < 3; ++s) Ik[kk][s] = 0.0;
      QCell kids[4];
      for (int c = 0; c < 4; ++c) {
        q_child(cell, c, !self, kids[c]);
        q_cell(kids[c], k, np, cX, x0, x1, x2, n0, n1, n2, xs, self, phi, fv, It, &rt);
        for (int kk = 0; kk < 4; ++kk)
          for (int s = 0; s < 3; ++s) Ik[kk][s] += It[kk][s];
        rk += rt;
      }
      ncells += 5;
      // children sum and difference of the estimates, mapped to the Lagrange weights
      double err = 0.0, mag = 0.0;
      for (int pass = 0; pass < 2; ++pass) {
        for (int kk = 0; kk < 4; ++kk)
          for (int s = 0; s < 3; ++s)
            if (lane + 32 * s < np) acc[kk * np + lane + 32 * s] = pass ? Ik[kk][s] : Ik[kk][s] - Ip[kk][s];
        __syncwarp();
        double m = 0.0;
        for (int q = lane; q < np; q += 32) {
          double e4[4] = {0, 0, 0, 0};
          for (int b = 0; b < np; ++b) {
            const double vb = Vinv[b * np + q];
            for (int kk = 0; kk < 4; ++kk) e4[kk] = fma(acc[kk * np + b], vb, e4[kk]);
          }
          for (int kk = 0; kk < 4; ++kk) m = fmax(m, fabs(e4[kk]));
        }
        for (int off = 16; off > 0; off >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, off));
        if (pass) mag = m; else err = m;
        __syncwarp();
      }
      const bool accept = err <= fmax(tol, fscale * rk) || mag <= tol || cell.depth + 1 >= QMAXDEPTH ||
                          sp + 4 > QSTACK || ncells > QMAXCELLS;
      if (cell.depth + 1 >= QMAXDEPTH || sp + 4 > QSTACK || ncells > QMAXCELLS) overflow = true;
      if (accept) {
        for (int kk = 0; kk < 4; ++kk)
          for (int s = 0; s < 3; ++s) tot[kk][s] += Ik[kk][s];
      } else {
        if (lane == 0)
          for (int c = 0; c < 4; ++c) stack[warp][sp + c] = kids[c];
        sp += 4;
      }
      __syncwarp();
    }
    if (overflow && lane == 0) atomicAdd(status, 1);
    // to the Lagrange basis: W[k][q] = sum_b I[k][b] Vinv[b][q]
    for (int kk = 0; kk < 4; ++kk)
      for (int s = 0; s < 3; ++s)
        if (lane + 32 * s < np) acc[kk * np + lane + 32 * s] = tot[kk][s];
    __syncwarp();
    double* out = vals + blk * (LB_NKERNELS * np);
    for (int q = lane; q < np; q += 32) {
      double w4[4] = {0, 0, 0, 0};
      for (int b = 0; b < np; ++b) {
        const double vb = Vinv[b * np + q];
        for (int kk = 0; kk < 4; ++kk) w4[kk] = fma(acc[kk * np + b], vb, w4[kk]);
      }
      for (int kk = 0; kk < 4; ++kk) out[kk * np + q] = w4[kk];
    }
    __syncwarp();
  }
}

extern "C" int lb_build_corrections(lb_ctx* c) {
  if (!c) return lb_fail(nullptr, LB_EINVAL, "null context");
  if (!c->have_geom) return lb_fail(c, LB_ESTATE, "no geometry uploaded");
  LB_CUDA(c, cudaSetDevice(c->device));
  if (!c->have_near) LB_CHECK(lb_build_near(c));
  const int np = c->np;
  if (np > 96) return lb_fail(c, LB_EINVAL, "order too high for the quadrature kernel");
  double gx[QM], gw[QM];
  gauss_legendre01(QM, gx, gw);
  LB_CUDA(c, cudaMemcpyToSymbolAsync(c_gx, gx, sizeof gx, 0, cudaMemcpyHostToDevice, c->stream));
  LB_CUDA(c, cudaMemcpyToSymbolAsync(c_gw, gw, sizeof gw, 0, cudaMemcpyHostToDevice, c->stream));
  // Lebesgue constant of the node set: max over a fine grid of T0 of
  // sum_q |l_q(u, v)|, l_q(u, v) = sum_b phi_b(u, v) Vinv[b][q]
  double leb = 1.0;
  {
    const int G = 60;
    std::vector<double> ph(np);
    for (int a = 0; a <= G; ++a)
      for (int bb = 0; a + bb <= G; ++bb) {
        lb_basis_eval(c->order, (double)a / G, (double)bb / G,
                      [&](int b, double f, double, double) { ph[b] = f; });
        double sum = 0;
        for (int q = 0; q < np; ++q) {
          double l = 0;
          for (int b = 0; b < np; ++b) l += ph[b] * c->Vinv[(size_t)b * np + q];
          sum += std::fabs(l);
        }
        leb = std::max(leb, sum);
      }
  }
  lb_free(&c->vals_hi);
  lb_free(&c->vals_lo);
  lb_free(&c->phi0);
  c->phi0_prec = -1;
  lb_free_transpose(c);
  LB_CHECK(lb_alloc(c, &c->vals, (size_t)c->nnzb * LB_NKERNELS * np));
  LB_CHECK(lb_ensure(c, c->ws_quad, (size_t)(3 * c->npatch * np + 16) * sizeof(double)));
  double* cX = (double*)c->ws_quad.p;
  int* status = (int*)(cX + 3 * c->npatch * np);
  LB_CUDA(c, cudaMemsetAsync(status, 0, sizeof(int), c->stream));
  k_chart_coeffs<<<lb_div_up(c->npatch * np, 128), 128, 0, c->stream>>>(c->npatch, np, c->X, c->dVinv, cX);
  LB_LAUNCH(c);
  const size_t shm = (size_t)QWARPS * (32 * np + 32 * 4 + 4 * np) * sizeof(double);
  LB_CUDA(c, cudaFuncSetAttribute(k_near_quad, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm));
  const unsigned grid = (unsigned)std::min<int64_t>(lb_div_up(c->nnzb, QWARPS), 8LL * c->sm_count);
  ProfScope prof(c, LB_PROF_QUAD);
  k_near_quad<<<grid, 32 * QWARPS, shm, c->stream>>>(c->N, np, c->order, c->row_ptr, c->near_patch, c->nnzb, c->X,
                                                     c->inrm, c->dref, cX, c->dVinv, c->area_p, c->rad,
                                                     c->params.eps_quad, leb, c->vals, status);
  LB_LAUNCH(c);
  int bad = 0;
  LB_CUDA(c, cudaMemcpyAsync(&bad, status, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  LB_CUDA(c, cudaStreamSynchronize(c->stream));
  c->have_corr = true;
  if (bad)
    return lb_fail(c, LB_EGEOM, "near quadrature hit its depth/stack/cell limit on %d blocks (results kept)", bad);
  return LB_OK;
}
