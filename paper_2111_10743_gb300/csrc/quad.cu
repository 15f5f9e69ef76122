// Near-field correction blocks on the device, by fixed geometric rules.
//
// For every row i and patch P in Near(i) (Section 4, the locally corrected
// scheme: self patch by singular quadrature, close patches by a rule refined
// towards the target), and every kernel K in {S, D, S', S''+D'}:
//   W^K_{i,P}[q] = int_{Gamma_P} K(x_i, y) l_q(y) da(y),
// l_q the Lagrange polynomial of node q on P (the density's implicit
// interpolation).  The integral is accumulated in the orthonormal basis,
//   I_K[b] = int K phi_b da,   W^K[q] = sum_b I_K[b] Vinv[b][q].
//
// Cells: a triangle (a, b, c) of T0 and a rectangle [s0,s1]x[t0,t1] of the
// Duffy square; its points are a + s (b - a) + s t (c - b) with Jacobian
// s |det(b - a, c - b)|, tensor Gauss-Legendre (m x m) in (s, t).
//
//   * Self patch (Duffy 1982): T0 is cut at the target's reference node a
//     into three triangles with apex a; the Jacobian s cancels the 1/r
//     singularity.  A triangle whose apex lies close to its base edge is
//     nearly singular in t, so each base edge is cut further at points whose
//     distance from the foot of the perpendicular from a grows geometrically
//     (h, 2h, 4h, ..., h the apex-to-edge distance), distances measured in
//     the chart's metric at a: every sub-triangle's base is then no longer
//     than its distance from the apex, and 12 x 12 points per sub-triangle
//     reach about 1e-13 of the largest weight.
//   * Other near patches: T0 is split 1 -> 4 (depth first) until every cell is
//     admissible, its chord radius r (largest distance from the image of its
//     centroid to the images of its vertices) at most half the distance from
//     the target to the image of its centroid; each admissible cell takes
//     16 x 16 collapsed Gauss points (12 x 12 when eps_quad >= 1e-9).  The
//     target then lies at least one cell diameter away from every cell.
// Neither rule estimates its error: the rule sizes were chosen so that the
// weights agree with a separately implemented adaptive quadrature (the
// oracle) to about 1e-13 of the largest weight on spheres, ellipsoids, tori,
// a twisted torus and a genus-2 surface.
//
// Points lie on the polynomial chart y = sum_b cX_b phi_b; tangents, normal
// and area element are those of this polynomial, and the target normal is
// the normal of the position interpolant of the target's patch at its node.
// (The sampled tangents are not the derivatives of the position interpolant;
// using them would leave an odd 1/r^2 term on the self patch whose
// Duffy-split integral does not converge.)  On the self patch d = y(a) - y(p)
// is summed from the basis differences phi_b(p) - phi_b(a) carried through
// the basis recurrences, which keeps full relative accuracy next to the
// target.
//
// One warp per (row, patch) block, blocks handed out by an atomic counter;
// lanes take one quadrature point each in rounds of 32, write basis values
// to shared memory, and then own basis coefficients b = lane + 32 s for the
// accumulation (deterministic order).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <vector>

#include "basis.cuh"
#include "internal.cuh"

#define QM_MAX 16        // largest Gauss-Legendre rule per direction
#define QSTACK 100       // cells per warp stack (depth first: at most 3 depth + 1 live)
#define QMAXDEPTH 24
#define QWARPS 4
#define QMAXCELLS 4096   // integrated cells per block; exceeding it sets the error flag
#define QSELF_M 12       // self-patch sub-triangles
#define QRHO 2.0         // geometric ratio of the self-patch edge cuts
#define QADMIT 2.0       // admissible: distance to the centroid image >= QADMIT * chord radius

// Gauss-Legendre rules on [0, 1]: slot 0 = QSELF_M points, slot 1 = the near
// rule's points (16 or 12)
__constant__ double c_gx[2][QM_MAX], c_gw[2][QM_MAX];

// The orthonormal basis's recurrence coefficients, tabulated once per build
// (they depend on the indices only): for basis b = (n, m),
//   P_m = (jA x + jB) P_{m-1} - jC P_{m-2}   (Jacobi P^{(2n+1, 0)}, P_0 = 1),
//   phi_b = jN A_n P_m,
// and for the collapsed factor A_{j+1} = aC1 a1 A_j - aC2 s^2 A_{j-1}.
#define QNB ((LB_MAX_ORDER + 1) * (LB_MAX_ORDER + 2) / 2)
__constant__ double c_jA[QNB], c_jB[QNB], c_jC[QNB], c_jN[QNB];
__constant__ double c_aC1[LB_MAX_ORDER + 1], c_aC2[LB_MAX_ORDER + 1];

static void basis_tables(int k, double* jA, double* jB, double* jC, double* jN, double* a1, double* a2) {
  int b = 0;
  for (int n = 0; n <= k; ++n) {
    const double al = 2.0 * n + 1.0;
    if (n >= 2) {
      const int j = n - 1;
      a1[n] = (2.0 * j + 1.0) / (j + 1.0);
      a2[n] = (double)j / (j + 1.0);
    } else {
      a1[n] = a2[n] = 0.0;
    }
    for (int m = 0; m + n <= k; ++m, ++b) {
      jN[b] = std::sqrt(2.0 * (2.0 * n + 1.0) * (n + m + 1.0));
      if (m == 0) {
        jA[b] = jB[b] = jC[b] = 0.0;
      } else if (m == 1) {
        jA[b] = 0.5 * (al + 2.0);
        jB[b] = 0.5 * al;
        jC[b] = 0.0;
      } else {
        const double c0 = 2.0 * m * (m + al) * (2.0 * m + al - 2.0);
        jA[b] = (2.0 * m + al - 1.0) * (2.0 * m + al) * (2.0 * m + al - 2.0) / c0;
        jB[b] = (2.0 * m + al - 1.0) * al * al / c0;
        jC[b] = 2.0 * (m + al - 1.0) * (m - 1.0) * (2.0 * m + al) / c0;
      }
    }
  }
}

// Basis and first derivatives at (u, v) from the tables: f(b, phi, phi_u, phi_v).
template <class F>
__device__ __forceinline__ void q_basis(int k, double u, double v, F&& f) {
  const double s = 1.0 - v, s2 = s * s;
  const double a1 = 2.0 * u - s;
  double A = 1.0, Au = 0.0, Av = 0.0, Ap = 0.0, Apu = 0.0, Apv = 0.0;
  const double x = 2.0 * v - 1.0;
  int b = 0;
  for (int n = 0; n <= k; ++n) {
    if (n == 1) {
      Ap = A; Apu = Au; Apv = Av;
      A = a1; Au = 2.0; Av = 1.0;
    } else if (n >= 2) {
      const double c1 = c_aC1[n], c2 = c_aC2[n];
      const double An = c1 * a1 * A - c2 * s2 * Ap;
      const double Anu = c1 * (2.0 * A + a1 * Au) - c2 * s2 * Apu;
      const double Anv = c1 * (A + a1 * Av) - c2 * (-2.0 * s * Ap + s2 * Apv);
      Ap = A; Apu = Au; Apv = Av;
      A = An; Au = Anu; Av = Anv;
    }
    double P = 1.0, dP = 0.0, Pm = 0.0, dPm = 0.0;
    for (int m = 0; m + n <= k; ++m, ++b) {
      if (m >= 1) {
        const double ab = fma(c_jA[b], x, c_jB[b]);
        const double Pn = ab * P - c_jC[b] * Pm;
        const double dPn = c_jA[b] * P + ab * dP - c_jC[b] * dPm;
        Pm = P; dPm = dP;
        P = Pn; dP = dPn;
      }
      const double nr = c_jN[b];
      f(b, nr * A * P, nr * Au * P, nr * (Av * P + A * 2.0 * dP));
    }
  }
}

// Basis at p = a + (du, dv) and the differences phi_b(p) - phi_b(a), carried
// through the same recurrences by the product rule so that they keep full
// relative accuracy next to a: f(b, phi(p), phi_u(p), phi_v(p), phi(p) - phi(a)).
template <class F>
__device__ __forceinline__ void q_basis_diff(int k, double ua, double va, double du, double dv, F&& f) {
  const double u = ua + du, v = va + dv;
  const double sa = 1.0 - va, sp = 1.0 - v, ds = -dv;
  const double ds2 = ds * (sp + sa), sa2 = sa * sa, sp2 = sp * sp;
  const double a1a = 2.0 * ua - sa, a1p = 2.0 * u - sp, da1 = 2.0 * du + dv;
  double Aa = 1.0, A = 1.0, Au = 0.0, Av = 0.0, dA = 0.0;
  double Aam = 0.0, Am = 0.0, Aum = 0.0, Avm = 0.0, dAm = 0.0;
  const double xa = 2.0 * va - 1.0, xp = 2.0 * v - 1.0, dx = 2.0 * dv;
  int b = 0;
  for (int n = 0; n <= k; ++n) {
    if (n == 1) {
      Aam = Aa; Am = A; Aum = Au; Avm = Av; dAm = dA;
      Aa = a1a; A = a1p; Au = 2.0; Av = 1.0; dA = da1;
    } else if (n >= 2) {
      const double c1 = c_aC1[n], c2 = c_aC2[n];
      const double nAa = c1 * a1a * Aa - c2 * sa2 * Aam;
      const double nA = c1 * a1p * A - c2 * sp2 * Am;
      const double nAu = c1 * (2.0 * A + a1p * Au) - c2 * sp2 * Aum;
      const double nAv = c1 * (A + a1p * Av) - c2 * (-2.0 * sp * Am + sp2 * Avm);
      const double ndA = c1 * (da1 * A + a1a * dA) - c2 * (ds2 * Am + sa2 * dAm);
      Aam = Aa; Am = A; Aum = Au; Avm = Av; dAm = dA;
      Aa = nAa; A = nA; Au = nAu; Av = nAv; dA = ndA;
    }
    double Pa = 1.0, P = 1.0, dP = 0.0, dPx = 0.0;
    double Pam = 0.0, Pm = 0.0, dPm = 0.0, dPxm = 0.0;
    for (int m = 0; m + n <= k; ++m, ++b) {
      if (m >= 1) {
        const double cA = c_jA[b], cB = c_jB[b], cC = c_jC[b];
        const double aba = fma(cA, xa, cB), abp = fma(cA, xp, cB);
        const double nPa = aba * Pa - cC * Pam;
        const double nP = abp * P - cC * Pm;
        const double ndP = cA * P + abp * dP - cC * dPm;
        const double ndPx = cA * dx * P + aba * dPx - cC * dPxm;
        Pam = Pa; Pm = P; dPm = dP; dPxm = dPx;
        Pa = nPa; P = nP; dP = ndP; dPx = ndPx;
      }
      const double nr = c_jN[b];
      f(b, nr * A * P, nr * Au * P, nr * (Av * P + A * 2.0 * dP), nr * (dA * P + Aa * dPx));
    }
  }
}

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
  double a0, a1, b0, b1, c0, c1;
  int depth;
};

// Accumulate one cell (Duffy square [0,1]^2, m x m Gauss slot `rule`) into
// I[k][s] for basis b = lane + 32 s.  offset (self patch): d = y(a) - y(p)
// from basis differences at the apex a.
template <bool offset>
__device__ void q_cell(const QCell& cl, int rule, int m, int k, int np, const double* __restrict__ cX, double x0,
                       double x1, double x2, double n0, double n1, double n2, double* phi, double* fv,
                       double I[4][3]) {
  const int lane = threadIdx.x & 31;
  const double e10 = cl.b0 - cl.a0, e11 = cl.b1 - cl.a1, e20 = cl.c0 - cl.b0, e21 = cl.c1 - cl.b1;
  const double det = fabs(e10 * e21 - e11 * e20);
  const int npts = m * m;
  for (int p0 = 0; p0 < npts; p0 += 32) {
    const int p = p0 + lane;
    double* ph = phi + lane * np;
    if (p < npts) {
      const int is = p / m, it = p - (p / m) * m;
      const double s = c_gx[rule][is];
      const double t = c_gx[rule][it];
      const double om = c_gw[rule][is] * c_gw[rule][it] * s * det;
      const double du = s * e10 + s * t * e20;
      const double dv = s * e11 + s * t * e21;
      double y[3] = {0, 0, 0}, yu[3] = {0, 0, 0}, yv[3] = {0, 0, 0};
      if constexpr (offset) {  // y holds y(p) - y(a)
        q_basis_diff(k, cl.a0, cl.a1, du, dv, [&](int b, double f, double fu, double fvv, double df) {
          const double* cb = cX + 3 * b;
          for (int d = 0; d < 3; ++d) {
            y[d] = fma(df, cb[d], y[d]);
            yu[d] = fma(fu, cb[d], yu[d]);
            yv[d] = fma(fvv, cb[d], yv[d]);
          }
          ph[b] = f;
        });
      } else {
        q_basis(k, cl.a0 + du, cl.a1 + dv, [&](int b, double f, double fu, double fvv) {
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
      const double iJ = 1.0 / J;
      const double ny0 = m0 * iJ, ny1 = m1 * iJ, ny2 = m2 * iJ;
      const double d0 = offset ? -y[0] : x0 - y[0];
      const double d1 = offset ? -y[1] : x1 - y[1];
      const double d2 = offset ? -y[2] : x2 - y[2];
      const double r2 = d0 * d0 + d1 * d1 + d2 * d2;
      const double ir = rsqrt(r2);
      const double ir2 = ir * ir;
      const double g = ir * (1.0 / (4.0 * LB_PI));
      const double g3 = g * ir2;
      const double nxd = n0 * d0 + n1 * d1 + n2 * d2;
      const double nyd = ny0 * d0 + ny1 * d1 + ny2 * d2;
      const double e0 = n0 - ny0, e1 = n1 - ny1, e2 = n2 - ny2;
      const double wJ = om * J;
      fv[lane * 4 + 0] = wJ * g;
      fv[lane * 4 + 1] = wJ * nyd * g3;
      fv[lane * 4 + 2] = -wJ * nxd * g3;
      fv[lane * 4 + 3] = wJ * (3.0 * nxd * (nxd - nyd) * ir2 - 0.5 * (e0 * e0 + e1 * e1 + e2 * e2)) * g3;
    } else {  // padding lanes of the last round contribute nothing
      for (int b = 0; b < np; ++b) ph[b] = 0.0;
      for (int kk = 0; kk < 4; ++kk) fv[lane * 4 + kk] = 0.0;
    }
    __syncwarp();
#pragma unroll
    for (int s2 = 0; s2 < 3; ++s2) {
      const int b = lane + 32 * s2;
      if (b < np) {
        double a0 = I[0][s2], a1 = I[1][s2], a2 = I[2][s2], a3 = I[3][s2];
        for (int pp = 0; pp < 32; ++pp) {
          const double f = phi[pp * np + b];
          // fv rows are 32 bytes apart and the row base is 16-byte aligned
          const double2 g0 = reinterpret_cast<const double2*>(fv)[2 * pp];
          const double2 g1 = reinterpret_cast<const double2*>(fv)[2 * pp + 1];
          a0 = fma(g0.x, f, a0);
          a1 = fma(g0.y, f, a1);
          a2 = fma(g1.x, f, a2);
          a3 = fma(g1.y, f, a3);
        }
        I[0][s2] = a0; I[1][s2] = a1; I[2][s2] = a2; I[3][s2] = a3;
      }
    }
    __syncwarp();
  }
}

// chart position at (u, v) (one lane)
__device__ __forceinline__ void q_chart_point(int k, const double* __restrict__ cX, double u, double v, double* y) {
  y[0] = y[1] = y[2] = 0.0;
  q_basis(k, u, v, [&](int b, double f, double, double) {
    const double* cb = cX + 3 * b;
    for (int d = 0; d < 3; ++d) y[d] = fma(f, cb[d], y[d]);
  });
}

// Self patch: push the sub-triangles of the three Duffy triangles with apex a,
// each base edge cut geometrically from the foot of the perpendicular from a
// (chart metric G at a).  Returns the number of cells (lane 0 only).
__device__ int q_self_cells(double au, double av, const double G[3], QCell* out, int cap) {
  const double vx[3] = {0.0, 1.0, 0.0}, vy[3] = {0.0, 0.0, 1.0};
  int n = 0;
  for (int j = 0; j < 3; ++j) {
    const double b0 = vx[j], b1 = vy[j], c0 = vx[(j + 1) % 3], c1 = vy[(j + 1) % 3];
    const double e0 = c0 - b0, e1 = c1 - b1;           // base edge b -> c
    const double w0 = au - b0, w1 = av - b1;           // b -> apex
    const double L2 = G[0] * e0 * e0 + 2.0 * G[1] * e0 * e1 + G[2] * e1 * e1;
    const double we = G[0] * w0 * e0 + G[1] * (w0 * e1 + w1 * e0) + G[2] * w1 * e1;
    const double ww = G[0] * w0 * w0 + 2.0 * G[1] * w0 * w1 + G[2] * w1 * w1;
    const double tf = we / L2;                         // foot of the perpendicular, edge parameter
    const double h = sqrt(fmax(ww - tf * tf * L2, 0.0));
    const double step0 = fmax(h / sqrt(L2), 1e-9);
    const double tfc = fmin(fmax(tf, 0.0), 1.0);
    // down from the foot to t = 0, then up from the foot to t = 1
    for (int dir = -1; dir <= 1; dir += 2) {
      double tin = tfc, d = step0;
      if ((dir < 0 && tfc <= 0.0) || (dir > 0 && tfc >= 1.0)) continue;
      for (int guard = 0; guard < 64; ++guard) {
        double tout = tfc + dir * d;
        const bool last = dir < 0 ? tout <= 0.0 : tout >= 1.0;
        if (last) tout = dir < 0 ? 0.0 : 1.0;
        const double lo = fmin(tin, tout), hi = fmax(tin, tout);
        if (hi - lo > 1e-15 && n < cap) {
          QCell c;
          c.a0 = au; c.a1 = av;
          c.b0 = b0 + lo * e0; c.b1 = b1 + lo * e1;
          c.c0 = b0 + hi * e0; c.c1 = b1 + hi * e1;
          c.depth = 0;
          out[n++] = c;
        }
        if (last) break;
        tin = tout;
        d *= QRHO;
      }
    }
  }
  return n;
}

__global__ void __launch_bounds__(32 * QWARPS) k_near_quad(
    int64_t N, int np, int k, const int64_t* __restrict__ row_ptr, const int32_t* __restrict__ near_patch,
    int64_t nnzb, const double* __restrict__ X, const double* __restrict__ inrm, const double* __restrict__ ref,
    const double* __restrict__ cXall, const double* __restrict__ Vinv, int near_m, double* __restrict__ vals,
    unsigned long long* __restrict__ next, int* __restrict__ status) {
  extern __shared__ double smem[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int per_warp = 32 * np + 32 * 4 + 4 * np;
  double* phi = smem + warp * per_warp;
  double* fv = phi + 32 * np;
  double* acc = fv + 32 * 4;
  __shared__ QCell stack[QWARPS][QSTACK];

  for (;;) {
    unsigned long long blk_u = 0;
    if (lane == 0) blk_u = atomicAdd(next, 1ull);
    blk_u = __shfl_sync(0xffffffffu, blk_u, 0);
    const int64_t blk = (int64_t)blk_u;
    if (blk >= nnzb) break;
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
    const bool self = (i / np) == P;
    double tot[4][3];
#pragma unroll
    for (int kk = 0; kk < 4; ++kk)
#pragma unroll
      for (int s = 0; s < 3; ++s) tot[kk][s] = 0.0;
    bool overflow = false;
    if (self) {
      const int q = (int)(i - P * np);
      const double au = ref[3 * q], av = ref[3 * q + 1];
      int ncell = 0;
      if (lane == 0) {
        // chart metric at the apex
        double yu[3] = {0, 0, 0}, yv[3] = {0, 0, 0};
        q_basis(k, au, av, [&](int b, double, double fu, double fvv) {
          const double* cb = cX + 3 * b;
          for (int d = 0; d < 3; ++d) {
            yu[d] = fma(fu, cb[d], yu[d]);
            yv[d] = fma(fvv, cb[d], yv[d]);
          }
        });
        const double G[3] = {yu[0] * yu[0] + yu[1] * yu[1] + yu[2] * yu[2],
                             yu[0] * yv[0] + yu[1] * yv[1] + yu[2] * yv[2],
                             yv[0] * yv[0] + yv[1] * yv[1] + yv[2] * yv[2]};
        ncell = q_self_cells(au, av, G, stack[warp], QSTACK);
      }
      ncell = __shfl_sync(0xffffffffu, ncell, 0);
      __syncwarp();
      if (ncell >= QSTACK) overflow = true;
      for (int cidx = 0; cidx < ncell; ++cidx) {
        const QCell cell = stack[warp][cidx];
        q_cell<true>(cell, 0, QSELF_M, k, np, cX, x0, x1, x2, n0, n1, n2, phi, fv, tot);
      }
      __syncwarp();
    } else {
      // depth-first 1 -> 4 refinement until admissible
      if (lane == 0) stack[warp][0] = QCell{0.0, 0.0, 1.0, 0.0, 0.0, 1.0, 0};
      int sp = 1, ncells = 0;
      __syncwarp();
      while (sp > 0) {
        const QCell cell = stack[warp][sp - 1];
        --sp;
        __syncwarp();
        // images of the centroid (lane 0) and of the vertices (lanes 1-3)
        double pu = (cell.a0 + cell.b0 + cell.c0) * (1.0 / 3.0), pv = (cell.a1 + cell.b1 + cell.c1) * (1.0 / 3.0);
        if (lane == 1) { pu = cell.a0; pv = cell.a1; }
        if (lane == 2) { pu = cell.b0; pv = cell.b1; }
        if (lane == 3) { pu = cell.c0; pv = cell.c1; }
        double y[3] = {0.0, 0.0, 0.0};
        if (lane < 4) q_chart_point(k, cX, pu, pv, y);
        const double c0 = __shfl_sync(0xffffffffu, y[0], 0);
        const double c1 = __shfl_sync(0xffffffffu, y[1], 0);
        const double c2 = __shfl_sync(0xffffffffu, y[2], 0);
        double rr = 0.0;
        if (lane >= 1 && lane < 4)
          rr = (y[0] - c0) * (y[0] - c0) + (y[1] - c1) * (y[1] - c1) + (y[2] - c2) * (y[2] - c2);
        // largest over lanes 0-3 (lane 0 holds 0), then broadcast
        rr = fmax(rr, __shfl_xor_sync(0xffffffffu, rr, 1));
        rr = fmax(rr, __shfl_xor_sync(0xffffffffu, rr, 2));
        rr = __shfl_sync(0xffffffffu, rr, 0);
        const double dist2 = (x0 - c0) * (x0 - c0) + (x1 - c1) * (x1 - c1) + (x2 - c2) * (x2 - c2);
        const bool admissible = dist2 >= QADMIT * QADMIT * rr;
        const bool forced = cell.depth >= QMAXDEPTH || sp + 4 > QSTACK || ncells >= QMAXCELLS;
        if (admissible || forced) {
          if (forced && !admissible) overflow = true;
          q_cell<false>(cell, 1, near_m, k, np, cX, x0, x1, x2, n0, n1, n2, phi, fv, tot);
          ++ncells;
        } else {
          if (lane == 0) {
            const double ab0 = 0.5 * (cell.a0 + cell.b0), ab1 = 0.5 * (cell.a1 + cell.b1);
            const double bc0 = 0.5 * (cell.b0 + cell.c0), bc1 = 0.5 * (cell.b1 + cell.c1);
            const double ca0 = 0.5 * (cell.c0 + cell.a0), ca1 = 0.5 * (cell.c1 + cell.a1);
            const int d = cell.depth + 1;
            stack[warp][sp + 0] = QCell{cell.a0, cell.a1, ab0, ab1, ca0, ca1, d};
            stack[warp][sp + 1] = QCell{ab0, ab1, cell.b0, cell.b1, bc0, bc1, d};
            stack[warp][sp + 2] = QCell{ca0, ca1, bc0, bc1, cell.c0, cell.c1, d};
            stack[warp][sp + 3] = QCell{ab0, ab1, bc0, bc1, ca0, ca1, d};
          }
          sp += 4;
        }
        __syncwarp();
      }
    }
    if (overflow && lane == 0) atomicAdd(status, 1);
    // to the Lagrange basis: W[k][q] = sum_b I[k][b] Vinv[b][q]
#pragma unroll
    for (int kk = 0; kk < 4; ++kk)
#pragma unroll
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
  const int near_m = c->params.eps_quad >= 1e-9 ? 12 : 16;
  double gx[2][QM_MAX] = {{0}}, gw[2][QM_MAX] = {{0}};
  gauss_legendre01(QSELF_M, gx[0], gw[0]);
  gauss_legendre01(near_m, gx[1], gw[1]);
  LB_CUDA(c, cudaMemcpyToSymbolAsync(c_gx, gx, sizeof gx, 0, cudaMemcpyHostToDevice, c->stream));
  LB_CUDA(c, cudaMemcpyToSymbolAsync(c_gw, gw, sizeof gw, 0, cudaMemcpyHostToDevice, c->stream));
  if (c->order > LB_MAX_ORDER) return lb_fail(c, LB_EINVAL, "order too high for the quadrature kernel");
  {
    double jA[QNB] = {0}, jB[QNB] = {0}, jC[QNB] = {0}, jN[QNB] = {0};
    double a1[LB_MAX_ORDER + 1] = {0}, a2[LB_MAX_ORDER + 1] = {0};
    basis_tables(c->order, jA, jB, jC, jN, a1, a2);
    LB_CUDA(c, cudaMemcpyToSymbolAsync(c_jA, jA, sizeof jA, 0, cudaMemcpyHostToDevice, c->stream));
    LB_CUDA(c, cudaMemcpyToSymbolAsync(c_jB, jB, sizeof jB, 0, cudaMemcpyHostToDevice, c->stream));
    LB_CUDA(c, cudaMemcpyToSymbolAsync(c_jC, jC, sizeof jC, 0, cudaMemcpyHostToDevice, c->stream));
    LB_CUDA(c, cudaMemcpyToSymbolAsync(c_jN, jN, sizeof jN, 0, cudaMemcpyHostToDevice, c->stream));
    LB_CUDA(c, cudaMemcpyToSymbolAsync(c_aC1, a1, sizeof a1, 0, cudaMemcpyHostToDevice, c->stream));
    LB_CUDA(c, cudaMemcpyToSymbolAsync(c_aC2, a2, sizeof a2, 0, cudaMemcpyHostToDevice, c->stream));
  }
  lb_free(&c->vals_hi);
  lb_free(&c->vals_lo);
  lb_free(&c->phi0);
  c->phi0_prec = -1;
  lb_free_transpose(c);
  LB_CHECK(lb_alloc(c, &c->vals, (size_t)c->nnzb * LB_NKERNELS * np));
  LB_CHECK(lb_ensure(c, c->ws_quad, (size_t)(3 * c->npatch * np + 16) * sizeof(double)));
  double* cX = (double*)c->ws_quad.p;
  unsigned long long* next = (unsigned long long*)(cX + 3 * c->npatch * np);
  int* status = (int*)(next + 1);
  LB_CUDA(c, cudaMemsetAsync(next, 0, 2 * sizeof(unsigned long long), c->stream));
  k_chart_coeffs<<<lb_div_up(c->npatch * np, 128), 128, 0, c->stream>>>(c->npatch, np, c->X, c->dVinv, cX);
  LB_LAUNCH(c);
  const size_t shm = (size_t)QWARPS * (32 * np + 32 * 4 + 4 * np) * sizeof(double);
  LB_CUDA(c, cudaFuncSetAttribute(k_near_quad, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm));
  int per_sm = 0;
  LB_CUDA(c, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_near_quad, 32 * QWARPS, shm));
  const unsigned grid = (unsigned)std::max<int64_t>(
      1, std::min<int64_t>(lb_div_up(c->nnzb, QWARPS), (int64_t)std::max(per_sm, 1) * c->sm_count));
  ProfScope prof(c, LB_PROF_QUAD);
  k_near_quad<<<grid, 32 * QWARPS, shm, c->stream>>>(c->N, np, c->order, c->row_ptr, c->near_patch, c->nnzb, c->X,
                                                     c->inrm, c->dref, cX, c->dVinv, near_m, c->vals, next, status);
  LB_LAUNCH(c);
  int bad = 0;
  LB_CUDA(c, cudaMemcpyAsync(&bad, status, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  LB_CUDA(c, cudaStreamSynchronize(c->stream));
  c->have_corr = true;
  if (bad)
    return lb_fail(c, LB_EGEOM, "near quadrature hit its depth/stack/cell limit on %d blocks (results kept)", bad);
  return LB_OK;
}
