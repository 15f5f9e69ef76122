// Host-side matrices of the node rule: Vandermonde inverse and nodal
// differentiation (Section 4: "spectral differentiation" of the sampled
// tangents for the mean curvature; Section 2 for surface gradients).
//   V_qb = phi_b(u_q, v_q),  Vinv = V^-1,  D_u = V_u Vinv,  D_v = V_v Vinv.
#include <cmath>
#include <vector>

#include "basis.cuh"
#include "internal.cuh"

// Gauss-Jordan inverse with partial pivoting; returns false when singular.
static bool invert(int n, std::vector<double> a, std::vector<double>& inv) {
  inv.assign((size_t)n * n, 0.0);
  for (int i = 0; i < n; ++i) inv[(size_t)i * n + i] = 1.0;
  for (int col = 0; col < n; ++col) {
    int piv = col;
    for (int r = col + 1; r < n; ++r)
      if (std::fabs(a[(size_t)r * n + col]) > std::fabs(a[(size_t)piv * n + col])) piv = r;
    if (!(std::fabs(a[(size_t)piv * n + col]) > 1e-13)) return false;
    if (piv != col)
      for (int k = 0; k < n; ++k) {
        std::swap(a[(size_t)piv * n + k], a[(size_t)col * n + k]);
        std::swap(inv[(size_t)piv * n + k], inv[(size_t)col * n + k]);
      }
    const double d = 1.0 / a[(size_t)col * n + col];
    for (int k = 0; k < n; ++k) {
      a[(size_t)col * n + k] *= d;
      inv[(size_t)col * n + k] *= d;
    }
    for (int r = 0; r < n; ++r) {
      if (r == col) continue;
      const double f = a[(size_t)r * n + col];
      if (f == 0.0) continue;
      for (int k = 0; k < n; ++k) {
        a[(size_t)r * n + k] -= f * a[(size_t)col * n + k];
        inv[(size_t)r * n + k] -= f * inv[(size_t)col * n + k];
      }
    }
  }
  return true;
}

int lb_host_basis_matrices(lb_ctx* c) {
  const int np = c->np, k = c->order;
  std::vector<double> V((size_t)np * np), Vu((size_t)np * np), Vv((size_t)np * np);
  for (int q = 0; q < np; ++q) {
    lb_basis_eval(k, c->ref_uv[2 * q], c->ref_uv[2 * q + 1], [&](int b, double p, double pu, double pv) {
      V[(size_t)q * np + b] = p;
      Vu[(size_t)q * np + b] = pu;
      Vv[(size_t)q * np + b] = pv;
    });
  }
  if (!invert(np, V, c->Vinv)) return lb_fail(c, LB_EGEOM, "node rule is not unisolvent for degree %d", k);
  c->Du.assign((size_t)np * np, 0.0);
  c->Dv.assign((size_t)np * np, 0.0);
  for (int q = 0; q < np; ++q)
    for (int r = 0; r < np; ++r) {
      double su = 0, sv = 0;
      for (int b = 0; b < np; ++b) {
        su += Vu[(size_t)q * np + b] * c->Vinv[(size_t)b * np + r];
        sv += Vv[(size_t)q * np + b] * c->Vinv[(size_t)b * np + r];
      }
      c->Du[(size_t)q * np + r] = su;
      c->Dv[(size_t)q * np + r] = sv;
    }
  return LB_OK;
}
