// Orthonormal polynomials of total degree <= k on T0 = {u, v >= 0, u + v <= 1}.
//
// A patch chart and every density are polynomials of total degree <= k on
// each patch, known by their samples at the node rule (Section 4).  The
// library works in the orthonormal collapsed-coordinate basis
//   phi_{n,m}(u, v) = sqrt(2 (2n+1)(n+m+1)) A_n(u, v) B_{n,m}(v),  n + m <= k,
//   A_n = (1-v)^n Leg_n((2u - 1 + v)/(1 - v))   (homogeneous, a polynomial),
//   B_{n,m} = Jac_m^{(2n+1, 0)}(2v - 1),
// evaluated with value and first derivatives by three-term recurrences.
// Basis index b runs over n (outer) and m (inner).
#pragma once

#define LB_MAX_ORDER 10

// Calls f(b, phi, dphi/du, dphi/dv) for every basis function at (u, v).
template <class F>
__host__ __device__ inline void lb_basis_eval(int k, double u, double v, F&& f) {
  const double s = 1.0 - v;
  const double a1 = 2.0 * u - s;  // A_1
  double A = 1.0, Au = 0.0, Av = 0.0;          // A_n and derivatives
  double Ap = 0.0, Apu = 0.0, Apv = 0.0;       // A_{n-1}
  const double x = 2.0 * v - 1.0;
  int b = 0;
  for (int n = 0; n <= k; ++n) {
    if (n == 1) {
      Ap = A; Apu = Au; Apv = Av;
      A = a1; Au = 2.0; Av = 1.0;
    } else if (n >= 2) {
      const int j = n - 1;  // A_{j+1} from A_j, A_{j-1}
      const double c1 = (2.0 * j + 1.0), c2 = (double)j, d = 1.0 / (j + 1.0);
      const double An = (c1 * a1 * A - c2 * s * s * Ap) * d;
      const double Anu = (c1 * (2.0 * A + a1 * Au) - c2 * s * s * Apu) * d;
      const double Anv = (c1 * (A + a1 * Av) - c2 * (-2.0 * s * Ap + s * s * Apv)) * d;
      Ap = A; Apu = Au; Apv = Av;
      A = An; Au = Anu; Av = Anv;
    }
    // Jacobi P_m^{(al,0)}(x) and d/dx by recurrence in m
    const double al = 2.0 * n + 1.0;
    double P = 1.0, dP = 0.0, Pm = 0.0, dPm = 0.0;
    for (int m = 0; m + n <= k; ++m) {
      if (m == 1) {
        Pm = P; dPm = dP;
        P = 0.5 * ((al + 2.0) * x + al);
        dP = 0.5 * (al + 2.0);
      } else if (m >= 2) {
        const double c0 = 2.0 * m * (m + al) * (2.0 * m + al - 2.0);
        const double ca = (2.0 * m + al - 1.0) * (2.0 * m + al) * (2.0 * m + al - 2.0);
        const double cb = (2.0 * m + al - 1.0) * al * al;
        const double cc = 2.0 * (m + al - 1.0) * (m - 1.0) * (2.0 * m + al);
        const double Pn = ((ca * x + cb) * P - cc * Pm) / c0;
        const double dPn = (ca * P + (ca * x + cb) * dP - cc * dPm) / c0;
        Pm = P; dPm = dP;
        P = Pn; dP = dPn;
      }
      const double nrm = sqrt(2.0 * (2.0 * n + 1.0) * (n + m + 1.0));
      // d/dv of B(2v-1) = 2 P'(x)
      f(b, nrm * A * P, nrm * Au * P, nrm * (Av * P + A * 2.0 * dP));
      ++b;
    }
  }
}

// Basis at p = a + (du, dv) together with the differences phi_b(p) - phi_b(a).
// The differences run through the same recurrences by the product rule
// D(P Q) = DP Q(p) + P(a) DQ, starting from Du = du, Dv = dv, so they keep
// full relative accuracy however close p is to a.  Calls
// f(b, phi(p), dphi/du(p), dphi/dv(p), phi(p) - phi(a)).
template <class F>
__host__ __device__ inline void lb_basis_eval_diff(int k, double ua, double va, double du, double dv, F&& f) {
  const double u = ua + du, v = va + dv;
  const double sa = 1.0 - va, sp = 1.0 - v, ds = -dv;
  const double ds2 = ds * (sp + sa);
  const double a1a = 2.0 * ua - sa, a1p = 2.0 * u - sp, da1 = 2.0 * du + dv;
  // A_n at a (Aa), at p with derivatives (A, Au, Av), and the difference dA
  double Aa = 1.0, A = 1.0, Au = 0.0, Av = 0.0, dA = 0.0;
  double Aam = 0.0, Am = 0.0, Aum = 0.0, Avm = 0.0, dAm = 0.0;
  const double xa = 2.0 * va - 1.0, xp = 2.0 * v - 1.0, dx = 2.0 * dv;
  int b = 0;
  for (int n = 0; n <= k; ++n) {
    if (n == 1) {
      Aam = Aa; Am = A; Aum = Au; Avm = Av; dAm = dA;
      Aa = a1a; A = a1p; Au = 2.0; Av = 1.0; dA = da1;
    } else if (n >= 2) {
      const int j = n - 1;
      const double c1 = 2.0 * j + 1.0, c2 = (double)j, inv = 1.0 / (j + 1.0);
      const double nAa = (c1 * a1a * Aa - c2 * sa * sa * Aam) * inv;
      const double nA = (c1 * a1p * A - c2 * sp * sp * Am) * inv;
      const double nAu = (c1 * (2.0 * A + a1p * Au) - c2 * sp * sp * Aum) * inv;
      const double nAv = (c1 * (A + a1p * Av) - c2 * (-2.0 * sp * Am + sp * sp * Avm)) * inv;
      const double ndA = (c1 * (da1 * A + a1a * dA) - c2 * (ds2 * Am + sa * sa * dAm)) * inv;
      Aam = Aa; Am = A; Aum = Au; Avm = Av; dAm = dA;
      Aa = nAa; A = nA; Au = nAu; Av = nAv; dA = ndA;
    }
    const double al = 2.0 * n + 1.0;
    double Pa = 1.0, P = 1.0, dP = 0.0, dPx = 0.0;        // at a, at p, d/dx at p, difference
    double Pam = 0.0, Pm = 0.0, dPm = 0.0, dPxm = 0.0;
    for (int m = 0; m + n <= k; ++m) {
      if (m == 1) {
        Pam = Pa; Pm = P; dPm = dP; dPxm = dPx;
        Pa = 0.5 * ((al + 2.0) * xa + al);
        P = 0.5 * ((al + 2.0) * xp + al);
        dP = 0.5 * (al + 2.0);
        dPx = 0.5 * (al + 2.0) * dx;
      } else if (m >= 2) {
        const double c0 = 2.0 * m * (m + al) * (2.0 * m + al - 2.0);
        const double ca = (2.0 * m + al - 1.0) * (2.0 * m + al) * (2.0 * m + al - 2.0);
        const double cb = (2.0 * m + al - 1.0) * al * al;
        const double cc = 2.0 * (m + al - 1.0) * (m - 1.0) * (2.0 * m + al);
        const double nPa = ((ca * xa + cb) * Pa - cc * Pam) / c0;
        const double nP = ((ca * xp + cb) * P - cc * Pm) / c0;
        const double ndP = (ca * P + (ca * xp + cb) * dP - cc * dPm) / c0;
        const double ndPx = (ca * dx * P + (ca * xa + cb) * dPx - cc * dPxm) / c0;
        Pam = Pa; Pm = P; dPm = dP; dPxm = dPx;
        Pa = nPa; P = nP; dP = ndP; dPx = ndPx;
      }
      const double nrm = sqrt(2.0 * (2.0 * n + 1.0) * (n + m + 1.0));
      f(b, nrm * A * P, nrm * Au * P, nrm * (Av * P + A * 2.0 * dP), nrm * (dA * P + Aa * dPx));
      ++b;
    }
  }
}
