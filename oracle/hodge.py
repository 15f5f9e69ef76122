"""Surface gradient of S, and the harmonic-field decomposition (oracle, FP64).

Test infrastructure only (see oracle/__init__.py).

grad S on Gamma (principal value) = n S'[sigma] + grad_Gamma S[sigma]: the
normal part is the principal-value normal derivative, the tangential part is
the surface gradient of the (continuous) potential S[sigma], computed by
nodal differentiation on each patch (Section 2).

Harmonic fields (Section 5): for a tangential field F solve
  Delta alpha = div_Gamma F,  Delta beta = -div_Gamma (n x F)
(the printed second equation names alpha; it is the equation for beta) and
set H = F - grad_Gamma alpha - n x grad_Gamma beta; n x H is the companion
harmonic field.
"""
from __future__ import annotations

import numpy as np

from .geometry import surface_divergence, surface_gradient
from .gmres import solve_lb


def grad_S(disc, sigma):
    p = disc.potentials(sigma)[0]
    g = disc.geo
    return surface_gradient(g, p[0]) + g.n * p[2][:, None]


def harmonic_field(disc, F, formulation="A3", tol=1e-10):
    g = disc.geo
    rhs_a = surface_divergence(g, F)
    rhs_b = -surface_divergence(g, np.cross(g.n, F))
    a, _, ia, _ = solve_lb(disc, rhs_a, formulation, tol)
    b, _, ib, _ = solve_lb(disc, rhs_b, formulation, tol)
    H = F - surface_gradient(g, a) - np.cross(g.n, surface_gradient(g, b))
    return H, np.cross(g.n, H), (ia, ib)
