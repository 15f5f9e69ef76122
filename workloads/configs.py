"""Named workloads: surface, right-hand sides and solver settings, all seeded.

Seeds follow numpy.random.default_rng(1000 + config index).  The shapes mirror
the paper's experiments (Section 6): closed triangulated surfaces with
high-order patches, smooth mean-zero data, GMRES to a relative residual.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

from . import implicit as I
from . import rhs as R
from . import surfaces as S


@dataclass
class Workload:
    name: str
    surface: S.Surface
    f: np.ndarray                 # [nrhs, N] raw right-hand sides (not projected)
    tol: float = 1e-10
    eps_quad: float = 1e-12
    near_factor: float = 2.0
    formulation: str = "A3"
    extra: dict = field(default_factory=dict)


def _tangential(surf: S.Surface, V: np.ndarray) -> np.ndarray:
    """F = -n x (n x V): the tangential part of V (Section 5 / Section 6.3)."""
    n = np.cross(surf.Xu, surf.Xv)
    n /= np.linalg.norm(n, axis=1, keepdims=True)
    return -np.cross(n, np.cross(n, V))


def sphere_y32(level: int = 0, order: int = 4) -> Workload:
    """Unit sphere from the icosahedron, f = Y_3^2, exact u = -f/12."""
    s = S.icosphere(level, order)
    f = R.y32(s.X)
    return Workload(f"sphere-ico{level}-k{order}", s, f[None, :], tol=1e-12, eps_quad=1e-13,
                    extra={"u_exact": -f / 12.0})


def ellipsoid_gauss(level: int = 3, order: int = 8, seed: int = 1002) -> Workload:
    """Ellipsoid (1, 1.5, 2) with a sum of 8 Gaussian bumps as data."""
    s = S.ellipsoid((1.0, 1.5, 2.0), level, order)
    rng = np.random.default_rng(seed)
    f = R.gaussian_bumps(s.X, rng)
    return Workload(f"ellipsoid-ico{level}-k{order}", s, f[None, :])


def torus_batch(n_theta: int = 32, n_phi: int = 32, order: int = 6, nrand: int = 16,
                seed: int = 1003) -> Workload:
    """Torus R=2, r=0.75: one Hodge field F plus nrand random Legendre f."""
    s = S.torus(2.0, 0.75, n_theta, n_phi, order)
    rng = np.random.default_rng(seed)
    F = _tangential(s, R.current_source_field(s.X))
    L = 2.75
    f = np.stack([R.legendre_field(s.X, rng, 4, L) for _ in range(nrand)]) if nrand else \
        np.zeros((0, s.N))
    return Workload(f"torus-{n_theta}x{n_phi}-k{order}", s, f, extra={"F": F})


def _centred(surf: S.Surface):
    """Node positions about the bounding-box centre, and the box's half-extent."""
    lo, hi = surf.X.min(axis=0), surf.X.max(axis=0)
    return surf.X - 0.5 * (lo + hi)[None, :], 0.5 * float(np.max(hi - lo))


def genus2_autograd(h: float = 0.135, order: int = 6, seed: int = 1004) -> Workload:
    """Two blended tori (genus 2), about 4,000 order-6 patches: one random
    Legendre f and a Legendre target u_t for the loss |u - u_t|^2."""
    s = I.tori_chain(2, h, order)
    rng = np.random.default_rng(seed)
    Xc, L = _centred(s)
    f = R.legendre_field(Xc, rng, 4, L)
    ut = R.legendre_field(Xc, rng, 4, L)
    return Workload(f"tori2-h{h:g}-k{order}", s, f[None, :], extra={"u_target": ut})


def genus5_batch(h: float = 0.07, order: int = 6, nF: int = 5, nrand: int = 22, seed: int = 1005) -> Workload:
    """Five blended tori (genus 5), about 36,000 order-6 patches: nF random
    tangential fields F (2 nF Hodge solves) and nrand random Legendre f."""
    s = I.tori_chain(5, h, order)
    rng = np.random.default_rng(seed)
    Xc, L = _centred(s)
    F = np.stack([_tangential(s, R.legendre_field(Xc, rng, 4, L, ncomp=3)) for _ in range(nF)])
    f = np.stack([R.legendre_field(Xc, rng, 4, L) for _ in range(nrand)])
    return Workload(f"tori5-h{h:g}-k{order}", s, f, tol=1e-9, extra={"F": F})


# the configurations of the scope table, by index
def config(index: int) -> Workload:
    if index == 1:
        return sphere_y32(0, 4)
    if index == 2:
        return ellipsoid_gauss(3, 8, 1002)
    if index == 3:
        return torus_batch(32, 32, 6, 16, 1003)
    if index == 4:
        return genus2_autograd(0.135, 6, 1004)
    if index == 5:
        return genus5_batch(0.07, 6, 5, 22, 1005)
    raise ValueError(f"configuration {index} is not built")
