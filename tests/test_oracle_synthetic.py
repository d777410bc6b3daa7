"""Pins of the oracle's synthetic iterative scheme of the steady solver (Sec. 3.5), no GPU.

Between sweeps the scheme corrects the lattice temperature by a macroscopic (diffusion-type)
equation.  The pins check the discrete Laplacian of that equation against an independently
coded stencil and against the closed-form eigenvalues of the periodic second difference, that
the scheme's fixed point is the sequential scheme's (the steady state of the step) on every wall
mix, singular (no thermalizing wall) or not, and that it removes the slow convergence of the
sequential scheme in the near-diffusive regime, which is what the paper introduces it for.
"""
import math

import numpy as np
import pytest

from oracle.oracle import BC_DIFFUSE, BC_ISOTHERMAL, BC_PERIODIC, BC_SPECULAR, LIM_FIRST_ORDER, LIM_VANALBADA
from tests.support import oracle_problem, small_cfg

ISO, DIF, SPE, PER = BC_ISOTHERMAL, BC_DIFFUSE, BC_SPECULAR, BC_PERIODIC
TW = [0.3, -0.2, 0.1, 0.4, -0.3, 0.2]


def _stencil(P, f):
    """The Laplacian of a cell field by shifted copies: a thermalizing wall's ghost is minus the
    wall cell, a reflecting wall's equals it, a periodic pair wraps."""
    f = np.asarray(f, dtype=np.float64).reshape(P.nz, P.ny, P.nx)
    out = np.zeros_like(f)
    h = (P.dx, P.dy, P.dz)
    for a in range(P.dim):
        ax = 2 - a  # array axis of grid axis a
        lo_bc, hi_bc = P.bc[2 * a], P.bc[2 * a + 1]
        first = np.take(f, [0], axis=ax)
        last = np.take(f, [f.shape[ax] - 1], axis=ax)
        if lo_bc == PER:
            glo, ghi = last, first
        else:
            glo = -first if lo_bc == ISO else first
            ghi = -last if hi_bc == ISO else last
        ext = np.concatenate([glo, f, ghi], axis=ax)
        n = f.shape[ax]
        left = np.take(ext, range(0, n), axis=ax)
        right = np.take(ext, range(2, n + 2), axis=ax)
        out += (left - 2 * f + right) / (h[a] * h[a])
    return out


CASES = [
    (1, (11, 1, 1), [ISO, DIF, PER, PER, PER, PER], ("gl1d", 8)),
    (1, (10, 1, 1), [PER, PER, PER, PER, PER, PER], ("gl1d", 8)),
    (2, (9, 7, 1), [DIF, SPE, ISO, DIF, PER, PER], ("octant", 2, 2)),
    (2, (8, 6, 1), [PER, PER, SPE, DIF, PER, PER], ("octant", 1, 2)),
    (3, (5, 4, 4), [PER, PER, SPE, DIF, ISO, DIF], ("octant", 1, 2)),
    (3, (4, 5, 3), [SPE, DIF, PER, PER, SPE, SPE], ("octant", 1, 2)),
]


@pytest.mark.parametrize("dim,n,bc,quad", CASES)
def test_laplacian_matches_an_independent_stencil(dim, n, bc, quad):
    P = oracle_problem(small_cfg(dim, n, bc, Tw=TW, nb=2, quad=quad))
    f = np.random.default_rng(3).standard_normal(P.ncell)
    assert np.allclose(P.laplacian() @ f, _stencil(P, f).reshape(-1), rtol=1e-13, atol=1e-13 * 4 / P.dx ** 2)


def test_periodic_laplacian_eigenvalues():
    """cos(2 pi j (x + 1/2) / n) is an eigenvector of the periodic second difference with the
    eigenvalue -(4 / h^2) sin^2(pi j / n)."""
    P = oracle_problem(small_cfg(1, (16, 1, 1), [PER] * 6, nb=1, quad=("gl1d", 4)))
    L = P.laplacian()
    x = np.arange(16) + 0.5
    for j in range(0, 9):
        f = np.cos(2 * math.pi * j * x / 16)
        lam = -4.0 / P.dx ** 2 * math.sin(math.pi * j / 16) ** 2
        assert np.allclose(L @ f, lam * f, rtol=0, atol=1e-12 / P.dx ** 2)


# problems with a thermalizing wall (a closed box relaxes to uniform equilibrium, where q -> 0 and
# the loop condition's eps_q has no limit; both schemes converge slowly there, see the GPU tests)
STEADY = [
    CASES[0], CASES[2], CASES[4],
    (2, (8, 6, 1), [ISO, ISO, SPE, SPE, PER, PER], ("octant", 1, 2)),
    (3, (4, 5, 3), [ISO, SPE, PER, PER, SPE, DIF], ("octant", 1, 2)),
]


@pytest.mark.parametrize("limiter", [LIM_FIRST_ORDER, LIM_VANALBADA])
@pytest.mark.parametrize("dim,n,bc,quad", STEADY)
def test_fixed_point_is_the_sequential_one(dim, n, bc, quad, limiter):
    """Converged synthetic and sequential iterations reach the same state, the steady state of
    the step."""
    cfg = small_cfg(dim, n, bc, Tw=TW, nb=3, quad=quad)
    P = oracle_problem(cfg, limiter)
    Q = (np.random.default_rng(4).random((P.nz, P.ny, P.nx)) * 1e17).astype(np.float32)
    e0 = P.equilibrium(np.random.default_rng(5).uniform(-0.2, 0.2, (P.nz, P.ny, P.nx)))
    es, ns, _, _ = P.run_sis(e0, 4000, 1e-13, 1e-13, Q)
    ey, ny_, eT, eq = P.run_synthetic(e0, 4000, 1e-13, 1e-13, Q)
    assert eT < 1e-13 and eq < 1e-13
    assert np.max(np.abs(ey - es)) <= 1e-9 * np.max(np.abs(es))
    assert np.max(np.abs(P.step(ey, Q) - ey)) <= 1e-10 * np.max(np.abs(ey))
    # at the fixed point the macroscopic correction vanishes
    dT = P.synthetic_correction(P.energy_residual(ey, Q))
    assert np.max(np.abs(dT)) <= 1e-9 * max(np.max(np.abs(P.lattice_temperature(ey))), 1e-300)


def test_near_diffusive_convergence_is_fast():
    """Relaxation times far below a cell's flight time, 30 cells between two walls 1 K apart:
    the sequential scheme needs over a thousand iterations, the synthetic one a few tens, to the
    same state."""
    cfg = small_cfg(1, (30, 1, 1), [ISO, ISO, PER, PER, PER, PER], Tw=[0.5, -0.5, 0, 0, 0, 0], nb=1,
                    quad=("gl1d", 16), h=1e-9, tau=1e-12, v=1e3)
    cfg["C"] = np.array([1.66e6])
    P = oracle_problem(cfg, LIM_VANALBADA)
    e0 = P.equilibrium(0.0)
    es, ns, _, _ = P.run_sis(e0, 5000, 1e-10, 1e-10)
    ey, ny_, _, _ = P.run_synthetic(e0, 5000, 1e-10, 1e-10)
    assert ns > 1000 and ny_ < 60
    assert np.max(np.abs(ey - es)) <= 1e-7 * np.max(np.abs(es))


def test_diffusive_film_workload():
    """The benchmark's near-diffusive film (gray silicon, 4 um, 100 cells): the synthetic scheme
    reaches eps_T, eps_q < 1e-6 in a few tens of iterations, the sequential one in over five
    hundred, to the same flux."""
    from paper_2306_14181_gb300 import inputs
    P = oracle_problem(inputs.diffusive_film_1d(), LIM_VANALBADA)
    es, ns, _, _ = P.run_sis(P.equilibrium(0.0), 5000, 1e-6, 1e-6)
    ey, ny_, _, _ = P.run_synthetic(P.equilibrium(0.0), 5000, 1e-6, 1e-6)
    assert ny_ < 40 and ns > 500
    qs = P.moments(es)[2][0].mean()
    qy = P.moments(ey)[2][0].mean()
    assert abs(qy - qs) <= 1e-3 * abs(qs)
