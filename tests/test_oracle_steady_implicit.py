"""Pins of the oracle's steady implicit DOM, sequential iterative scheme (Sec. 3.3-3.5), no GPU.

One iteration solves, plane by plane, the first-order upwind system of Eq. (disretized_BTE) in
delta form for the increment, with the transient step's own right-hand side.  The pins check it
against a dense linear solve of that system assembled from its definition, a stationary state
that must stay put, the steady equation at convergence (the explicit step no longer moves the
state), the ballistic flux between two walls in closed form, and the diffusive limit.
"""

import numpy as np
import pytest

from oracle.oracle import BC_DIFFUSE, BC_ISOTHERMAL, BC_PERIODIC, BC_SPECULAR, LIM_FIRST_ORDER, LIM_MINMOD, LIM_VANALBADA
from tests.support import oracle_problem, rel_linf, small_cfg

ISO, DIF, SPE, PER = BC_ISOTHERMAL, BC_DIFFUSE, BC_SPECULAR, BC_PERIODIC
TW = [0.3, -0.2, 0.1, 0.4, -0.3, 0.2]


def _dense_increment(P, e, Q):
    """De of one iteration from the definition: for each (k, d) the matrix with 1/tau_k +
    sum_a v_k |s_a| / h_a on the diagonal and -v_k |s_a| / h_a at each cell's upwind neighbour
    along a inside the domain, solved against R = (step(e) - e) / dt by a dense solver."""
    R = (P.step(e, Q) - e) / P.dt
    nx, ny, nz = P.nx, P.ny, P.nz
    h = (P.dx, P.dy, P.dz)
    n = (nx, ny, nz)
    De = np.zeros(P.shape)
    idx = np.arange(P.ncell).reshape(nz, ny, nx)
    for k in range(P.nb):
        for d in range(P.nd):
            M = np.zeros((P.ncell, P.ncell))
            M[np.arange(P.ncell), np.arange(P.ncell)] = 1.0 / P.tau[k]
            for a in range(P.dim):
                sa = P.s[d, a]
                c = P.v[k] * abs(sa) / h[a]
                M[np.arange(P.ncell), np.arange(P.ncell)] += c
                if sa == 0.0:
                    continue
                step = 1 if sa > 0 else -1
                for z in range(nz):
                    for y in range(ny):
                        for x in range(nx):
                            cc = [x, y, z]
                            up = list(cc)
                            up[a] -= step
                            if 0 <= up[a] < n[a]:
                                M[idx[z, y, x], idx[up[2], up[1], up[0]]] -= c
            De[k, d] = np.linalg.solve(M, R[k, d].reshape(-1)).reshape(nz, ny, nx)
    return De


CASES = [
    (1, (9, 1, 1), [ISO, DIF, PER, PER, PER, PER], ("gl1d", 8)),
    (1, (8, 1, 1), [PER, PER, PER, PER, PER, PER], ("gl1d", 6)),
    (2, (6, 5, 1), [DIF, SPE, ISO, DIF, PER, PER], ("octant", 2, 2)),
    (2, (5, 4, 1), [PER, PER, SPE, ISO, PER, PER], ("octant", 1, 2)),
    (3, (4, 3, 3), [PER, PER, SPE, DIF, ISO, DIF], ("octant", 1, 2)),
]


@pytest.mark.parametrize("limiter", [LIM_FIRST_ORDER, LIM_VANALBADA])
@pytest.mark.parametrize("dim,n,bc,quad", CASES)
def test_iteration_solves_the_upwind_system(dim, n, bc, quad, limiter):
    cfg = small_cfg(dim, n, bc, Tw=TW, nb=3, quad=quad)
    P = oracle_problem(cfg, limiter)
    rng = np.random.default_rng(12)
    e = P.equilibrium(rng.uniform(-0.5, 0.5, (P.nz, P.ny, P.nx))) * (1 + 0.3 * rng.standard_normal(P.shape))
    Q = (rng.random((P.nz, P.ny, P.nx)) * 1e17).astype(np.float32)
    De = P.sis_iteration(e, Q) - e
    expect = _dense_increment(P, e, Q)
    assert np.max(np.abs(De - expect)) <= 1e-9 * np.max(np.abs(expect))


@pytest.mark.parametrize("limiter", [LIM_FIRST_ORDER, LIM_VANALBADA])
def test_uniform_gradient_is_a_fixed_point(limiter):
    """The periodic pair with a temperature difference: the uniform-gradient state is stationary
    (Sec. 2.2 (iv)), so its right-hand side vanishes and an iteration leaves it unchanged."""
    dT = 0.8
    cfg = small_cfg(2, (12, 4, 1), [PER] * 6, nb=3, quad=("octant", 2, 2), jump=(dT, 0.0, 0.0))
    P = oracle_problem(cfg, limiter)
    G = dT / (P.nx * P.dx)
    xc = (np.arange(P.nx) + 0.5) * P.dx
    e = np.empty(P.shape)
    for k in range(P.nb):
        for d in range(P.nd):
            e[k, d] = (P.C[k] / P.W) * (-G * xc + P.tau[k] * P.v[k] * P.s[d, 0] * G)[None, None, :]
    e1 = P.sis_iteration(e)
    assert np.max(np.abs(e1 - e)) <= 1e-12 * np.max(np.abs(e))


@pytest.mark.parametrize("limiter", [LIM_FIRST_ORDER, LIM_MINMOD, LIM_VANALBADA])
@pytest.mark.parametrize("dim,n,bc,quad", [CASES[0], CASES[2], CASES[4]])
def test_converged_state_is_steady_for_the_step(dim, n, bc, quad, limiter):
    """At convergence of the residual loop (Sec. 3.5) the state solves the steady equation: the
    transient step (Eq. disretized_transientBTE) no longer moves it."""
    cfg = small_cfg(dim, n, bc, Tw=TW, nb=3, quad=quad)
    P = oracle_problem(cfg, limiter)
    Q = (np.random.default_rng(2).random((P.nz, P.ny, P.nx)) * 1e17).astype(np.float32)
    e, it, eT, eq = P.run_sis(P.equilibrium(0.0), 3000, 1e-13, 1e-13, Q)
    assert eT < 1e-13 and eq < 1e-13
    moved = P.step(e, Q) - e
    assert np.max(np.abs(moved)) <= 1e-10 * np.max(np.abs(e))


@pytest.mark.parametrize("limiter", [LIM_FIRST_ORDER, LIM_VANALBADA])
def test_ballistic_film_flux(limiter):
    """Two thermalizing walls 1 K apart, relaxation times far longer than the flight time: the
    steady flux is sum_k C_k v_k dT (sum_{s_x>0} w s_x) / W everywhere (the ballistic limit)."""
    cfg = small_cfg(1, (20, 1, 1), [ISO, ISO, PER, PER, PER, PER], Tw=[0.5, -0.5, 0, 0, 0, 0], nb=3,
                    quad=("gl1d", 16), h=1e-9, tau=1e3)
    P = oracle_problem(cfg, limiter)
    e, it, eT, eq = P.run_sis(P.equilibrium(0.0), 200, 1e-13, 1e-13)
    assert it < 50  # ballistic: each direction is settled by its own sweep
    _, _, q = P.moments(e)
    half = float((P.w * np.clip(P.s[:, 0], 0, None)).sum()) / P.W
    expect = float(np.sum(P.C * P.v)) * 1.0 * half
    assert rel_linf(q[0].ravel(), np.full(P.nx, expect)) <= 1e-9


def test_diffusive_limit_fourier_law():
    """Relaxation times far below the flight time across a cell: a linear interior profile whose
    flux obeys Fourier's law with kappa = sum C v^2 tau / 3 (Sec. 3.5, k_bulk)."""
    cfg = small_cfg(1, (30, 1, 1), [ISO, ISO, PER, PER, PER, PER], Tw=[0.5, -0.5, 0, 0, 0, 0], nb=1,
                    quad=("gl1d", 16), h=1e-9, tau=1e-12, v=1e3)
    cfg["C"] = np.array([1.66e6])
    P = oracle_problem(cfg, LIM_VANALBADA)
    x = (np.arange(P.nx) + 0.5) / P.nx
    e, it, eT, eq = P.run_sis(P.equilibrium((0.5 - x)[None, None, :]), 5000, 1e-10, 1e-10)
    assert eT < 1e-10
    _, TL, q = P.moments(e)
    TL = TL.ravel()
    sl = slice(6, 24)
    xs = (np.arange(P.nx) + 0.5) * P.dx
    slope, icpt = np.polyfit(xs[sl], TL[sl], 1)
    assert np.max(np.abs(TL[sl] - (slope * xs[sl] + icpt))) <= 1e-3 * np.ptp(TL)
    kappa = float(np.sum(P.C * P.v ** 2 * P.tau)) / 3.0
    assert abs(np.mean(q[0].ravel()[sl]) / (-kappa * slope) - 1.0) <= 1e-2


@pytest.mark.parametrize("dim,n,bc,quad", [CASES[0], CASES[2], CASES[4]])
def test_iteration_with_a_given_lattice_temperature(dim, n, bc, quad):
    """The iteration that relaxes towards a given T_L (the synthetic scheme's corrected one):
    with T_L of the state it is the plain iteration bit for bit; raising T_L by dT in one cell
    adds to that cell's right-hand side C_k dT / (W tau_k) in every direction, so the increment
    changes by the dense upwind solve of that source."""
    cfg = small_cfg(dim, n, bc, Tw=TW, nb=3, quad=quad)
    P = oracle_problem(cfg, LIM_VANALBADA)
    rng = np.random.default_rng(21)
    e = P.equilibrium(rng.uniform(-0.5, 0.5, (P.nz, P.ny, P.nx))) * (1 + 0.3 * rng.standard_normal(P.shape))
    TL = P.lattice_temperature(e)
    base = P.sis_iteration_tl(e, TL)
    assert np.array_equal(base, P.sis_iteration(e))
    cell = (P.nz // 2, P.ny // 2, P.nx // 2)
    dT = 0.25
    TL2 = TL.copy()
    TL2[cell] += dT
    change = P.sis_iteration_tl(e, TL2) - base
    # the same change from the dense upwind solve of a source C_k dT / (W tau_k) in that cell
    h = (P.dx, P.dy, P.dz)
    nn = (P.nx, P.ny, P.nz)
    idx = np.arange(P.ncell).reshape(P.nz, P.ny, P.nx)
    for k in range(P.nb):
        for d in range(P.nd):
            M = np.zeros((P.ncell, P.ncell))
            M[np.arange(P.ncell), np.arange(P.ncell)] = 1.0 / P.tau[k]
            for a in range(P.dim):
                sa = P.s[d, a]
                c = P.v[k] * abs(sa) / h[a]
                M[np.arange(P.ncell), np.arange(P.ncell)] += c
                if sa == 0.0:
                    continue
                step = 1 if sa > 0 else -1
                for z in range(P.nz):
                    for y in range(P.ny):
                        for x in range(P.nx):
                            up = [x, y, z]
                            up[a] -= step
                            if 0 <= up[a] < nn[a]:
                                M[idx[z, y, x], idx[up[2], up[1], up[0]]] -= c
            rhs = np.zeros(P.ncell)
            rhs[idx[cell]] = P.C[k] * dT / (P.W * P.tau[k])
            expect = np.linalg.solve(M, rhs).reshape(P.nz, P.ny, P.nx)
            assert np.max(np.abs(change[k, d] - expect)) <= 1e-9 * np.max(np.abs(expect)) + 1e-12 * np.max(np.abs(base))
