"""Pins of the FP64 oracle against what the paper and the mathematics fix (no GPU).

Each test names the passage of arXiv 2306.14181 it follows.  None of them retypes the
oracle's formulas: they check closed forms, conservation laws, invariances, limits and an
independently built Fourier-mode amplification matrix.
"""
import math

import numpy as np
import pytest

from oracle import quadrature as oq
from oracle.oracle import (BC_DIFFUSE, BC_ISOTHERMAL, BC_PERIODIC, BC_SPECULAR, LIM_FIRST_ORDER, LIM_MINMOD,
                           LIM_VANALBADA)
from paper_2306_14181_gb300 import inputs
from oracle import ttg
from tests.support import oracle_problem, oracle_quadrature, rel_linf, small_cfg

ISO, DIF, SPE, PER = BC_ISOTHERMAL, BC_DIFFUSE, BC_SPECULAR, BC_PERIODIC
FOURPI = 4.0 * math.pi


# ---------------------------------------------------------------------------------------
# P1  quadrature identities (Sec. 3.2, Eq. directiondis)
# ---------------------------------------------------------------------------------------
@pytest.mark.parametrize("rule", [("gl1d", 16), ("gl1d", 8), ("octant", 4, 4), ("octant", 4, 3),
                                  ("octant", 2, 4), ("octant", 2, 1), ("octant", 3, 5), ("octant", 8, 8)])
def test_p1_quadrature_identities(rule):
    s, w, mirror = oracle_quadrature(rule)
    assert abs(w.sum() - FOURPI) <= 1e-14 * FOURPI
    assert np.all(w > 0)
    if rule[0] == "octant":      # the 1-D rule keeps only the projection mu = s_x
        assert np.allclose(np.linalg.norm(s, axis=1), 1.0, atol=1e-15, rtol=0)
    first = (w[:, None] * s).sum(axis=0)
    assert np.max(np.abs(first)) <= 1e-14
    second = np.einsum("d,di,dj->ij", w, s, s)
    expect = np.diag([FOURPI / 3, 0, 0]) if rule[0] == "gl1d" else FOURPI / 3 * np.eye(3)
    assert np.max(np.abs(second - expect)) <= 1e-14
    # number of directions: 8 Ntheta Nphi (octant rule)
    if rule[0] == "octant":
        assert s.shape[0] == 8 * rule[1] * rule[2]
    # mirror table: component a negated, everything else kept
    for a in range(3):
        t = s.copy()
        t[:, a] *= -1
        assert np.array_equal(s[mirror[a]], t)
        assert np.array_equal(w[mirror[a]], w)


def test_p1_paper_theta_rule_is_only_approximate():
    """The literal reading (GL in theta times sin(theta)) meets the identities only to
    quadrature error, which shrinks with Ntheta."""
    errs = []
    for nt in (2, 4, 8):
        s, w, _ = oq.octant_rule(nt, 4, paper_theta_rule=True)
        errs.append(abs(w.sum() - FOURPI) / FOURPI)
    assert errs[0] > 1e-4 and errs[2] < errs[1] < errs[0]


def test_p1_half_range_flux_moment_near_one_quarter():
    """sum_{s_x>0} w s_x / W -> 1/4 (the hemispherical flux factor behind q = C v dT / 4)."""
    for rule in [("gl1d", 16), ("octant", 4, 4)]:
        s, w, _ = oracle_quadrature(rule)
        f = (w * np.clip(s[:, 0], 0, None)).sum() / w.sum()
        assert abs(f - 0.25) < 3e-3


# ---------------------------------------------------------------------------------------
# P2  discrete global energy balance (Eq. disretized_transientBTE summed over cells, bands
#     and directions; the relaxation term conserves energy through Eq. BTE_get_e0)
# ---------------------------------------------------------------------------------------
P2_CASES = [
    (1, (17, 1, 1), [ISO, ISO, PER, PER, PER, PER]),
    (1, (13, 1, 1), [DIF, SPE, PER, PER, PER, PER]),
    (1, (11, 1, 1), [PER, PER, PER, PER, PER, PER]),
    (2, (9, 7, 1), [DIF, SPE, ISO, DIF, PER, PER]),
    (2, (8, 6, 1), [PER, PER, ISO, ISO, PER, PER]),
    (2, (6, 5, 1), [SPE, SPE, SPE, SPE, PER, PER]),
    (3, (6, 5, 4), [PER, PER, SPE, DIF, ISO, DIF]),
    (3, (5, 4, 6), [DIF, ISO, PER, PER, SPE, ISO]),
]


@pytest.mark.parametrize("limiter", [LIM_FIRST_ORDER, LIM_MINMOD, LIM_VANALBADA])
@pytest.mark.parametrize("dim,n,bc", P2_CASES)
def test_p2_energy_balance(dim, n, bc, limiter):
    cfg = small_cfg(dim, n, bc, Tw=[0.3, -0.2, 0.1, 0.4, -0.3, 0.2])
    P = oracle_problem(cfg, limiter)
    e = inputs.random_state(P.shape, 11) * 1e3
    rng = np.random.default_rng(3)
    Q = (rng.random((P.nz, P.ny, P.nx)) * 1e17).astype(np.float32)
    amp = 0.7
    E0, F0 = P.energy(e)
    e1 = P.step(e, Q, amp)
    E1, _ = P.energy(e1)
    V = P.cell_volume
    rhs = P.dt * (V * amp * float(Q.astype(np.float64).sum()) - F0.sum())
    scale = max(abs(E0), abs(E1), P.dt * np.abs(F0).sum())
    assert abs((E1 - E0) - rhs) <= 1e-12 * scale


@pytest.mark.parametrize("bc", [[DIF, SPE, SPE, DIF, SPE, DIF], [PER, PER, DIF, SPE, DIF, SPE]])
def test_p2_adiabatic_walls_conserve_energy(bc):
    """With adiabatic (specular/diffuse) or periodic walls and no source, E is constant over
    many steps and each wall's net heat flow vanishes."""
    cfg = small_cfg(3, (5, 6, 4), bc)
    P = oracle_problem(cfg)
    e = inputs.random_state(P.shape, 5) * 10.0
    E0, _ = P.energy(e)
    for _ in range(20):
        e = P.step(e)
        E, F = P.energy(e)
        tol = 1e-12 * np.abs(E0) / P.dt
        for a in range(3):
            if bc[2 * a] == PER:          # flow leaving one periodic side re-enters the other
                assert abs(F[2 * a] + F[2 * a + 1]) <= tol
            else:
                assert abs(F[2 * a]) <= tol and abs(F[2 * a + 1]) <= tol
    assert abs(E - E0) <= 1e-12 * abs(E0)


# ---------------------------------------------------------------------------------------
# P3  a uniform equilibrium state without source stays uniform (Eq. BTE_get_e0: e = e0)
# ---------------------------------------------------------------------------------------
@pytest.mark.parametrize("dim,n", [(2, (7, 6, 1)), (3, (5, 4, 6))])
@pytest.mark.parametrize("bc,exact", [([PER] * 6, True), ([SPE] * 6, True), ([SPE, PER, PER, SPE, SPE, PER], False),
                                      ([ISO] * 6, False), ([DIF] * 6, False)])
def test_p3_uniform_state_stays_uniform(dim, n, bc, exact):
    if any(b == PER for b in bc):
        # periodic must pair up on an axis
        bc = [bc[0], bc[0], bc[2], bc[2], bc[4], bc[4]]
    dT = 0.37
    cfg = small_cfg(dim, n, bc, Tw=[dT] * 6)
    P = oracle_problem(cfg)
    e = P.equilibrium(dT)
    for _ in range(6):
        e = P.step(e)
        planes = e.reshape(P.nb * P.nd, -1)
        spread = planes.max(axis=1) - planes.min(axis=1)
        if exact:
            assert np.all(spread == 0.0)
        else:
            assert np.all(spread <= 4e-15 * np.abs(planes).max(axis=1))
    TL = P.lattice_temperature(e)
    assert np.max(np.abs(TL - dT)) <= 1e-14 * dT


# ---------------------------------------------------------------------------------------
# P4  ballistic limit between black isothermal walls (Eq. thermal, Eq. getTQ):
#     q = sum_k C_k v_k dT (sum_{s_x>0} w s_x) / W
# ---------------------------------------------------------------------------------------
@pytest.mark.parametrize("limiter", [LIM_FIRST_ORDER, LIM_VANALBADA])
def test_p4_ballistic_flux(limiter):
    cfg = small_cfg(1, (20, 1, 1), [ISO, ISO, PER, PER, PER, PER], Tw=[0.5, -0.5, 0, 0, 0, 0], nb=3,
                    quad=("gl1d", 16), h=1e-9, tau=1e3)
    P = oracle_problem(cfg, limiter)
    s, w = P.s, P.w
    mu_min = np.min(np.abs(s[:, 0]))
    cross = P.nx * P.dx / (np.min(P.v) * mu_min) / P.dt
    e = P.run(P.equilibrium(0.0), int(4 * cross))
    _, _, q = P.moments(e)
    half = float((w * np.clip(s[:, 0], 0, None)).sum()) / P.W
    expect = float(np.sum(P.C * P.v)) * 1.0 * half
    assert rel_linf(q[0].ravel(), np.full(P.nx, expect)) <= 1e-6


# ---------------------------------------------------------------------------------------
# P5  diffusive limit: local Fourier law with kappa = sum C v^2 tau / 3 (Sec. 3.4, k_bulk)
# ---------------------------------------------------------------------------------------
def test_p5_diffusive_limit_fourier_law():
    C = np.array([1.66e6])
    cfg = small_cfg(1, (100, 1, 1), [ISO, ISO, PER, PER, PER, PER], Tw=[0.5, -0.5, 0, 0, 0, 0], nb=1,
                    quad=("gl1d", 16), h=1e-9, tau=1e-12, v=1e3)
    cfg["C"] = C
    P = oracle_problem(cfg, LIM_VANALBADA)
    x = (np.arange(P.nx) + 0.5) / P.nx
    e = P.run(P.equilibrium((0.5 - x)[None, None, :]), 4000)
    _, TL, q = P.moments(e)
    TL = TL.ravel()
    sl = slice(20, 80)
    xs = (np.arange(P.nx) + 0.5) * P.dx
    slope, icpt = np.polyfit(xs[sl], TL[sl], 1)
    resid = TL[sl] - (slope * xs[sl] + icpt)
    assert np.max(np.abs(resid)) <= 1e-3 * np.ptp(TL)        # linear interior profile
    kappa = float(np.sum(P.C * P.v ** 2 * P.tau)) / 3.0
    ratio = np.mean(q[0].ravel()[sl]) / (-kappa * slope)
    assert abs(ratio - 1.0) <= 1e-2


# ---------------------------------------------------------------------------------------
# P6  transient thermal grating (Sec. 4.2): with the first-order face value the fully
#     discrete scheme maps each Fourier mode to itself, e_hat^{n+1} = G(theta) e_hat^n.
# ---------------------------------------------------------------------------------------
@pytest.mark.parametrize("nb,quad", [(1, ("gl1d", 8)), (3, ("gl1d", 6))])
def test_p6_ttg_fourier_mode_exact(nb, quad):
    cfg = small_cfg(1, (24, 1, 1), [PER] * 6, nb=nb, quad=quad, h=1e-9)
    P = oracle_problem(cfg, LIM_FIRST_ORDER)
    theta = 2 * math.pi / P.nx
    j = np.arange(P.nx)
    e0 = P.equilibrium(np.cos(theta * (j + 0.5))[None, None, :])
    nsteps = 150
    e = P.run(e0, nsteps)
    G = ttg.discrete_first_order_matrix(P, theta)
    col = ttg.moment_row(P)
    a = ttg.equilibrium_mode(P) * np.exp(0.5j * theta)
    a = np.linalg.matrix_power(G, nsteps) @ a
    pred_e = np.real(a[:, None] * np.exp(1j * theta * j)[None, :])
    assert rel_linf(e.reshape(P.nb * P.nd, P.nx), pred_e) <= 1e-12
    pred_TL = np.real((col @ a) * np.exp(1j * theta * j))
    assert rel_linf(P.lattice_temperature(e).ravel(), pred_TL) <= 1e-12


def test_p6_limited_scheme_order_of_accuracy():
    """Free streaming of a smooth periodic profile (tau -> infinity).  Forward Euler is first
    order in time, so dt is scaled with dx^2 to expose the spatial reconstruction: the limited
    face values then converge at about second order, the first-order face value at first."""
    def err(N, limiter):
        beta = 0.02 * (64.0 / N)
        cfg = small_cfg(1, (N, 1, 1), [PER] * 6, nb=1, quad=("gl1d", 4), h=64e-9 / N, tau=1e3, v=1e3,
                        beta=beta)
        P = oracle_problem(cfg, limiter)
        L = N * P.dx
        xc = (np.arange(N) + 0.5) * P.dx
        nsteps = int(round(0.25 * L / (P.v[0] * P.dt)))
        t = nsteps * P.dt
        e = P.run(P.equilibrium(np.sin(2 * math.pi * xc / L)[None, None, :]), nsteps)
        ex = np.array([np.sin(2 * math.pi * (xc - P.v[0] * P.s[d, 0] * t) / L) for d in range(P.nd)])
        ex = ex * P.C[0] / P.W
        return np.mean(np.abs(e.reshape(P.nd, N) - ex))
    for limiter, lo, hi in [(LIM_FIRST_ORDER, 0.8, 1.2), (LIM_MINMOD, 1.4, 2.3), (LIM_VANALBADA, 1.7, 2.3)]:
        e1, e2 = err(64, limiter), err(128, limiter)
        order = math.log2(e1 / e2)
        assert lo <= order <= hi, (limiter, order)


# ---------------------------------------------------------------------------------------
# P7  specular wall (Sec. 2.2 (ii)) == the mirror image of the domain across the wall
# ---------------------------------------------------------------------------------------
def test_p7_specular_equals_mirrored_double_domain():
    nx, ny = 6, 5
    Tw = [0.0, 0.3, 0.2, 0.0, 0, 0]
    base = small_cfg(2, (nx, ny, 1), [SPE, ISO, ISO, DIF, PER, PER], Tw=Tw, nb=2)
    P = oracle_problem(base)
    dbl = dict(base)
    dbl["n"] = (2 * nx, ny, 1)
    dbl["bc"] = [ISO, ISO, ISO, DIF, PER, PER]
    dbl["Tw"] = [0.3, 0.3, 0.2, 0.0, 0, 0]
    P2 = oracle_problem(dbl)
    e = inputs.random_state(P.shape, 21)
    Q = (np.random.default_rng(2).random((1, ny, nx)) * 1e17).astype(np.float32)
    mx = P.mirror[0]
    e2 = np.concatenate([e[:, mx][..., ::-1], e], axis=-1)
    Q2 = np.concatenate([Q[..., ::-1], Q], axis=-1)
    one = P.step(e, Q)
    one2 = P2.step(e2, Q2)
    assert np.array_equal(one2[..., nx:], one)            # one step: bitwise
    many = P.run(e, 15, Q)
    many2 = P2.run(e2, 15, Q2)
    assert rel_linf(many2[..., nx:], many) <= 1e-13        # later steps: sums over mirrored order


# ---------------------------------------------------------------------------------------
# P8  translation invariance with periodic walls (Eq. periodic)
# ---------------------------------------------------------------------------------------
def test_p8_periodic_translation():
    cfg = small_cfg(2, (8, 6, 1), [PER] * 6, nb=2)
    P = oracle_problem(cfg)
    e = inputs.random_state(P.shape, 31)
    Q = (np.random.default_rng(4).random((1, 6, 8)) * 1e17).astype(np.float32)
    a = P.run(e, 12, Q)
    b = P.run(np.roll(e, (2, 3), axis=(3, 4)), 12, np.roll(Q, (2, 3), axis=(1, 2)))
    assert np.array_equal(np.roll(b, (-2, -3), axis=(3, 4)), a)


# ---------------------------------------------------------------------------------------
# P9  uniform source from equilibrium with adiabatic walls: T = T_L = sum_n a_n dt Q / sum C
#     (heat split in proportion to C, uniform in angle; Sec. 6.2)
# ---------------------------------------------------------------------------------------
@pytest.mark.parametrize("bc", [[SPE] * 6, [DIF] * 6, [PER] * 6])
def test_p9_uniform_source(bc):
    cfg = small_cfg(3, (4, 5, 3), bc, nb=3)
    P = oracle_problem(cfg)
    Qv = 3e17
    Q = np.full((P.nz, P.ny, P.nx), Qv, dtype=np.float32)
    amps = np.linspace(0.2, 1.0, 25)
    e = P.run(P.equilibrium(0.0), 25, Q, amps)
    T, TL, _ = P.moments(e)
    expect = float(np.sum(amps)) * P.dt * float(np.float32(Qv)) / float(np.sum(P.C))
    assert np.max(np.abs(T - expect)) <= 1e-13 * expect
    assert np.max(np.abs(TL - expect)) <= 1e-13 * expect


# ---------------------------------------------------------------------------------------
# P11 mirror symmetry: a setup symmetric under x -> -x gives a symmetric solution
# ---------------------------------------------------------------------------------------
def test_p11_mirror_symmetry():
    nx, ny = 8, 6
    cfg = small_cfg(2, (nx, ny, 1), [DIF, DIF, ISO, SPE, PER, PER], Tw=[0, 0, 0.4, 0, 0, 0], nb=2)
    P = oracle_problem(cfg)
    Q = inputs.gaussian_spot((nx, ny, 1), cfg["h"], (0.5 * nx * cfg["h"][0], 0.3 * ny * cfg["h"][1]), 4e-9, 1e18)
    e = P.run(P.equilibrium(0.0), 30, Q)
    mirrored = e[:, P.mirror[0]][..., ::-1]
    assert rel_linf(mirrored, e) <= 1e-13


def test_source_and_band_generators_are_seeded():
    a = inputs.bands(1002, 40)
    b = inputs.bands(1002, 40)
    for x, y in zip(a, b):
        assert np.array_equal(x, y)
    C, v, tau = a
    assert abs(C.sum() - 1.66e6) < 1e-6 * 1.66e6
    assert v.min() >= 1e3 and v.max() <= 8e3 and tau.min() >= 1e-12 and tau.max() <= 1e-8


# ---------------------------------------------------------------------------------------
# Isothermal wall heat flow (Eq. thermal): incoming directions carry the wall emission
# C_k T_w / W, outgoing directions leave with the wall cell's own value (first-order wall
# face).  The heat flow is formed here from the state alone and must equal -dE/dt.
# ---------------------------------------------------------------------------------------
@pytest.mark.parametrize("limiter", [LIM_MINMOD, LIM_VANALBADA])
@pytest.mark.parametrize("dim,n", [(1, (9, 1, 1)), (2, (7, 5, 1))])
def test_isothermal_wall_heat_flow(dim, n, limiter):
    Tw = 0.3
    bc = [ISO, SPE, SPE, SPE, SPE, SPE]
    cfg = small_cfg(dim, n, bc, Tw=[Tw, 0, 0, 0, 0, 0])
    P = oracle_problem(cfg, limiter)
    e = inputs.random_state(P.shape, 41) + 2.0
    E0, _ = P.energy(e)
    E1, _ = P.energy(P.step(e))
    S = P.cell_volume / P.dx
    F = 0.0                                   # outward flow through the -x wall
    for k in range(P.nb):
        for d in range(P.nd):
            sn = -P.s[d, 0]
            if sn > 0:
                F += S * P.w[d] * P.v[k] * sn * e[k, d, :, :, 0].sum()
            elif sn < 0:
                F += S * P.w[d] * P.v[k] * sn * (P.C[k] * Tw / P.W) * (P.ny * P.nz)
    assert abs((E1 - E0) + P.dt * F) <= 1e-12 * max(abs(E0), P.dt * abs(F))


# ---------------------------------------------------------------------------------------
# Discrete maximum principle: free streaming of a square wave at CFL 0.4 creates no new
# extrema with the limited (total-variation-diminishing) face values.
# ---------------------------------------------------------------------------------------
@pytest.mark.parametrize("limiter", [LIM_FIRST_ORDER, LIM_MINMOD, LIM_VANALBADA])
def test_limited_streaming_has_no_new_extrema(limiter):
    N = 40
    cfg = small_cfg(1, (N, 1, 1), [PER] * 6, nb=1, quad=("gl1d", 4), h=1e-9, tau=1e3, v=1e3, beta=0.4)
    P = oracle_problem(cfg, limiter)
    x = np.arange(N)
    e0 = P.equilibrium(((x >= 10) & (x < 22)).astype(float)[None, None, :])
    lo, hi = e0.min(), e0.max()
    e = e0
    for _ in range(12):
        e = P.run(e, 10)
        assert e.min() >= lo - 1e-12 * hi and e.max() <= hi * (1 + 1e-12)


@pytest.mark.parametrize("limiter", [LIM_MINMOD, LIM_VANALBADA])
@pytest.mark.parametrize("dim,n,quad", [(2, (20, 20, 1), ("octant", 4, 4)), (3, (12, 12, 12), ("octant", 4, 3))])
def test_multid_time_step_keeps_maximum_principle(dim, n, quad, limiter):
    """The time step of the multi-dimensional workloads (beta = 0.5 over sqrt(dim) times the
    largest speed) keeps the limited unsplit update free of new extrema."""
    cfg = small_cfg(dim, n, [PER] * 6, nb=2, quad=quad, h=1e-9, tau=1e3)
    P = oracle_problem(cfg, limiter)
    z, y, x = np.meshgrid(np.arange(n[2]), np.arange(n[1]), np.arange(n[0]), indexing="ij")
    f = (x >= 3) & (x < 10) & (y >= 4) & (y < 11)
    if dim == 3:
        f &= (z >= 2) & (z < 9)
    e = P.equilibrium(f.astype(float))
    lo, hi = e.min(), e.max()
    for _ in range(6):
        e = P.run(e, 4)
        assert e.min() >= lo - 1e-12 * hi and e.max() <= hi * (1 + 1e-12)


# ---------------------------------------------------------------------------------------
# Sampled step: orc_step_points (the checker of the full-size GPU tests) forms T_L at one
# cell and e^{n+1} at one (k, d, cell) with its own index decoding; it must give exactly the
# elements of the whole-grid step (Eq. disretized_transientBTE with Eq. BTE_get_e0).
# ---------------------------------------------------------------------------------------
def _point_samples(P, n, seed):
    """n random (k, d, cell) triples plus every plane at each corner cell of the domain."""
    rng = np.random.default_rng(seed)
    pts = [np.stack([rng.integers(0, P.nb, n), rng.integers(0, P.nd, n), rng.integers(0, P.ncell, n)], axis=1)]
    zs = (0, P.nz - 1)
    ys = (0, P.ny - 1)
    xs = (0, 1, P.nx - 1)
    for z in zs:
        for y in ys:
            for x in xs:
                i = (z * P.ny + y) * P.nx + x
                kk, dd = np.meshgrid(np.arange(P.nb), np.arange(P.nd), indexing="ij")
                pts.append(np.stack([kk.ravel(), dd.ravel(), np.full(kk.size, i)], axis=1))
    return np.concatenate(pts)


@pytest.mark.parametrize("limiter", [LIM_FIRST_ORDER, LIM_MINMOD, LIM_VANALBADA])
@pytest.mark.parametrize("dim,n,bc", P2_CASES)
def test_step_points_equal_whole_step(dim, n, bc, limiter):
    cfg = small_cfg(dim, n, bc, Tw=[0.3, -0.2, 0.1, 0.4, -0.3, 0.2])
    P = oracle_problem(cfg, limiter)
    e = inputs.random_state(P.shape, 21) * 1e3
    Q = (np.random.default_rng(4).random((P.nz, P.ny, P.nx)) * 1e17).astype(np.float32)
    amp = 0.6
    full = P.step(e, Q, amp).reshape(P.nb * P.nd, P.ncell)
    pts = _point_samples(P, 400, 9)
    got = P.step_points(e, pts, Q, amp)
    want = full[pts[:, 0] * P.nd + pts[:, 1], pts[:, 2]]
    assert np.array_equal(got, want)


# ---------------------------------------------------------------------------------------
# Periodic pair with a temperature difference (Sec. 2.2 (iv)): e(r_B1) = e(r_B2) + C dT/W.
# A uniform gradient G = dT/L along x in an unbounded (periodic) medium has the exact
# solution e_{k,d}(x) = C_k/W (T(x) + tau_k v_k s_x G), T(x) = -G x: the advection of the
# linear profile, -v s_x de/dx = v s_x C G/W, cancels the relaxation (e - e0)/tau =
# C tau v s_x G/W / tau (sum_d w s_x = 0 leaves T_L = T).  Every limiter reproduces a linear
# profile's face values exactly, so the discrete step keeps this state, and its heat flux is
# q_x = sum_k C_k v_k^2 tau_k G sum_d w s_x^2 / W = G sum_k C_k v_k^2 tau_k / 3, the bulk
# conductivity of Sec. 2.1 times the gradient, at any Knudsen number.
# ---------------------------------------------------------------------------------------
def _gradient_state(P, G):
    xc = (np.arange(P.nx) + 0.5) * P.dx
    T = -G * xc
    e = np.empty(P.shape)
    for k in range(P.nb):
        for d in range(P.nd):
            e[k, d] = (P.C[k] / P.W) * (T + P.tau[k] * P.v[k] * P.s[d, 0] * G)[None, None, :]
    return e, T


@pytest.mark.parametrize("limiter", [LIM_FIRST_ORDER, LIM_MINMOD, LIM_VANALBADA])
@pytest.mark.parametrize("dim,n,quad", [(1, (24, 1, 1), ("gl1d", 16)), (2, (20, 5, 1), ("octant", 2, 3)),
                                        (3, (16, 4, 3), ("octant", 2, 2))])
def test_p13_periodic_jump_uniform_gradient_is_stationary(dim, n, quad, limiter):
    dT = 0.8
    cfg = small_cfg(dim, n, [PER] * 6, nb=4, quad=quad, jump=(dT, 0.0, 0.0))
    P = oracle_problem(cfg, limiter)
    G = dT / (P.nx * P.dx)
    e, T = _gradient_state(P, G)
    e1 = P.step(e)
    scale = np.max(np.abs(e))
    assert np.max(np.abs(e1 - e)) <= 1e-12 * scale
    Tm, TL, q = P.moments(e1)
    kappa = float(np.sum(P.C * P.v ** 2 * P.tau) / 3.0)
    assert np.max(np.abs(q[0] - kappa * G)) <= 1e-12 * kappa * G
    assert np.max(np.abs(q[1:])) <= 1e-12 * kappa * G
    assert np.max(np.abs(TL - T[None, None, :])) <= 1e-12 * dT


def test_p13_jump_sign_and_size():
    """A uniform state in a periodic box with a jump: only the cells next to the two walls see
    the ghost offset, +C dT/W at the -x wall for directions entering there, with the sign
    that makes heat flow towards +x."""
    dT = 0.5
    cfg = small_cfg(1, (12, 1, 1), [PER] * 6, nb=2, quad=("gl1d", 8), jump=(dT, 0.0, 0.0))
    P = oracle_problem(cfg, LIM_FIRST_ORDER)
    e = P.equilibrium(0.0)
    e1 = P.step(e)
    k, W = 1, P.W
    for d in range(P.nd):
        nu = P.dt * P.v[k] * P.s[d, 0] / P.dx
        if nu > 0:   # enters through -x: first-order inflow e_ghost = C dT / W at cell 0
            assert e1[k, d, 0, 0, 0] == pytest.approx(nu * P.C[k] * dT / W, rel=1e-12)
            assert e1[k, d, 0, 0, -1] == 0.0
        else:        # enters through +x from the -x side: ghost = -C dT / W
            assert e1[k, d, 0, 0, -1] == pytest.approx(nu * P.C[k] * dT / W, rel=1e-12)
            assert e1[k, d, 0, 0, 0] == 0.0
    # the net flow through the pair moves energy towards +x: the -x wall takes energy in
    E0, F0 = P.energy(e)
    assert F0[0] < 0 and F0[1] > 0


@pytest.mark.parametrize("limiter", [LIM_FIRST_ORDER, LIM_MINMOD, LIM_VANALBADA])
@pytest.mark.parametrize("dim,n,bc,jump", [
    (1, (11, 1, 1), [PER] * 6, (0.4, 0, 0)),
    (2, (9, 7, 1), [PER, PER, DIF, SPE, PER, PER], (-0.3, 0, 0)),
    (3, (6, 5, 4), [PER, PER, PER, PER, ISO, DIF], (0.2, 0.5, 0)),
])
def test_p2_energy_balance_with_periodic_jump(dim, n, bc, jump, limiter):
    """The discrete energy balance holds with the jump's ghost values in the wall face values."""
    cfg = small_cfg(dim, n, bc, Tw=[0.3, -0.2, 0.1, 0.4, -0.3, 0.2], jump=jump)
    P = oracle_problem(cfg, limiter)
    e = inputs.random_state(P.shape, 12) * 1e3
    Q = (np.random.default_rng(3).random((P.nz, P.ny, P.nx)) * 1e17).astype(np.float32)
    E0, F0 = P.energy(e)
    e1 = P.step(e, Q, 0.9)
    E1, _ = P.energy(e1)
    rhs = P.dt * (P.cell_volume * 0.9 * float(Q.astype(np.float64).sum()) - F0.sum())
    scale = max(abs(E0), abs(E1), P.dt * np.abs(F0).sum())
    assert abs((E1 - E0) - rhs) <= 1e-12 * scale
    # the jump shifts every ghost of the pair by the same C dT/W with opposite signs on the two
    # sides, so it moves heat through the pair but adds no energy (sum_d w v s_x = 0)
    assert abs(F0[0] + F0[1]) <= 1e-12 * scale / P.dt


# ---------------------------------------------------------------------------------------
# Residuals of the transient loop condition (Sec. 4.1, Algorithm 2)
# ---------------------------------------------------------------------------------------
def test_residuals_closed_forms():
    """A uniform temperature shift delta between the two states gives eps_T = |delta| / T_max
    exactly; doubling a state of uniform flux (the uniform gradient of P13) gives eps_q = 1/2;
    that gradient state is stationary, so one step gives eps_T = eps_q = 0 to round-off."""
    cfg = small_cfg(2, (8, 6, 1), [PER] * 6, nb=3, quad=("octant", 2, 2))
    P = oracle_problem(cfg)
    eT, _ = P.residuals(P.equilibrium(0.25), P.equilibrium(0.25 + 0.125), 300.0)
    assert eT == pytest.approx(0.125 / 300.375, rel=1e-12)
    dT = 0.6
    cfg = small_cfg(1, (20, 1, 1), [PER] * 6, nb=3, quad=("gl1d", 8), jump=(dT, 0, 0))
    P = oracle_problem(cfg)
    e, _ = _gradient_state(P, dT / (P.nx * P.dx))
    _, eq = P.residuals(e, 2.0 * e, 300.0)
    assert eq == pytest.approx(0.5, rel=1e-12)
    eT, eq = P.residuals(e, P.step(e), 300.0)
    assert eT <= 1e-15 and eq <= 1e-12


# ---------------------------------------------------------------------------------------
# Transient thermal grating (Sec. 4.2): the semi-discrete mode solution exp(M t) that the
# scheme approaches as dx, dt -> 0.  Its two closed-form limits for one gray band:
#  - ballistic (tau -> infinity): each direction's mode advects unchanged, so
#    A(t)/A0 = sum_d w_d cos(q v mu_d t) / W;
#  - diffusive (Kn = v tau / L << 1): A(t)/A0 -> exp(-alpha q^2 t), alpha = v^2 tau / 3.
# The limited scheme of the oracle converges to it under grid refinement.
# ---------------------------------------------------------------------------------------
def _ttg_problem(N, L, v, tau, nd, limiter=LIM_VANALBADA, beta=0.5):
    cfg = small_cfg(1, (N, 1, 1), [PER] * 6, nb=1, quad=("gl1d", nd), h=L / N, tau=tau, v=v, beta=beta)
    return oracle_problem(cfg, limiter)


def test_ttg_semidiscrete_ballistic_limit():
    L, v = 1e-6, 2677.0
    P = _ttg_problem(10, L, v, 1e3, 32)
    q = 2 * math.pi / L
    t = np.linspace(0.0, 3 * L / v, 13)
    A = ttg.semidiscrete_amplitudes(P, q, t)
    exact = np.array([np.sum(P.w * np.cos(q * v * P.s[:, 0] * tt)) / P.W for tt in t])
    assert np.max(np.abs(A - exact)) <= 1e-9


def test_ttg_semidiscrete_diffusive_limit():
    L, v, tau = 1e-6, 2677.0, 39.9e-12 * 1e-3   # Kn = v tau / L ~ 1e-4
    P = _ttg_problem(10, L, v, tau, 32)
    q = 2 * math.pi / L
    alpha = v * v * tau / 3.0
    t = np.array([0.5, 1.0, 2.0]) / (alpha * q * q)
    A = ttg.semidiscrete_amplitudes(P, q, t)
    assert np.max(np.abs(A - np.exp(-alpha * q * q * t))) <= 1e-4


def test_ttg_limited_scheme_converges_to_the_mode_solution():
    """xi = 2 pi Kn = 1 gray grating: the van Albada scheme's amplitude error against exp(M t)
    at t* = t/tau = 4 falls with refinement (dt tied to dx by the CFL rule)."""
    v, tau = 2677.0, 39.9e-12
    L = 2 * math.pi * v * tau / 1.0
    errs = []
    for N in (50, 100, 200):
        P = _ttg_problem(N, L, v, tau, 16)
        x = (np.arange(N) + 0.5) * P.dx
        nsteps = int(round(4 * tau / P.dt))
        e = P.run(P.equilibrium(np.cos(2 * math.pi * x / L)[None, None, :]), nsteps)
        T = P.moments(e)[0].ravel()
        A = 2.0 / N * float(np.sum(T * np.cos(2 * math.pi * x / L)))
        errs.append(abs(A - ttg.semidiscrete_amplitudes(P, 2 * math.pi / L, [nsteps * P.dt])[0]))
    assert errs[1] < 0.6 * errs[0] and errs[2] < 0.6 * errs[1], errs
