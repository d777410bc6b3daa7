"""Pins of the oracle's interface between two materials (Sec. 2.2 (v), diffuse mismatch), no GPU.

The interface couples wall wa of material A with wall wb of material B.  The pins check what the
boundary condition fixes without restating it: with no transmission each side is a plain diffuse
wall; a uniform equilibrium stays put exactly when the transmissions satisfy detailed balance
(and moves when they are swapped); with equal group speeds the energy that leaves one side
arrives in the other; and one step from a single outgoing pulse puts the transmitted share,
computed by hand, into exactly one cell of the other side.
"""
import numpy as np
import pytest

from oracle.oracle import (BC_DIFFUSE, BC_ISOTHERMAL, BC_PERIODIC, BC_SPECULAR, LIM_FIRST_ORDER, LIM_MINMOD,
                           LIM_VANALBADA, interface_energy, interface_run, interface_step)
from tests.support import oracle_problem, small_cfg

ISO, DIF, SPE, PER = BC_ISOTHERMAL, BC_DIFFUSE, BC_SPECULAR, BC_PERIODIC


def pair_cfgs(dim, nA, nB, bcA, bcB, quad=None, same_v=False, TwA=(0,) * 6, TwB=(0,) * 6):
    """Material A (band table of seed 7) and material B (seed 11), one common time step."""
    cA = small_cfg(dim, nA, bcA, Tw=TwA, nb=3, quad=quad)
    cB = small_cfg(dim, nB, bcB, Tw=TwB, nb=3, quad=quad, seed=11, v=cA["v"] if same_v else None)
    dt = min(cA["dt"], cB["dt"])
    cA["dt"] = cB["dt"] = dt
    return cA, cB


# (dim, nA, nB, wa, wb, other walls of A, other walls of B): the interface walls are set to DIF
GEOMS = [
    (1, (9, 1, 1), (6, 1, 1), 1, 0, [ISO, None, PER, PER, PER, PER], [None, SPE, PER, PER, PER, PER]),
    (2, (7, 5, 1), (4, 5, 1), 1, 0, [SPE, None, PER, PER, PER, PER], [None, DIF, SPE, SPE, PER, PER]),
    (2, (6, 4, 1), (6, 5, 1), 3, 2, [PER, PER, SPE, None, PER, PER], [PER, PER, None, ISO, PER, PER]),
    (3, (4, 3, 5), (4, 3, 3), 4, 5, [SPE, SPE, PER, PER, None, DIF], [PER, PER, SPE, SPE, DIF, None]),
    (3, (3, 4, 4), (5, 4, 4), 0, 1, [None, SPE, PER, PER, SPE, SPE], [SPE, None, SPE, DIF, PER, PER]),
]


def _walls(bc, w):
    bc = list(bc)
    bc[w] = DIF
    return bc


def _problems(geom, limiter, same_v=False, adiabatic=False, Tw=(0.2, -0.1)):
    dim, nA, nB, wa, wb, bcA, bcB = geom
    bcA, bcB = _walls(bcA, wa), _walls(bcB, wb)
    if adiabatic:  # every other wall reflecting or periodic, so that no heat leaves the pair
        bcA = [SPE if (b in (ISO, DIF) and j != wa) else b for j, b in enumerate(bcA)]
        bcB = [SPE if (b in (ISO, DIF) and j != wb) else b for j, b in enumerate(bcB)]
    cA, cB = pair_cfgs(dim, nA, nB, bcA, bcB, same_v=same_v, TwA=(Tw[0],) * 6, TwB=(Tw[1],) * 6)
    return cA, cB, oracle_problem(cA, limiter), oracle_problem(cB, limiter)


def _random_states(A, B, seed):
    rng = np.random.default_rng(seed)
    eA = A.equilibrium(rng.uniform(-1, 1, (A.nz, A.ny, A.nx))) * (1 + 0.3 * rng.standard_normal(A.shape))
    eB = B.equilibrium(rng.uniform(-1, 1, (B.nz, B.ny, B.nx))) * (1 + 0.3 * rng.standard_normal(B.shape))
    return eA, eB


@pytest.mark.parametrize("geom", GEOMS)
@pytest.mark.parametrize("limiter", [LIM_FIRST_ORDER, LIM_VANALBADA])
def test_no_transmission_is_two_diffuse_walls(geom, limiter):
    """beta = 0 both ways: each side reflects everything diffusely, i.e. it is the plain diffuse
    wall of Eq. (diff_bound), bit for bit."""
    cA, cB, A, B = _problems(geom, limiter)
    eA, eB = _random_states(A, B, 3)
    oA, oB = interface_step(A, eA, geom[3], B, eB, geom[4], 0.0, 0.0)
    assert np.array_equal(oA, A.step(eA))
    assert np.array_equal(oB, B.step(eB))


@pytest.mark.parametrize("geom", GEOMS)
def test_equilibrium_kept_under_detailed_balance(geom):
    """A common uniform temperature is stationary when beta_BA C_B = beta_AB C_A band by band
    (the energy A sends into B equals what B sends back); with the two transmissions swapped the
    same state leaves equilibrium."""
    # isothermal walls at the common temperature, so that only the interface can disturb it
    T = 0.7
    cA, cB, A, B = _problems(geom, LIM_VANALBADA, Tw=(T, T))
    assert np.any(np.abs(A.C - B.C) > 0.1 * A.C)
    bAB = B.C / (A.C + B.C)
    bBA = A.C / (A.C + B.C)
    eA, eB = A.equilibrium(T), B.equilibrium(T)
    fA, fB = interface_run(A, eA, geom[3], B, eB, geom[4], bAB, bBA, 5)
    assert np.max(np.abs(fA - eA)) <= 1e-13 * np.max(np.abs(eA))
    assert np.max(np.abs(fB - eB)) <= 1e-13 * np.max(np.abs(eB))
    gA, gB = interface_run(A, eA, geom[3], B, eB, geom[4], bBA, bAB, 5)
    assert max(np.max(np.abs(gA - eA)) / np.max(np.abs(eA)), np.max(np.abs(gB - eB)) / np.max(np.abs(eB))) > 1e-4


@pytest.mark.parametrize("geom", GEOMS)
@pytest.mark.parametrize("limiter", [LIM_FIRST_ORDER, LIM_MINMOD, LIM_VANALBADA])
def test_energy_crosses_the_interface_unchanged(geom, limiter):
    """Equal group speeds on both sides and no other heat path: E_A + E_B is constant, each
    side's energy changes by dt times the heat through the interface, and the two interface
    flows cancel (Eq. (disretized_transientBTE) summed over both materials)."""
    cA, cB, A, B = _problems(geom, limiter, same_v=True, adiabatic=True)
    eA, eB = _random_states(A, B, 5)
    bAB = np.array([0.2, 0.55, 0.9])
    bBA = np.array([0.7, 0.35, 0.1])
    E0A, F0A, E0B, F0B = interface_energy(A, eA, geom[3], B, eB, geom[4], bAB, bBA)
    scale = abs(F0A[geom[3]]) + abs(F0B[geom[4]])
    assert scale > 0
    assert abs(F0A[geom[3]] + F0B[geom[4]]) <= 1e-12 * scale
    oA, oB = interface_step(A, eA, geom[3], B, eB, geom[4], bAB, bBA)
    E1A, _, E1B, _ = interface_energy(A, oA, geom[3], B, oB, geom[4], bAB, bBA)
    Esc = abs(E0A) + abs(E0B)
    assert abs((E1A - E0A) + A.dt * F0A[geom[3]]) <= 1e-12 * Esc
    assert abs((E1B - E0B) + B.dt * F0B[geom[4]]) <= 1e-12 * Esc
    fA, fB = interface_run(A, oA, geom[3], B, oB, geom[4], bAB, bBA, 9)
    E2A, _, E2B, _ = interface_energy(A, fA, geom[3], B, fB, geom[4], bAB, bBA)
    assert abs((E2A + E2B) - (E0A + E0B)) <= 1e-12 * Esc


@pytest.mark.parametrize("geom", GEOMS)
def test_one_pulse_transmits_its_share_into_one_cell(geom):
    """First order, both states zero but one outgoing direction d0 of band k0 at one interface
    cell of A, value delta.  After one step the only change in B is at the facing cell, in band
    k0 and the directions entering B: dt v_B |s_a| / h_a times beta_AB[k0] times A's diffuse
    value w_d0 |s_a,d0| delta / sum_{incoming} w |s_a| (Eq. (diff_bound)'s discrete normaliser)."""
    dim, nA, nB, wa, wb, _, _ = geom
    cA, cB, A, B = _problems(geom, LIM_FIRST_ORDER, Tw=(0.0, 0.0))
    ax = wa >> 1
    s = A.s
    out_sign = 1.0 if wa & 1 else -1.0  # outward normal of A's interface wall along ax
    rng = np.random.default_rng(17)
    k0 = 1
    d0 = int(rng.choice(np.flatnonzero(out_sign * s[:, ax] > 0)))
    cell = [int(rng.integers(0, n)) for n in (A.nx, A.ny, A.nz)]
    cell[ax] = (A.nx, A.ny, A.nz)[ax] - 1 if wa & 1 else 0
    delta = 0.37
    eA = np.zeros(A.shape)
    eB = np.zeros(B.shape)
    eA[k0, d0, cell[2], cell[1], cell[0]] = delta
    bAB = np.array([0.15, 0.6, 0.85])
    bBA = np.array([0.5, 0.25, 0.05])
    _, oB = interface_step(A, eA, wa, B, eB, wb, bAB, bBA)
    den = float(np.sum(A.w * np.abs(s[:, ax]) * (out_sign * s[:, ax] < 0)))
    SA = A.w[d0] * abs(s[d0, ax]) * delta / den
    h = (B.dx, B.dy, B.dz)[ax]
    cellB = list(cell)
    cellB[ax] = (B.nx, B.ny, B.nz)[ax] - 1 if wb & 1 else 0
    expect = np.zeros(B.shape)
    entering = np.flatnonzero(out_sign * s[:, ax] > 0)  # B's incoming directions move like A's outgoing ones
    for d in entering:
        expect[k0, d, cellB[2], cellB[1], cellB[0]] = B.dt * B.v[k0] * abs(s[d, ax]) / h * bAB[k0] * SA
    assert np.max(np.abs(oB - expect)) <= 1e-14 * np.max(np.abs(expect))
    assert np.count_nonzero(oB) == len(entering)


def test_walls_that_do_not_face_are_refused():
    cA, cB, A, B = _problems(GEOMS[1], LIM_VANALBADA)
    eA, eB = _random_states(A, B, 1)
    with pytest.raises(ValueError):
        interface_step(A, eA, 1, B, eB, 1, 0.5, 0.5)        # same side
    with pytest.raises(ValueError):
        interface_step(A, eA, 1, B, eB, 2, 0.5, 0.5)        # other axis
    cC, _ = pair_cfgs(2, (7, 6, 1), (4, 5, 1), _walls(GEOMS[1][5], 1), _walls(GEOMS[1][6], 0))
    C = oracle_problem(cC, LIM_VANALBADA)
    with pytest.raises(ValueError):                          # 6 rows against 5
        interface_step(C, C.equilibrium(0.0), 1, B, eB, 0, 0.5, 0.5)


def test_interface_workload_transmissions():
    """The benchmark's two-material workload: transmissions in [0, 1] that sum to one band by
    band and satisfy detailed balance, facing walls on one axis, one time step for both sides."""
    from paper_2306_14181_gb300 import inputs
    cfg = inputs.interface_2d(nx=128, ny=24, nb=4, ntheta=2, nphi=2)
    A, B = cfg["A"], cfg["B"]
    bab, bba = cfg["beta_ab"], cfg["beta_ba"]
    assert np.all((bab > 0) & (bab < 1)) and np.allclose(bab + bba, 1.0, rtol=0, atol=1e-15)
    assert np.allclose(bba * B["C"], bab * A["C"], rtol=1e-15, atol=0)
    assert A["dt"] == B["dt"] and A["n"][1:] == B["n"][1:]
    assert A["bc"][cfg["wall_a"]] == BC_DIFFUSE and B["bc"][cfg["wall_b"]] == BC_DIFFUSE
    assert (cfg["wall_a"] >> 1) == (cfg["wall_b"] >> 1) and cfg["wall_a"] != cfg["wall_b"]


@pytest.mark.parametrize("t", [0.25, 0.5, 0.8])
def test_ballistic_flux_through_the_interface(t):
    """Ballistic limit (relaxation times far beyond the flight time), one gray material on both
    sides, thermalizing outer walls 1 K apart and an interface that transmits a share t both ways:
    every emitter is diffuse, so the steady flux is the ballistic flux between the two walls times
    t (the series law of diffuse transmitters: 1 / tau_eff = 1 + 1 + (1 / t - 1) - 1)."""
    cA = small_cfg(1, (10, 1, 1), [ISO, DIF, PER, PER, PER, PER], Tw=[0.5, 0, 0, 0, 0, 0], nb=1, quad=("gl1d", 16),
                   h=1e-9, tau=1e3, v=1e3)
    cB = small_cfg(1, (10, 1, 1), [DIF, ISO, PER, PER, PER, PER], Tw=[0, -0.5, 0, 0, 0, 0], nb=1, quad=("gl1d", 16),
                   h=1e-9, tau=1e3, v=1e3)
    for c in (cA, cB):
        c["C"] = np.array([1.66e6])
    A, B = oracle_problem(cA, LIM_VANALBADA), oracle_problem(cB, LIM_VANALBADA)
    eA, eB = interface_run(A, A.equilibrium(0.0), 1, B, B.equilibrium(0.0), 0, t, t, 3000)
    half = float((A.w * np.clip(A.s[:, 0], 0, None)).sum()) / A.W
    expect = t * 1.66e6 * 1e3 * 1.0 * half
    for P, e in ((A, eA), (B, eB)):
        q = P.moments(e)[2][0].ravel()
        assert np.max(np.abs(q - expect)) <= 1e-10 * expect
