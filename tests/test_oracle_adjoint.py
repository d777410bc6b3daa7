"""Pins of the oracle's discrete adjoint (the exact transpose of the step; the paper has no
adjoint, so each pin ties it to the forward step rather than to a printed value).

- dot test: the reverse-mode step J^T and an independently coded forward-mode step J agree,
  <lam, J de> = <J^T lam, de> to round-off, on every wall type, limiter and dimension;
- the forward-mode step equals central differences of the forward step;
- the run adjoint's gradients with respect to the per-cell source Q and log tau_k equal
  central differences of J = sum_i p_i T_L,i (exactly for the first-order scheme, which is
  affine in Q; to 1e-4 for the limited scheme).
"""
import numpy as np
import pytest

from paper_2306_14181_gb300 import inputs
from tests.support import oracle_problem, small_cfg

ISO, DIF, SPE, PER = 0, 1, 2, 3
TW = [0.3, -0.2, 0.1, 0.4, -0.3, 0.2]

GRIDS = [
    (1, (12, 1, 1), [ISO, DIF, PER, PER, PER, PER]),
    (1, (10, 1, 1), [SPE, ISO, PER, PER, PER, PER]),
    (2, (7, 6, 1), [DIF, SPE, ISO, DIF, PER, PER]),
    (2, (6, 5, 1), [PER, PER, SPE, DIF, PER, PER]),
    (3, (5, 4, 4), [SPE, SPE, PER, PER, DIF, ISO]),
    (3, (4, 5, 3), [DIF, ISO, SPE, SPE, PER, PER]),
]


@pytest.mark.parametrize("limiter", [0, 1, 2])
@pytest.mark.parametrize("dim,n,bc", GRIDS)
def test_adjoint_step_dot_test(dim, n, bc, limiter):
    cfg = small_cfg(dim, n, bc, Tw=TW, nb=2)
    P = oracle_problem(cfg, limiter)
    e = inputs.random_state(P.shape, 3)
    de = inputs.random_state(P.shape, 4, smooth=False)
    lam = inputs.random_state(P.shape, 5, smooth=False)
    a = float(np.vdot(lam, P.step_tangent(e, de)))
    b = float(np.vdot(P.adjoint_step(e, lam), de))
    assert abs(a - b) <= 1e-13 * max(abs(a), np.linalg.norm(lam) * np.linalg.norm(de))


@pytest.mark.parametrize("limiter", [0, 1, 2])
@pytest.mark.parametrize("dim,n,bc", GRIDS[::2])
def test_tangent_step_matches_central_differences(dim, n, bc, limiter):
    """The forward-mode step against the forward step itself (so the dot test pins the
    transpose of the actual step, not of a shared mistake)."""
    cfg = small_cfg(dim, n, bc, Tw=TW, nb=2)
    P = oracle_problem(cfg, limiter)
    e = inputs.random_state(P.shape, 13)
    de = inputs.random_state(P.shape, 14, smooth=False)
    t = P.step_tangent(e, de)
    # first order: the step is affine, any h; van Albada: smooth away from ab = 0, small h
    h = 1e-2 if limiter == 0 else 1e-5
    fd = (P.step(e + h * de) - P.step(e - h * de)) / (2 * h)
    tol = 1e-9 if limiter == 0 else 1e-5
    assert np.max(np.abs(fd - t)) <= tol * np.max(np.abs(fd))


def _probe(P):
    """J = mean T_L over a box in the upper part of the domain."""
    p = np.zeros((P.nz, P.ny, P.nx))
    z0 = P.nz // 2 if P.nz > 1 else 0
    y0 = P.ny // 2 if P.ny > 1 else 0
    p[z0:, y0:, P.nx // 2:] = 1.0
    return p / p.sum()


def _J(P, e0, nsteps, probe, Q, amps):
    return float(np.sum(probe * P.lattice_temperature(P.run(e0, nsteps, Q, amps))))


@pytest.mark.parametrize("limiter,tol", [(0, 1e-9), (2, 1e-4)])
@pytest.mark.parametrize("dim,n,bc", [GRIDS[0], GRIDS[2], GRIDS[4]])
def test_run_adjoint_matches_finite_differences(dim, n, bc, limiter, tol):
    cfg = small_cfg(dim, n, bc, Tw=TW, nb=2)
    P = oracle_problem(cfg, limiter)
    nsteps = 12
    rng = np.random.default_rng(8)
    Q = (rng.random((P.nz, P.ny, P.nx)) * 2e17).astype(np.float32)
    amps = np.linspace(1.0, 0.3, nsteps)
    e0 = P.equilibrium(rng.random((P.nz, P.ny, P.nx)) - 0.5)
    probe = _probe(P)
    J, gQ, gt = P.adjoint(e0, nsteps, probe, Q, amps)
    assert J == pytest.approx(_J(P, e0, nsteps, probe, Q, amps), rel=1e-14, abs=1e-300)
    # source: additive h max Q at three cells (the realised float32 perturbation is used)
    hq = 1e-4 * float(Q.max())
    for ci in rng.choice(P.ncell, 3, replace=False):
        Qp, Qm = Q.copy().reshape(-1), Q.copy().reshape(-1)
        Qp[ci] = np.float32(Q.reshape(-1)[ci] + hq)
        Qm[ci] = np.float32(Q.reshape(-1)[ci] - hq)
        fd = (_J(P, e0, nsteps, probe, Qp.reshape(Q.shape), amps) - _J(P, e0, nsteps, probe, Qm.reshape(Q.shape), amps))
        fd /= float(Qp[ci]) - float(Qm[ci])
        assert abs(fd - gQ.reshape(-1)[ci]) <= tol * np.max(np.abs(gQ)) + 1e-300
    # log tau_k: additive h in log tau
    ht = 1e-5 if limiter == 0 else 1e-4
    for k in range(P.nb):
        Js = []
        for sgn in (1, -1):
            tau = np.array(cfg["tau"], float)
            tau[k] *= np.exp(sgn * ht)
            Pk = oracle_problem(dict(cfg, tau=tau), limiter)
            Js.append(_J(Pk, e0, nsteps, probe, Q, amps))
        fd = (Js[0] - Js[1]) / (2 * ht)
        assert abs(fd - gt[k]) <= max(tol, 1e-7) * np.max(np.abs(gt))


def test_uniform_source_gradient_is_the_summed_gradient():
    """A uniform change of Q moves J by the sum of dJ/dQ_i (J is affine in Q): periodic box,
    first-order scheme, one step from a random state, mean T_L probe."""
    cfg = small_cfg(2, (6, 5, 1), [PER] * 6, nb=3)
    P = oracle_problem(cfg, 0)
    e0 = inputs.random_state(P.shape, 21)
    probe = np.full((P.nz, P.ny, P.nx), 1.0 / P.ncell)
    J, gQ, gt = P.adjoint(e0, 1, probe)
    hq = 1e17
    Qu = np.full((P.nz, P.ny, P.nx), hq, np.float32)
    fd = (_J(P, e0, 1, probe, Qu, None) - _J(P, e0, 1, probe, -Qu, None)) / (2 * float(np.float32(hq)))
    assert abs(fd - gQ.sum()) <= 1e-10 * abs(fd)


# A periodic pair with a temperature difference (Sec. 2.2 (iv)) shifts the pair's ghosts by a
# constant: the step stays affine in e with the same Jacobian structure, the limiter's partials
# being taken at the shifted ghost values.
JUMP_GRIDS = [
    (1, (12, 1, 1), [PER] * 6, (0.7, 0, 0)),
    (2, (7, 6, 1), [PER, PER, DIF, ISO, PER, PER], (-0.4, 0, 0)),
    (3, (5, 4, 4), [PER, PER, PER, PER, DIF, ISO], (0.3, 0.6, 0)),
]


@pytest.mark.parametrize("limiter", [0, 1, 2])
@pytest.mark.parametrize("dim,n,bc,jump", JUMP_GRIDS)
def test_adjoint_and_tangent_with_periodic_jump(dim, n, bc, jump, limiter):
    cfg = small_cfg(dim, n, bc, Tw=TW, nb=2, jump=jump)
    P = oracle_problem(cfg, limiter)
    # a state on the scale of the jump's ghost offset C_k dT / W (~1e4), so that the limiter's
    # arguments are not dominated by the offset (central differences would straddle its kink)
    e = inputs.random_state(P.shape, 23) * 1e4
    de = inputs.random_state(P.shape, 24, smooth=False)
    lam = inputs.random_state(P.shape, 25, smooth=False)
    t = P.step_tangent(e, de)
    a = float(np.vdot(lam, t))
    b = float(np.vdot(P.adjoint_step(e, lam), de))
    assert abs(a - b) <= 1e-13 * max(abs(a), np.linalg.norm(lam) * np.linalg.norm(de))
    h = 1e-2 if limiter == 0 else 1e-5
    fd = (P.step(e + h * de) - P.step(e - h * de)) / (2 * h)
    assert np.max(np.abs(fd - t)) <= (1e-9 if limiter == 0 else 1e-5) * np.max(np.abs(fd))


@pytest.mark.parametrize("dim,n,bc", [GRIDS[2], GRIDS[4]])
def test_checkpointed_run_adjoint_is_bitwise_the_stored_one(dim, n, bc):
    """Keeping every ckpt-th state and recomputing the rest gives bitwise the gradients of
    keeping every state (ckpt = 0): the forward step is deterministic."""
    cfg = small_cfg(dim, n, bc, Tw=TW, nb=3)
    P = oracle_problem(cfg, 2)
    e0 = inputs.random_state(P.shape, 3) * 1e3
    Q = (np.random.default_rng(1).random((P.nz, P.ny, P.nx)) * 1e17).astype(np.float32)
    p = np.random.default_rng(2).random((P.nz, P.ny, P.nx))
    amps = np.linspace(1, 0.2, 13)
    ref = P.adjoint(e0, 13, p, Q, amps, ckpt=0)
    for ck in (1, 4, 5, 13):
        J, gQ, gt = P.adjoint(e0, 13, p, Q, amps, ckpt=ck)
        assert J == ref[0] and np.array_equal(gQ, ref[1]) and np.array_equal(gt, ref[2])
