"""Steady implicit DOM, sequential iterative scheme (Sec. 3.3-3.5), on the GPU through the C ABI
against the FP64 oracle: element-wise parity of single and repeated iterations (tiled and
generic forward kernels, 1-D to 3-D, rows longer than one sweep chunk, two limiters, sources,
every wall type, a periodic temperature difference), a converged steady state, the in-plane
film's conductivity against the time-marched value, and the refused uses."""
import numpy as np
import pytest

from paper_2306_14181_gb300 import inputs
from tests.support import gpu_ctx, oracle_problem, small_cfg

pytestmark = pytest.mark.gpu

ISO, DIF, SPE, PER = 0, 1, 2, 3
TW = [0.3, -0.2, 0.1, 0.4, -0.3, 0.2]


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2306_14181_gb300 import build
    build.build()


# (dim, n, walls, quadrature, periodic jump, forward kernel)
CASES = [
    (1, (40, 1, 1), [ISO, DIF, PER, PER, PER, PER], ("gl1d", 16), None, "generic"),
    (2, (96, 20, 1), [DIF, SPE, ISO, DIF, PER, PER], None, None, "tiled"),
    (2, (200, 13, 1), [SPE, DIF, SPE, ISO, PER, PER], None, None, "tiled"),
    (2, (13, 9, 1), [ISO, SPE, DIF, DIF, PER, PER], None, None, "generic"),
    (2, (37, 11, 1), [PER, PER, DIF, SPE, PER, PER], None, (0.6, 0, 0), "generic"),
    (3, (32, 12, 6), [PER, PER, SPE, DIF, ISO, DIF], None, None, "tiled"),
    (3, (7, 5, 4), [DIF, ISO, PER, PER, SPE, ISO], None, None, "generic"),
]


def _start(P, seed):
    rng = np.random.default_rng(seed)
    e = P.equilibrium(rng.uniform(-0.5, 0.5, (P.nz, P.ny, P.nx))) * (1 + 0.2 * rng.standard_normal(P.shape))
    return e.astype(np.float32)


@pytest.mark.parametrize("limiter", [0, 2])
@pytest.mark.parametrize("case", CASES)
def test_iterations_elementwise(case, limiter):
    """One and then five more iterations from a seeded start with a source, element by element
    within 1e-5 of the largest |e| (the FP32 bar)."""
    from paper_2306_14181_gb300 import bte
    dim, n, bc, quad, jump, kern = case
    cfg = small_cfg(dim, n, bc, Tw=TW, nb=3, quad=quad, jump=jump)
    P = oracle_problem(cfg, limiter)
    ctx = gpu_ctx(cfg, limiter=limiter)
    assert ctx.info.kernel in ((bte.BTE_KERNEL_TILED,) if kern == "tiled" else
                               (bte.BTE_KERNEL_GENERIC, bte.BTE_KERNEL_PERSISTENT))
    e0 = _start(P, 31)
    Q = (np.random.default_rng(5).random((P.nz, P.ny, P.nx)) * 2e17).astype(np.float32)
    bte.bte_set_state(ctx, e0)
    bte.bte_set_source(ctx, Q)
    bte.bte_sis_iterate(ctx, 1)
    eo = P.sis_iteration(e0.astype(np.float64), Q)
    g = bte.bte_get_state(ctx)
    assert np.max(np.abs(g - eo)) <= 1e-5 * np.max(np.abs(eo))
    bte.bte_sis_iterate(ctx, 5)
    for _ in range(5):
        eo = P.sis_iteration(eo, Q)
    g = bte.bte_get_state(ctx)
    assert np.max(np.abs(g - eo)) <= 1e-5 * np.max(np.abs(eo))
    # T_L of the new state is formed after each iteration
    _, gTL, _ = bte.bte_moments(ctx)
    assert np.max(np.abs(gTL - P.lattice_temperature(eo))) <= 1e-5 * np.max(np.abs(P.lattice_temperature(eo)))


@pytest.mark.parametrize("case", [CASES[1], CASES[5]])
def test_converged_steady_state(case):
    """The residual loop to eps_T, eps_q < 1e-6 on the GPU against the oracle's converged
    (1e-12) steady state: T_L within 1e-4 of its largest value, the state solving the steady
    equation to the same level (the oracle's explicit step moves it by at most 1e-4 of the
    largest |e|; a change of 1e-6 between iterates leaves a residual about ten times larger)."""
    from paper_2306_14181_gb300 import bte
    dim, n, bc, quad, jump, kern = case
    cfg = small_cfg(dim, n, bc, Tw=TW, nb=3, quad=quad, jump=jump)
    P = oracle_problem(cfg, 2)
    ctx = gpu_ctx(cfg, limiter=2)
    Q = (np.random.default_rng(5).random((P.nz, P.ny, P.nx)) * 2e17).astype(np.float32)
    bte.bte_init_temperature(ctx, None)
    bte.bte_set_source(ctx, Q)
    it, eT, eq = bte.bte_run_steady_implicit(ctx, 3000, 10, 1e-6, 1e-6)
    assert eT < 1e-6 and eq < 1e-6
    eo, oit, oT, oq = P.run_sis(P.equilibrium(0.0), 5000, 1e-12, 1e-12, Q)
    _, gTL, _ = bte.bte_moments(ctx)
    oTL = P.lattice_temperature(eo)
    assert np.max(np.abs(gTL - oTL)) <= 1e-4 * np.max(np.abs(oTL))
    g = bte.bte_get_state(ctx).astype(np.float64)
    assert np.max(np.abs(P.step(g, Q) - g)) <= 1e-4 * np.max(np.abs(g))


def test_inplane_film_conductivity():
    """The in-plane film (periodic x with a 1 K difference, diffuse top and bottom) by implicit
    iterations: eps_T, eps_q < 1e-6 within 200 iterations (the FP32 right-hand side, a
    difference of two states, keeps the change between iterates near 1e-7), and its in-plane
    conductivity equals the oracle's converged one (the explicit step's steady state) within
    1e-4."""
    from paper_2306_14181_gb300 import bte
    cfg = inputs.inplane_film_2d()
    ctx = bte.bte_from_workload(cfg)
    it, eT, eq = bte.bte_run_steady_implicit(ctx, 200, 5, 1e-6, 1e-6)
    assert it < 200 and eT < 1e-6 and eq < 1e-6
    _, _, q = bte.bte_moments(ctx)
    L = cfg["n"][0] * cfg["h"][0]
    k_sis = float(np.mean(q[0])) * L / cfg["jump"][0]
    P = oracle_problem(cfg, 2)
    eo, oit, oT, oq = P.run_sis(P.equilibrium(0.0), 400, 1e-10, 1e-10)
    _, _, qo = P.moments(eo)
    k_orc = float(np.mean(qo[0])) * L / cfg["jump"][0]
    assert abs(k_sis - k_orc) <= 1e-4 * k_orc
    # the oracle's fixed point is the explicit step's steady state
    assert np.max(np.abs(P.step(eo) - eo)) <= 1e-9 * np.max(np.abs(eo))


def test_implicit_uses_that_are_refused():
    from paper_2306_14181_gb300 import bte
    cfg = small_cfg(2, (96, 20, 1), [DIF, SPE, ISO, DIF, PER, PER], Tw=TW, nb=3)
    ctx = gpu_ctx(cfg, storage=bte.BTE_STORE_F16)
    with pytest.raises(bte.BteError) as ei:
        bte.bte_sis_iterate(ctx, 1)
    assert ei.value.status == bte.BTE_EUNSUPPORTED
    ctx = gpu_ctx(cfg)
    with pytest.raises(bte.BteError) as ei:
        bte.bte_sis_iterate(ctx, -1)
    assert ei.value.status == bte.BTE_EINVAL
    with pytest.raises(bte.BteError) as ei:
        bte.bte_run_steady_implicit(ctx, 0, 1, 1e-6, 1e-6)
    assert ei.value.status == bte.BTE_EINVAL


# closed boxes (no thermalizing wall): the macroscopic equation is singular
SINGULAR = [
    (2, (96, 20, 1), [SPE, DIF, PER, PER, PER, PER], None, None, "tiled"),
    (3, (32, 8, 6), [PER, PER, SPE, DIF, SPE, DIF], None, None, "tiled"),
    (3, (7, 5, 4), [DIF, SPE, PER, PER, SPE, DIF], None, None, "generic"),
]


@pytest.mark.parametrize("limiter", [0, 2])
@pytest.mark.parametrize("case", CASES + SINGULAR)
def test_synthetic_iterations_elementwise(case, limiter):
    """Synthetic iterations (Sec. 3.5): one and then three more from a seeded start with a source
    (none when no wall is thermalizing, the macroscopic equation then being singular), the state
    element by element and the corrected lattice temperature against the oracle within 1e-5."""
    from paper_2306_14181_gb300 import bte
    dim, n, bc, quad, jump, kern = case
    cfg = small_cfg(dim, n, bc, Tw=TW, nb=3, quad=quad, jump=jump)
    P = oracle_problem(cfg, limiter)
    ctx = gpu_ctx(cfg, limiter=limiter)
    bte.bte_set_steady_scheme(ctx, bte.BTE_SCHEME_SYNTHETIC)
    e0 = _start(P, 33)
    regular = ISO in bc[:2 * dim]
    Q = (np.random.default_rng(6).random((P.nz, P.ny, P.nx)) * 2e17).astype(np.float32) if regular else None
    bte.bte_set_state(ctx, e0)
    if Q is not None:
        bte.bte_set_source(ctx, Q)
    eo = e0.astype(np.float64)
    TLo = P.lattice_temperature(eo)
    for m in (1, 3):
        bte.bte_sis_iterate(ctx, m)
        for _ in range(m):
            eo, TLo = P.synthetic_iteration(eo, TLo, Q)
        g = bte.bte_get_state(ctx)
        assert np.max(np.abs(g - eo)) <= 1e-5 * np.max(np.abs(eo))
        gTL = bte.bte_lattice_temperature(ctx).reshape(TLo.shape)
        assert np.max(np.abs(gTL - TLo)) <= 1e-5 * np.max(np.abs(TLo))


def test_synthetic_scheme_near_the_diffusive_limit():
    """A film between two walls 1 K apart with relaxation times far below a cell's flight time:
    the sequential scheme needs hundreds of iterations to eps_T, eps_q < 1e-6, the synthetic one a
    few tens to 1e-5 (in FP32 its change between iterates settles near 1e-6: a correction from the
    energy residual of an FP32 state), and both land on the oracle's steady lattice temperature
    within 1e-4."""
    from paper_2306_14181_gb300 import bte
    cfg = small_cfg(1, (30, 1, 1), [ISO, ISO, PER, PER, PER, PER], Tw=[0.5, -0.5, 0, 0, 0, 0], nb=1,
                    quad=("gl1d", 16), h=1e-9, tau=1e-12, v=1e3)
    cfg["C"] = np.array([1.66e6])
    P = oracle_problem(cfg, 2)
    eo, _, _, _ = P.run_synthetic(P.equilibrium(0.0), 500, 1e-12, 1e-12)
    oTL = P.lattice_temperature(eo)
    its = {}
    for scheme in (bte.BTE_SCHEME_SEQUENTIAL, bte.BTE_SCHEME_SYNTHETIC):
        ctx = gpu_ctx(cfg, limiter=2)
        bte.bte_set_steady_scheme(ctx, scheme)
        bte.bte_init_temperature(ctx, None)
        tol = 1e-6 if scheme == bte.BTE_SCHEME_SEQUENTIAL else 1e-5
        it, eT, eq = bte.bte_run_steady_implicit(ctx, 5000, 5, tol, tol)
        assert eT < tol and eq < tol
        _, gTL, _ = bte.bte_moments(ctx)
        assert np.max(np.abs(gTL.ravel() - oTL.ravel())) <= 1e-4 * np.max(np.abs(oTL))
        its[scheme] = it
    assert its[bte.BTE_SCHEME_SYNTHETIC] <= 60 and its[bte.BTE_SCHEME_SEQUENTIAL] >= 4 * its[bte.BTE_SCHEME_SYNTHETIC]
    with pytest.raises(bte.BteError) as ei:
        bte.bte_set_steady_scheme(ctx, 2)
    assert ei.value.status == bte.BTE_EINVAL


def test_time_steps_after_synthetic_iterations():
    """Time steps that follow synthetic iterations start from the state's own T_L (the corrected
    one is only the next sweep's): they match the oracle's steps from the same state."""
    from paper_2306_14181_gb300 import bte
    dim, n, bc, quad, jump, kern = CASES[1]
    cfg = small_cfg(dim, n, bc, Tw=TW, nb=3, quad=quad, jump=jump)
    P = oracle_problem(cfg, 2)
    ctx = gpu_ctx(cfg, limiter=2)
    bte.bte_set_steady_scheme(ctx, bte.BTE_SCHEME_SYNTHETIC)
    bte.bte_set_state(ctx, _start(P, 35))
    bte.bte_sis_iterate(ctx, 3)
    e3 = bte.bte_get_state(ctx).astype(np.float64)
    bte.bte_step(ctx, 2)
    eo = P.run(e3, 2)
    assert np.max(np.abs(bte.bte_get_state(ctx) - eo)) <= 1e-5 * np.max(np.abs(eo))
