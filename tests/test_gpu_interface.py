"""Interface between two materials (Sec. 2.2 (v), diffuse mismatch) on the GPU, through the C ABI,
against the FP64 oracle: element-wise parity of coupled runs on both sides (tiled and generic
kernels, every axis, two limiters, a source on one side), the exchanged heat and the energy of
the pair, re-initialising one side, uncoupling by destroying the partner, and the refused uses."""
import numpy as np
import pytest

from oracle.oracle import interface_energy, interface_run, interface_step
from tests.support import gpu_ctx, oracle_problem, small_cfg

pytestmark = pytest.mark.gpu

ISO, DIF, SPE, PER, IFC = 0, 1, 2, 3, 4


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2306_14181_gb300 import build
    build.build()


def pair(dim, nA, nB, wa, wb, bcA, bcB, same_v=False, TwA=0.3, TwB=-0.2, quad=None):
    """Configs of material A (band table of seed 7) and B (seed 11) with one time step; the
    interface walls are INTERFACE for the GPU and DIFFUSE for the oracle."""
    bcA, bcB = list(bcA), list(bcB)
    bcA[wa] = DIF
    bcB[wb] = DIF
    cA = small_cfg(dim, nA, bcA, Tw=[TwA] * 6, nb=3, quad=quad)
    cB = small_cfg(dim, nB, bcB, Tw=[TwB] * 6, nb=3, quad=quad, seed=11, v=cA["v"] if same_v else None)
    cA["dt"] = cB["dt"] = min(cA["dt"], cB["dt"])
    return cA, cB


def gpu_pair(cA, cB, wa, wb, bAB, bBA, limiter, kernel=0):
    from paper_2306_14181_gb300 import bte
    gA = dict(cA, bc=[IFC if j == wa else b for j, b in enumerate(cA["bc"])])
    gB = dict(cB, bc=[IFC if j == wb else b for j, b in enumerate(cB["bc"])])
    A = gpu_ctx(gA, limiter=limiter, kernel=kernel)
    B = gpu_ctx(gB, limiter=limiter, kernel=kernel)
    return A, B


def start_states(PA, PB, seed):
    rng = np.random.default_rng(seed)
    eA = PA.equilibrium(rng.uniform(-0.5, 0.5, (PA.nz, PA.ny, PA.nx))) * (1 + 0.2 * rng.standard_normal(PA.shape))
    eB = PB.equilibrium(rng.uniform(-0.5, 0.5, (PB.nz, PB.ny, PB.nx))) * (1 + 0.2 * rng.standard_normal(PB.shape))
    return eA.astype(np.float32), eB.astype(np.float32)


BAB = np.array([0.25, 0.6, 0.85])
BBA = np.array([0.7, 0.35, 0.1])

# (dim, nA, nB, wa, wb, walls of A, walls of B, kernel the pair runs on)
CASES = [
    (2, (96, 20, 1), (64, 20, 1), 1, 0, [ISO, None, SPE, DIF, PER, PER], [None, ISO, SPE, SPE, PER, PER], "tiled"),
    (2, (64, 24, 1), (64, 16, 1), 3, 2, [PER, PER, ISO, None, PER, PER], [PER, PER, None, DIF, PER, PER], "tiled"),
    (3, (64, 8, 6), (32, 8, 6), 1, 0, [DIF, None, SPE, ISO, PER, PER], [None, SPE, PER, PER, ISO, DIF], "tiled"),
    (3, (32, 12, 6), (32, 12, 4), 5, 4, [PER, PER, SPE, DIF, ISO, None], [PER, PER, ISO, SPE, None, SPE], "tiled"),
    (2, (13, 9, 1), (7, 9, 1), 1, 0, [ISO, None, DIF, SPE, PER, PER], [None, SPE, ISO, DIF, PER, PER], "generic"),
    (1, (40, 1, 1), (25, 1, 1), 0, 1, [None, ISO, PER, PER, PER, PER], [DIF, None, PER, PER, PER, PER], "generic"),
    (3, (9, 6, 5), (9, 6, 4), 5, 4, [ISO, DIF, SPE, SPE, DIF, None], [SPE, ISO, DIF, SPE, None, ISO], "generic"),
]


@pytest.mark.parametrize("limiter", [0, 2])
@pytest.mark.parametrize("case", CASES)
def test_interface_pair_elementwise(case, limiter):
    """Both sides after 30 coupled steps from a seeded start, with a heat source in A, element by
    element within 1e-5 of the largest |e| (the FP32 bar of every forward parity test)."""
    from paper_2306_14181_gb300 import bte
    dim, nA, nB, wa, wb, bcA, bcB, kern = case
    quad = ("gl1d", 16) if dim == 1 else None
    cA, cB = pair(dim, nA, nB, wa, wb, bcA, bcB, quad=quad)
    PA, PB = oracle_problem(cA, limiter), oracle_problem(cB, limiter)
    A, B = gpu_pair(cA, cB, wa, wb, BAB, BBA, limiter)
    assert A.info.kernel == (bte.BTE_KERNEL_TILED if kern == "tiled" else bte.BTE_KERNEL_GENERIC)
    eA, eB = start_states(PA, PB, 21)
    bte.bte_set_state(A, eA)
    bte.bte_set_state(B, eB)
    Q = (np.random.default_rng(4).random((PA.nz, PA.ny, PA.nx)) * 3e17).astype(np.float32)
    bte.bte_set_source(A, Q)
    bte.bte_interface(A, wa, B, wb, BAB, BBA)
    n = 30
    bte.bte_step_pair(A, B, n)
    gA, gB = bte.bte_get_state(A), bte.bte_get_state(B)
    oA, oB = eA.astype(np.float64), eB.astype(np.float64)
    for _ in range(n):
        oA, oB = interface_step(PA, oA, wa, PB, oB, wb, BAB, BBA, QA=Q)
    sc = max(np.max(np.abs(oA)), np.max(np.abs(oB)))
    assert np.max(np.abs(gA - oA)) <= 1e-5 * sc
    assert np.max(np.abs(gB - oB)) <= 1e-5 * sc
    # and the interface heat flow each side reports is the oracle's
    EA, FA = bte.bte_energy(A)
    EB, FB = bte.bte_energy(B)
    oEA, oFA, oEB, oFB = interface_energy(PA, oA, wa, PB, oB, wb, BAB, BBA)
    fs = abs(oFA[wa]) + abs(oFB[wb]) + 1e-300
    assert abs(FA[wa] - oFA[wa]) <= 1e-4 * fs
    assert abs(FB[wb] - oFB[wb]) <= 1e-4 * fs


@pytest.mark.parametrize("case", [CASES[0], CASES[3]])
def test_interface_energy_of_the_pair(case):
    """Equal group speeds and every other wall reflecting: the pair's energy E_A + E_B stays put
    over 200 steps (FP32 state: to 1e-5 of the energy moved through the interface), and the
    two sides' interface flows cancel at every check."""
    from paper_2306_14181_gb300 import bte
    dim, nA, nB, wa, wb, bcA, bcB, _ = case
    bcA = [SPE if b in (ISO, DIF) else b for b in bcA]
    bcB = [SPE if b in (ISO, DIF) else b for b in bcB]
    cA, cB = pair(dim, nA, nB, wa, wb, bcA, bcB, same_v=True)
    PA, PB = oracle_problem(cA, 2), oracle_problem(cB, 2)
    A, B = gpu_pair(cA, cB, wa, wb, BAB, BBA, 2)
    dA = np.zeros((PA.nz, PA.ny, PA.nx))
    dA[...] = 1.0  # A warm, B cold: heat flows into B
    bte.bte_init_temperature(A, dA.reshape(-1))
    bte.bte_init_temperature(B, None)
    bte.bte_interface(A, wa, B, wb, BAB, BBA)
    E0 = bte.bte_energy(A)[0] + bte.bte_energy(B)[0]
    EB0 = bte.bte_energy(B)[0]
    for _ in range(4):
        bte.bte_step_pair(A, B, 50)
        EA, FA = bte.bte_energy(A)
        EB, FB = bte.bte_energy(B)
        assert FA[wa] > 0 and FB[wb] < 0
        assert abs(FA[wa] + FB[wb]) <= 1e-5 * abs(FA[wa])
    moved = EB - EB0
    assert moved > 0
    assert abs(EA + EB - E0) <= 1e-5 * moved


def test_reinit_keeps_the_coupling_and_destroy_releases_it():
    """bte_init_temperature on one side forms the interface values again from both current
    states; after the partner is destroyed the wall is a plain diffuse wall."""
    from paper_2306_14181_gb300 import bte
    dim, nA, nB, wa, wb, bcA, bcB, _ = CASES[0]
    cA, cB = pair(dim, nA, nB, wa, wb, bcA, bcB)
    PA, PB = oracle_problem(cA, 2), oracle_problem(cB, 2)
    A, B = gpu_pair(cA, cB, wa, wb, BAB, BBA, 2)
    eA, eB = start_states(PA, PB, 8)
    bte.bte_set_state(A, eA)
    bte.bte_set_state(B, eB)
    bte.bte_interface(A, wa, B, wb, BAB, BBA)
    bte.bte_step_pair(A, B, 5)
    _, oB5 = interface_run(PA, eA.astype(np.float64), wa, PB, eB.astype(np.float64), wb, BAB, BBA, 5)
    dT = np.linspace(-0.4, 0.4, PA.ncell)
    bte.bte_init_temperature(A, dT)
    bte.bte_step_pair(A, B, 7)
    gA, gB = bte.bte_get_state(A), bte.bte_get_state(B)
    oA, oB = interface_run(PA, PA.equilibrium(dT.reshape(PA.nz, PA.ny, PA.nx)), wa, PB, oB5, wb, BAB, BBA, 7)
    sc = max(np.max(np.abs(oA)), np.max(np.abs(oB)))
    assert np.max(np.abs(gA - oA)) <= 1e-5 * sc
    assert np.max(np.abs(gB - oB)) <= 1e-5 * sc
    with pytest.raises(bte.BteError) as ei:
        bte.bte_step(A, 1)
    assert ei.value.status == bte.BTE_ESTATE
    with pytest.raises(bte.BteError) as ei:
        bte.bte_adjoint(B, 2, np.ones(PB.ncell))
    assert ei.value.status == bte.BTE_ESTATE
    bte.bte_destroy(B)
    before = bte.bte_get_state(A).astype(np.float64)
    bte.bte_step(A, 1)
    assert np.max(np.abs(bte.bte_get_state(A) - PA.step(before))) <= 1e-5 * np.max(np.abs(before))


def test_interface_uses_that_are_refused():
    from paper_2306_14181_gb300 import bte
    dim, nA, nB, wa, wb, bcA, bcB, _ = CASES[0]
    cA, cB = pair(dim, nA, nB, wa, wb, bcA, bcB)
    gA = dict(cA, bc=[IFC if j == wa else b for j, b in enumerate(cA["bc"])])
    with pytest.raises(bte.BteError) as ei:            # 16-bit storage
        gpu_ctx(gA, storage=bte.BTE_STORE_F16)
    assert ei.value.status == bte.BTE_EUNSUPPORTED
    with pytest.raises(bte.BteError) as ei:            # two interface walls
        gpu_ctx(dict(gA, bc=[IFC, IFC, SPE, DIF, PER, PER]))
    assert ei.value.status == bte.BTE_EINVAL
    A, B = gpu_pair(cA, cB, wa, wb, BAB, BBA, 2)
    for args in [(A, wa, A, wa), (A, wb, B, wb), (A, wa, B, wa)]:
        with pytest.raises(bte.BteError) as ei:        # same context, wrong walls, same side
            bte.bte_interface(*args, 0.5, 0.5)
        assert ei.value.status == bte.BTE_EINVAL
    with pytest.raises(bte.BteError) as ei:            # transmission outside [0, 1]
        bte.bte_interface(A, wa, B, wb, [0.5, 1.5, 0.5], 0.5)
    assert ei.value.status == bte.BTE_EINVAL
    cC, _ = pair(dim, (96, 24, 1), nB, wa, wb, bcA, bcB)
    C = gpu_ctx(dict(cC, bc=[IFC if j == wa else b for j, b in enumerate(cC["bc"])]))
    with pytest.raises(bte.BteError) as ei:            # 24 rows against 20
        bte.bte_interface(C, wa, B, wb, 0.5, 0.5)
    assert ei.value.status == bte.BTE_EINVAL
    with pytest.raises(bte.BteError) as ei:            # not coupled
        bte.bte_step_pair(A, B, 1)
    assert ei.value.status == bte.BTE_ESTATE


def test_interface_workload_reduced():
    """The benchmark's two-material workload at 128 x 24 cells a side, 4 bands and 32 directions
    (same walls, source placement, band draws and transmissions): 20 coupled steps on both
    sides against the oracle, element by element within 1e-5."""
    from paper_2306_14181_gb300 import bte, inputs
    cfg = inputs.interface_2d(nx=128, ny=24, nb=4, ntheta=2, nphi=2)
    wa, wb = cfg["wall_a"], cfg["wall_b"]
    PA, PB = oracle_problem(cfg["A"], 2), oracle_problem(cfg["B"], 2)
    ctx = []
    for side, w in (("A", wa), ("B", wb)):
        c = dict(cfg[side])
        c["bc"] = [IFC if j == w else b for j, b in enumerate(c["bc"])]
        ctx.append(bte.bte_from_workload(c))
    A, B = ctx
    assert A.info.kernel == bte.BTE_KERNEL_TILED and B.info.kernel == bte.BTE_KERNEL_TILED
    Q = inputs.source_field(cfg["A"])
    bte.bte_set_source(A, Q)
    bte.bte_interface(A, wa, B, wb, cfg["beta_ab"], cfg["beta_ba"])
    bte.bte_step_pair(A, B, 20)
    oA, oB = PA.equilibrium(0.0), PB.equilibrium(0.0)
    for _ in range(20):
        oA, oB = interface_step(PA, oA, wa, PB, oB, wb, cfg["beta_ab"], cfg["beta_ba"], QA=Q)
    sc = max(np.max(np.abs(oA)), np.max(np.abs(oB)))
    assert np.max(np.abs(oB)) > 1e-3 * sc  # heat reached B through the interface
    assert np.max(np.abs(bte.bte_get_state(A) - oA)) <= 1e-5 * sc
    assert np.max(np.abs(bte.bte_get_state(B) - oB)) <= 1e-5 * sc


def test_interface_with_a_periodic_jump_across():
    """The interface on x while y is a periodic pair with a temperature difference in A (Sec. 2.2
    (iv) and (v) together): 20 coupled steps against the oracle within 1e-5."""
    from paper_2306_14181_gb300 import bte
    cA, cB = pair(2, (40, 12, 1), (24, 12, 1), 1, 0, [ISO, None, PER, PER, PER, PER], [None, ISO, PER, PER, PER, PER])
    cA["jump"] = [0.0, 0.4, 0.0]
    PA, PB = oracle_problem(cA, 2), oracle_problem(cB, 2)
    A, B = gpu_pair(cA, cB, 1, 0, BAB, BBA, 2)
    eA, eB = start_states(PA, PB, 44)
    bte.bte_set_state(A, eA)
    bte.bte_set_state(B, eB)
    bte.bte_interface(A, 1, B, 0, BAB, BBA)
    bte.bte_step_pair(A, B, 20)
    oA, oB = interface_run(PA, eA.astype(np.float64), 1, PB, eB.astype(np.float64), 0, BAB, BBA, 20)
    sc = max(np.max(np.abs(oA)), np.max(np.abs(oB)))
    assert np.max(np.abs(bte.bte_get_state(A) - oA)) <= 1e-5 * sc
    assert np.max(np.abs(bte.bte_get_state(B) - oB)) <= 1e-5 * sc


def test_ballistic_flux_through_the_interface():
    """The series law on the GPU: ballistic transport between thermalizing walls 1 K apart
    through an interface of transmission 0.3 carries 0.3 of the wall-to-wall ballistic flux,
    within 1e-5 (FP32 state)."""
    from paper_2306_14181_gb300 import bte
    t = 0.3
    cA = small_cfg(1, (12, 1, 1), [ISO, DIF, PER, PER, PER, PER], Tw=[0.5, 0, 0, 0, 0, 0], nb=1, quad=("gl1d", 16),
                   h=1e-9, tau=1e3, v=1e3)
    cB = small_cfg(1, (12, 1, 1), [DIF, ISO, PER, PER, PER, PER], Tw=[0, -0.5, 0, 0, 0, 0], nb=1, quad=("gl1d", 16),
                   h=1e-9, tau=1e3, v=1e3)
    for c in (cA, cB):
        c["C"] = np.array([1.66e6])
    A, B = gpu_pair(cA, cB, 1, 0, t, t, 2)
    bte.bte_init_temperature(A, None)
    bte.bte_init_temperature(B, None)
    bte.bte_interface(A, 1, B, 0, t, t)
    bte.bte_step_pair(A, B, 3000)
    PA = oracle_problem(cA, 2)
    half = float((PA.w * np.clip(PA.s[:, 0], 0, None)).sum()) / PA.W
    expect = t * 1.66e6 * 1e3 * 1.0 * half
    for ctx in (A, B):
        _, _, q = bte.bte_moments(ctx)
        assert np.max(np.abs(q[0] - expect)) <= 1e-5 * expect
