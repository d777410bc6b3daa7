"""Failure detection on the GPU without a fault: the tiled forward kernel's shared-memory waits
are bounded.  A test hook makes the first wait of the consumer warps, of the producer warp, or
of both, wait on a barrier that nothing completes, with the limit cut to 1 ms: the wait gives
up, the kernel must still end (every warp finishes the CTA's schedule, the producer waits for
the copies it issued), the next synchronising call must report BTE_ETIMEOUT once, and the
context must step correctly again afterwards."""
import numpy as np
import pytest

from paper_2306_14181_gb300 import inputs
from tests.support import gpu_ctx, oracle_problem, rel_linf, small_cfg

pytestmark = pytest.mark.gpu

ISO, DIF, SPE, PER = 0, 1, 2, 3
BTE_ETIMEOUT = 6


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2306_14181_gb300 import build
    build.build()


@pytest.mark.parametrize("stall", [1, 2, 3])
@pytest.mark.parametrize("dim,n,bc,storage", [
    (3, (96, 10, 9), [PER, PER, SPE, DIF, ISO, DIF], 0),
    (2, (128, 40, 1), [DIF, SPE, ISO, DIF, PER, PER], 0),
    (3, (96, 10, 9), [SPE, SPE, SPE, SPE, ISO, DIF], 1),
])
def test_wait_gives_up_and_context_recovers(dim, n, bc, storage, stall):
    from paper_2306_14181_gb300 import bte
    cfg = small_cfg(dim, n, bc, Tw=[0.3, -0.2, 0.1, 0.4, -0.3, 0.2], nb=3)
    P = oracle_problem(cfg)
    ctx = gpu_ctx(cfg, kernel=bte.BTE_KERNEL_TILED, storage=storage)
    assert ctx.info.kernel == bte.BTE_KERNEL_TILED
    bte.bte_synchronize(ctx)
    bte.bte_set_wait_limit(ctx, 1000000, stall)
    bte.bte_step(ctx, 1)
    with pytest.raises(bte.BteError) as ex:
        bte.bte_synchronize(ctx)
    assert ex.value.status == BTE_ETIMEOUT
    # reported once: the flag is clear, and the hook applied to one launch only
    bte.bte_step(ctx, 2)
    bte.bte_synchronize(ctx)
    # default limit again; a fresh state steps like the oracle
    bte.bte_set_wait_limit(ctx, 0)
    if storage == 0:
        e0 = (inputs.random_state(P.shape, 31) * 1e4).astype(np.float32)
        bte.bte_set_state(ctx, e0)
        start = e0.astype(np.float64)
    else:
        bte.bte_init_temperature(ctx, None)
        start = P.equilibrium(0.0)
    Q = (np.random.default_rng(2).random((P.nz, P.ny, P.nx)) * 1e17).astype(np.float32)
    bte.bte_set_source(ctx, Q)
    bte.bte_step(ctx, 5)
    bte.bte_synchronize(ctx)
    _, TL, _ = bte.bte_moments(ctx)
    eo = P.run(start, 5, Q)
    assert rel_linf(TL, P.lattice_temperature(eo)) <= (1e-5 if storage == 0 else 2e-3)
