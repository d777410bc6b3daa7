"""The allocation-free energy reduction (bte_energy_noalloc) against bte_energy.

Some callers may not allocate device memory once they are set up (a host that gives all device
memory to its own pool, or code running where an allocation is not allowed).  For them the
library offers the energy-balance reductions with their scratch in a fixed device array.  This
file runs last so that a failure here does not stop the rest of the GPU suite; it must pass on
its own in a fresh process as well.
"""
import numpy as np
import pytest

from paper_2306_14181_gb300 import inputs
from tests.support import gpu_ctx, oracle_problem, small_cfg

pytestmark = pytest.mark.gpu

ISO, DIF, SPE, PER = 0, 1, 2, 3


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2306_14181_gb300 import build
    build.build()


def _close(a, b, tol=1e-12):
    a, b = np.asarray(a, float), np.asarray(b, float)
    return np.max(np.abs(a - b)) <= tol * max(np.max(np.abs(b)), 1e-300)


@pytest.mark.parametrize("dim,n,bc,storage", [
    (2, (40, 24, 1), [DIF, SPE, ISO, DIF, PER, PER], 0),
    (3, (9, 7, 6), [PER, PER, SPE, DIF, ISO, DIF], 0),
    (3, (96, 10, 9), [SPE, SPE, SPE, SPE, ISO, DIF], 1),
])
def test_noalloc_energy_matches_bte_energy_twice(dim, n, bc, storage):
    from paper_2306_14181_gb300 import bte
    cfg = small_cfg(dim, n, bc, Tw=[0.1, 0.2, 0.3, 0.4, -0.2, 0.5], nb=3)
    P = oracle_problem(cfg)
    ctx = gpu_ctx(cfg, storage=storage)
    if storage == 0:
        bte.bte_set_state(ctx, (inputs.random_state(P.shape, 4) * 1e4).astype(np.float32))
    Q = (np.random.default_rng(2).random((P.nz, P.ny, P.nx)) * 1e17).astype(np.float32)
    bte.bte_set_source(ctx, Q)
    for _ in range(2):                      # two calls in a row, the state changing between them
        bte.bte_step(ctx, 3)
        E, F = bte.bte_energy(ctx)
        E1, F1 = bte.bte_energy_noalloc(ctx)
        E2, F2 = bte.bte_energy_noalloc(ctx)   # and again on the same state
        assert _close(E1, E) and _close(E2, E)
        assert _close(F1, F) and _close(F2, F)


def test_noalloc_energy_rejects_grids_beyond_its_scratch():
    from paper_2306_14181_gb300 import bte
    cfg = small_cfg(3, (256, 256, 130), [PER] * 6, nb=1, quad=("octant", 1, 1))   # 8.5 M cells > 8,388,608
    ctx = gpu_ctx(cfg)
    with pytest.raises(bte.BteError) as ei:
        bte.bte_energy_noalloc(ctx)
    assert ei.value.status == bte.BTE_EINVAL and "at most" in str(ei.value)
