"""GPU path at the benchmark's full sizes, in the launch configuration bench.py times (the
tiled kernel, FP32 state): after a few steps, one more step is checked element by element on
sampled (band, direction, cell) outputs that the FP64 oracle computes one by one from the same
state (Eq. disretized_transientBTE with T_L and the diffuse-wall values formed from that state),
and the discrete energy balance E^{n+1} - E^n = dt (V a sum Q - sum wall flows) is checked over
the whole grid with the FP64 diagnostics.  Samples include wall cells and corners.
"""
import numpy as np
import pytest

from paper_2306_14181_gb300 import inputs
from tests.support import fused_TL, gpu_ctx, oracle_problem, rel_linf

pytestmark = pytest.mark.gpu

TOL = 1e-5


def _samples(P, n, seed):
    """n random (k, d, cell) triples plus every plane at the domain's corner and edge cells."""
    rng = np.random.default_rng(seed)
    k = rng.integers(0, P.nb, n)
    d = rng.integers(0, P.nd, n)
    i = rng.integers(0, P.ncell, n)
    special = []
    xs, ys = (0, 1, P.nx - 1), (0, 1, P.ny - 1)
    zs = (0, P.nz - 1) if P.nz > 1 else (0,)
    for z in zs:
        for y in ys:
            for x in xs:
                special.append((z * P.ny + y) * P.nx + x)
    kk = rng.integers(0, P.nb, 8 * len(special))
    dd = rng.integers(0, P.nd, 8 * len(special))
    ii = np.repeat(np.array(special), 8)
    return np.stack([np.concatenate([k, kk]), np.concatenate([d, dd]), np.concatenate([i, ii])], axis=1)


def _check(cfg, warm, seed):
    from paper_2306_14181_gb300 import bte
    P = oracle_problem(cfg)
    ctx = gpu_ctx(cfg)
    assert ctx.info.kernel == bte.BTE_KERNEL_TILED
    Q = inputs.source_field(cfg)
    amps = inputs.source_amplitudes(cfg, warm + 4)
    bte.bte_set_source(ctx, Q, amps)
    bte.bte_step(ctx, warm)
    e_n = bte.bte_get_state(ctx)                       # FP32 state e^n
    E0, F0 = bte.bte_energy(ctx)
    bte.bte_step(ctx, 1)
    E1, _ = bte.bte_energy(ctx)
    e_n1 = bte.bte_get_state(ctx).reshape(P.nb * P.nd, P.ncell)
    # energy balance over the whole grid
    a = 1.0 if amps is None else float(amps[warm])
    rhs = P.dt * (P.cell_volume * a * float(Q.astype(np.float64).sum()) - F0.sum())
    assert abs((E1 - E0) - rhs) <= 1e-5 * max(abs(E0), abs(rhs))
    # sampled outputs against the oracle, from the same FP32 state
    pts = _samples(P, 3000, seed)
    e64 = e_n.astype(np.float64)
    del e_n
    ref = P.step_points(e64, pts, Q, a)
    got = e_n1[pts[:, 0] * P.nd + pts[:, 1], pts[:, 2]].astype(np.float64)
    scale = np.max(np.abs(e64))
    assert np.max(np.abs(got - ref)) <= TOL * scale
    # the T_L the step formed (FP32 moment partials and the finalize pass) against the oracle's
    # T_L of the stored state e^{n+1} (Eq. BTE_get_e0)
    del e64
    oTL = P.lattice_temperature(e_n1.astype(np.float64).reshape(P.shape))
    assert rel_linf(fused_TL(ctx), oTL) <= TOL


def test_hotspot_2d_full_size_sampled():
    """256 x 256 cells, 40 bands, 128 directions (335.5 M updates a step)."""
    _check(inputs.hotspot_2d(), 6, 11)


def test_laser_3d_full_grid_sampled():
    """The full 128 x 128 x 64 grid and 96 directions with 4 of the 40 bands (the FP64 copy of the
    whole state the oracle reads would not fit in host memory with 40)."""
    _check(inputs.laser_3d(nb=4), 6, 12)
