"""The seeded synthetic workloads are the configurations the benchmark and the parity tests name:
grid, bands, quadrature, walls, seeds, steps, sources, probes and checkpoint spacing, and the
band and time-step recipes (so that an edit cannot change what a measurement refers to)."""
import math

import numpy as np
import pytest

from paper_2306_14181_gb300 import inputs

ISO, DIF, SPE, PER = 0, 1, 2, 3


@pytest.mark.parametrize("make,dim,n,h,nb,seed,quad,bc,steps", [
    (inputs.film_1d, 1, (100, 1, 1), 1e-9, 10, 1001, ("gl1d", 16), [ISO, ISO, PER, PER, PER, PER], 2000),
    (inputs.hotspot_2d, 2, (256, 256, 1), 2e-9, 40, 1002, ("octant", 4, 4), [DIF, DIF, ISO, DIF, PER, PER], 5000),
    (inputs.laser_3d, 3, (128, 128, 64), 5e-9, 40, 1003, ("octant", 4, 3), [PER, PER, PER, PER, ISO, DIF], 220),
    (inputs.film_adjoint_2d, 2, (128, 128, 1), 2e-9, 20, 1004, ("octant", 2, 4), [SPE, SPE, ISO, DIF, PER, PER], 2000),
    (inputs.block_adjoint_3d, 3, (96, 96, 96), 5e-9, 32, 1005, ("octant", 4, 3), [SPE, SPE, SPE, SPE, ISO, DIF], 1000),
])
def test_workload_definitions(make, dim, n, h, nb, seed, quad, bc, steps):
    cfg = make()
    assert cfg["dim"] == dim and tuple(cfg["n"]) == n and cfg["h"][0] == h
    assert cfg["nb"] == nb and cfg["seed"] == seed and tuple(cfg["quad"]) == quad
    assert list(cfg["bc"]) == bc and cfg["steps"] == steps
    # directions: 16 (1-D) or 8 x ntheta x nphi
    nd = quad[1] if quad[0] == "gl1d" else 8 * quad[1] * quad[2]
    assert nd == {1001: 16, 1002: 128, 1003: 96, 1004: 64, 1005: 96}[seed]
    # the bands of the seed, and the time step of the multi-dimensional CFL reading
    C, v, tau = inputs.bands(seed, nb)
    assert np.array_equal(cfg["C"], C) and np.array_equal(cfg["v"], v) and np.array_equal(cfg["tau"], tau)
    assert cfg["dt"] == pytest.approx(0.5 * h / (math.sqrt(dim) * v.max()), rel=1e-15)


def test_band_recipe():
    C, v, tau = inputs.bands(1002, 40)
    assert np.all((v >= 1e3) & (v <= 8e3)) and np.all((tau >= 1e-12) & (tau <= 1e-8))
    assert np.all(C > 0) and C.sum() == pytest.approx(1.66e6, rel=1e-14)
    C2, v2, tau2 = inputs.bands(1002, 40)
    assert np.array_equal(C, C2) and np.array_equal(v, v2) and np.array_equal(tau, tau2)


def test_sources_probes_and_checkpoints():
    hot = inputs.hotspot_2d()
    assert hot["source"]["kind"] == "gaussian" and hot["source"]["sigma"] == 20e-9 and hot["source"]["q0"] == 1e18
    assert hot["Tw"] == [0, 0, 0, 0, 0, 0]
    las = inputs.laser_3d()["source"]
    assert las["kind"] == "laser" and las["sigma"] == 50e-9 and las["depth"] == 1.5e-6
    assert las["q0"] == 4.64e18 and las["sigma_t"] == 1e-12 and las["t0"] == 4e-12
    film = inputs.film_1d()
    assert film["Tw"][:2] == [0.5, -0.5] and film["source"] is None
    c4, c5 = inputs.film_adjoint_2d(), inputs.block_adjoint_3d()
    assert c4["ckpt"] == 100 and c5["ckpt"] == 50
    # probes: a 16 x 16 box at the top centre of the film; the top layer of the block
    p4 = inputs.probe_weights(c4)
    assert p4.shape == (1, 128, 128) and np.count_nonzero(p4) == 256 and p4.sum() == pytest.approx(1.0)
    assert np.all(p4[0, 112:, 56:72] > 0)
    p5 = inputs.probe_weights(c5)
    assert np.count_nonzero(p5) == 96 * 96 and np.all(p5[95] > 0) and p5.sum() == pytest.approx(1.0)
