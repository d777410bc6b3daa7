"""Shared helpers for the tests: turn a workload dict into an oracle problem."""
import numpy as np

from oracle import Problem
from oracle import quadrature as oq
from oracle.oracle import LIM_VANALBADA


def oracle_quadrature(quad):
    if quad[0] == "gl1d":
        return oq.polar_1d(quad[1])
    return oq.octant_rule(quad[1], quad[2])


def oracle_problem(cfg, limiter=LIM_VANALBADA, **over):
    c = dict(cfg)
    c.update(over)
    s, w, mirror = oracle_quadrature(c["quad"])
    return Problem(c["dim"], c["n"], c["h"], c["C"], c["v"], c["tau"], s, w, mirror, c["bc"], c["Tw"], c["dt"],
                   limiter, jump=c.get("jump"))


def small_cfg(dim, n, bc, Tw=(0, 0, 0, 0, 0, 0), nb=3, quad=None, h=2e-9, seed=7, beta=0.5, tau=None, v=None,
              jump=None):
    """A small synthetic problem for pins."""
    from paper_2306_14181_gb300 import inputs
    C, vv, tt = inputs.bands(seed, nb)
    if tau is not None:
        tt = np.full(nb, float(tau)) if np.isscalar(tau) else np.asarray(tau, float)
    if v is not None:
        vv = np.full(nb, float(v)) if np.isscalar(v) else np.asarray(v, float)
    if quad is None:
        quad = ("gl1d", 8) if dim == 1 else ("octant", 2, 2)
    hh = (h, h, h)
    cfg = dict(dim=dim, n=tuple(n), h=hh, nb=nb, C=C, v=vv, tau=tt, quad=quad, bc=list(bc), Tw=list(Tw),
               dt=inputs.cfl_time_step(hh[:dim], vv, beta))
    if jump is not None:
        cfg["jump"] = list(jump)
    return cfg


def rel_linf(a, b):
    a = np.asarray(a, float)
    b = np.asarray(b, float)
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


def gpu_ctx(cfg, **opts):
    """A GPU context for a workload/small-config dict (imports the binding lazily)."""
    from paper_2306_14181_gb300 import bte
    if cfg.get("jump") is not None:
        opts.setdefault("dT_jump", cfg["jump"])
    return bte.bte_create(cfg["dim"], cfg["n"], cfg["h"], cfg["C"], cfg["v"], cfg["tau"], cfg["quad"], cfg["bc"],
                          cfg["Tw"], opts.pop("dt", cfg["dt"]), **opts)


def run_both(cfg, e0, nsteps, Q=None, amps=None, limiter=2, storage=0, kernel=0, T_scale=1.0, **opts):
    """Run the same start state on the GPU and on the oracle.  e0 is taken as float32 (the GPU
    state); the oracle starts from exactly those values.  Returns (gpu_e, gpu_TL, orc_e, orc_TL)."""
    from paper_2306_14181_gb300 import bte
    P = oracle_problem(cfg, limiter)
    ctx = gpu_ctx(cfg, limiter=limiter, storage=storage, kernel=kernel, T_scale=T_scale, **opts)
    e32 = np.ascontiguousarray(e0, dtype=np.float32)
    if storage == 0:
        bte.bte_set_state(ctx, e32)
        start = e32.astype(np.float64)
    else:
        bte.bte_init_temperature(ctx, None)
        start = P.equilibrium(0.0)
        assert not np.any(e0), "16-bit runs start from the zero state"
    if Q is not None:
        bte.bte_set_source(ctx, np.ascontiguousarray(Q, dtype=np.float32), amps)
    bte.bte_step(ctx, nsteps)
    g = bte.bte_get_state(ctx)
    _, gTL, _ = bte.bte_moments(ctx)
    eo = P.run(start, nsteps, Q, amps)
    return ctx, g, gTL, eo, P.lattice_temperature(eo)


def fused_TL(ctx):
    """The lattice temperature the step itself formed (the forward kernel's FP32 moment and the
    finalize pass), as opposed to the FP64 recomputation of bte_moments."""
    from paper_2306_14181_gb300 import bte
    return bte.bte_lattice_temperature(ctx).reshape(ctx.shape[2:])
