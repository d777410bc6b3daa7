"""Seeded synthetic inputs for the explicit DOM transient step (arXiv 2306.14181).

This module only draws and lays out input data: band properties, source fields, pulse
amplitudes, workload definitions and random states.  It holds none of the method's
arithmetic, so both the CUDA library's tests and the FP64 oracle can take their inputs from
it.  The paper's first-principles silicon data are not available; the band draws below stand
in for them (silicon-like ranges of group speed, relaxation time and heat capacity).

Boundary codes: 0 isothermal, 1 diffuse, 2 specular, 3 periodic; walls -x,+x,-y,+y,-z,+z.
"""
import math

import numpy as np

ISOTHERMAL, DIFFUSE, SPECULAR, PERIODIC = 0, 1, 2, 3
T_REF = 300.0
C_TOTAL = 1.66e6  # J/(m^3 K), sum of the band heat capacities


def bands(seed, nb):
    """Synthetic non-gray spectrum: |v| log-uniform in [1e3, 8e3] m/s, tau log-uniform in
    [1e-12, 1e-8] s, positive heat capacities summing to 1.66e6 J/(m^3 K).
    Draw order: u (speeds), u' (relaxation times), r (capacity weights)."""
    rng = np.random.default_rng(seed)
    u = rng.random(nb)
    up = rng.random(nb)
    r = rng.uniform(0.1, 1.0, nb)
    v = 1e3 * 8.0 ** u
    tau = 1e-12 * 1e4 ** up
    C = C_TOTAL * r / r.sum()
    return C, v, tau


def cfl_time_step(h, v, beta=0.5):
    """dt = beta * dx_min / (sqrt(dim) * max|v|), dim = len(h).

    Sec. 4.1 writes the CFL rule as dt = beta dx_min / v.  In more than one dimension the
    explicit update moves a cell's content along every active axis at once, so the speed
    that matters is v * sum_a |s_a| <= v * sqrt(dim); with the bare per-axis rule (beta = 0.5)
    the limited scheme overshoots in 2-D and grows without bound in 3-D.  In 1-D this is the
    paper's rule unchanged."""
    return beta * min(h) / (math.sqrt(len(h)) * float(np.max(v)))


def cell_centres(n, h):
    """Cell-centre coordinates (x, y, z) as broadcastable arrays of shape (nz, ny, nx)."""
    nx, ny, nz = n
    x = (np.arange(nx) + 0.5) * h[0]
    y = (np.arange(ny) + 0.5) * h[1]
    z = (np.arange(nz) + 0.5) * h[2]
    return x[None, None, :], y[None, :, None], z[:, None, None]


def gaussian_spot(n, h, centre, sigma, q0):
    """In-plane Gaussian heat source q0 exp(-r^2 / (2 sigma^2)) (W/m^3), float32 (nz, ny, nx)."""
    x, y, z = cell_centres(n, h)
    r2 = (x - centre[0]) ** 2 + (y - centre[1]) ** 2
    q = q0 * np.exp(-r2 / (2.0 * sigma * sigma)) + 0.0 * z
    return np.ascontiguousarray(q, dtype=np.float32)


def laser_source(n, h, centre_xy, sigma_r, depth, q0):
    """Laser-heating source q0 exp(-r^2/(2 sigma_r^2)) exp(-d/depth) with d the distance below
    the top (+z) surface; float32 (nz, ny, nx)."""
    nx, ny, nz = n
    x, y, z = cell_centres(n, h)
    r2 = (x - centre_xy[0]) ** 2 + (y - centre_xy[1]) ** 2
    d = nz * h[2] - z
    q = q0 * np.exp(-r2 / (2.0 * sigma_r * sigma_r)) * np.exp(-d / depth)
    return np.ascontiguousarray(np.broadcast_to(q, (nz, ny, nx)), dtype=np.float32)


def pulse_amplitudes(nsteps, dt, t0, sigma_t):
    """Temporal pulse a(t_n) = exp(-(t_n - t0)^2 / (2 sigma_t^2)), t_n = n dt."""
    t = np.arange(nsteps) * dt
    return np.exp(-((t - t0) ** 2) / (2.0 * sigma_t * sigma_t))


def random_state(shape, seed, scale=1.0, smooth=True):
    """A seeded random field of the state's shape (nb, nd, nz, ny, nx), float64.
    With ``smooth`` the field is a sum of a few long-wave modes plus small noise, so that
    both limited and unlimited slopes occur."""
    rng = np.random.default_rng(seed)
    nb, nd, nz, ny, nx = shape
    if not smooth:
        return scale * rng.standard_normal(shape)
    z = np.arange(nz)[:, None, None]
    y = np.arange(ny)[None, :, None]
    x = np.arange(nx)[None, None, :]
    f = np.zeros(shape)
    for _ in range(3):
        amp = rng.standard_normal((nb, nd, 1, 1, 1))
        kx, ky, kz = rng.uniform(0.0, 0.6, 3)
        ph = rng.uniform(0.0, 2 * math.pi, 3)
        f += amp * (np.cos(kx * x + ph[0]) * np.cos(ky * y + ph[1]) * np.cos(kz * z + ph[2]))[None, None]
    f += 0.3 * rng.standard_normal(shape)
    return scale * f


# ---------------------------------------------------------------------------------------
# Workloads.  Each is a plain dict; sizes follow the paper-shaped configurations:
#   film   - quasi-1D cross-plane film between isothermal walls (Sec. 3.6 shaped)
#   hotspot- 2D device hot spot, isothermal bottom, diffuse other walls (Sec. 6.2 shaped)
#   laser  - 3D laser-heated block, periodic sides (Sec. 6.3 shaped)
#   film_adjoint, block_adjoint - the workloads the adjoint gradients are taken on
# ---------------------------------------------------------------------------------------

def _base(name, dim, n, h, nb, seed, quad, bc, Tw, steps, source=None, **extra):
    C, v, tau = bands(seed, nb)
    cfg = dict(name=name, dim=dim, n=tuple(n), h=tuple(h), nb=nb, seed=seed, quad=quad,
               bc=list(bc), Tw=list(Tw), steps=steps, C=C, v=v, tau=tau,
               dt=cfl_time_step(h[:dim], v), source=source)
    cfg.update(extra)
    return cfg


def film_1d(nx=100, steps=2000):
    """1-D film: 100 cells of 1 nm, walls at +0.5 K / -0.5 K about T_ref, 10 bands, 16 polar
    directions, no source."""
    return _base("film_1d_100x10x16", 1, (nx, 1, 1), (1e-9, 1e-9, 1e-9), 10, 1001, ("gl1d", 16),
                 [ISOTHERMAL, ISOTHERMAL, PERIODIC, PERIODIC, PERIODIC, PERIODIC],
                 [0.5, -0.5, 0, 0, 0, 0], steps)


def hotspot_2d(nx=256, ny=256, nb=40, ntheta=4, nphi=4, steps=5000):
    """2-D hot spot: 256x256 cells of 2 nm, 40 bands, 128 directions; bottom isothermal at
    T_ref, other walls diffuse; Gaussian source sigma = 20 nm, 1e18 W/m^3, centred at
    (L/2, 0.75 L)."""
    h = (2e-9, 2e-9, 2e-9)
    L = (nx * h[0], ny * h[1])
    src = dict(kind="gaussian", centre=(0.5 * L[0], 0.75 * L[1]), sigma=20e-9, q0=1e18)
    return _base("hotspot_2d_%dx%d_%dx%d" % (nx, ny, nb, 8 * ntheta * nphi), 2, (nx, ny, 1), h, nb, 1002,
                 ("octant", ntheta, nphi), [DIFFUSE, DIFFUSE, ISOTHERMAL, DIFFUSE, PERIODIC, PERIODIC],
                 [0, 0, 0, 0, 0, 0], steps, src)


def laser_3d(nx=128, ny=128, nz=64, nb=40, ntheta=4, nphi=3, steps=220):
    """3-D laser block: 128x128x64 cells of 5 nm, 40 bands, 96 directions; periodic in x and y,
    isothermal bottom, diffuse top; Gaussian pulse sigma_r = 50 nm, penetration 1.5 um,
    Q0 = 4.64e18 W/m^3, sigma_t = 1 ps centred at t0 = 4 ps."""
    h = (5e-9, 5e-9, 5e-9)
    src = dict(kind="laser", centre=(0.5 * nx * h[0], 0.5 * ny * h[1]), sigma=50e-9, depth=1.5e-6,
               q0=4.64e18, t0=4e-12, sigma_t=1e-12)
    return _base("laser_3d_%dx%dx%d_%dx%d" % (nx, ny, nz, nb, 8 * ntheta * nphi), 3, (nx, ny, nz), h, nb, 1003,
                 ("octant", ntheta, nphi), [PERIODIC, PERIODIC, PERIODIC, PERIODIC, ISOTHERMAL, DIFFUSE],
                 [0, 0, 0, 0, 0, 0], steps, src)


def film_adjoint_2d(nx=128, ny=128, nb=20, ntheta=2, nphi=4, steps=2000, ckpt=100):
    """2-D adjoint film: 128x128 cells of 2 nm, 20 bands, 64 directions; specular side walls,
    isothermal bottom, diffuse top; Gaussian source sigma = 10 cells at the centre; probe =
    the top-centre 16x16 cells."""
    h = (2e-9, 2e-9, 2e-9)
    src = dict(kind="gaussian", centre=(0.5 * nx * h[0], 0.5 * ny * h[1]), sigma=10 * h[0], q0=1e18)
    px = min(16, nx)
    py = min(16, ny)
    probe = dict(x=(nx // 2 - px // 2, nx // 2 - px // 2 + px), y=(ny - py, ny), z=(0, 1))
    return _base("film_adjoint_2d_%dx%d_%dx%d" % (nx, ny, nb, 8 * ntheta * nphi), 2, (nx, ny, 1), h, nb, 1004,
                 ("octant", ntheta, nphi), [SPECULAR, SPECULAR, ISOTHERMAL, DIFFUSE, PERIODIC, PERIODIC],
                 [0, 0, 0, 0, 0, 0], steps, src, probe=probe, ckpt=ckpt)


def block_adjoint_3d(nx=96, ny=96, nz=96, nb=32, ntheta=4, nphi=3, steps=1000, ckpt=50):
    """3-D adjoint block: 96^3 cells of 5 nm, 32 bands, 96 directions; specular side walls
    (the symmetry planes of a quarter domain, beam centred on their common edge),
    isothermal bottom, diffuse top; the laser pulse of ``laser_3d``; probe = the top layer."""
    h = (5e-9, 5e-9, 5e-9)
    src = dict(kind="laser", centre=(0.0, 0.0), sigma=50e-9, depth=1.5e-6, q0=4.64e18, t0=4e-12,
               sigma_t=1e-12)
    probe = dict(x=(0, nx), y=(0, ny), z=(nz - 1, nz))
    return _base("block_adjoint_3d_%dx%dx%d_%dx%d" % (nx, ny, nz, nb, 8 * ntheta * nphi), 3, (nx, ny, nz), h, nb,
                 1005, ("octant", ntheta, nphi), [SPECULAR, SPECULAR, SPECULAR, SPECULAR, ISOTHERMAL, DIFFUSE],
                 [0, 0, 0, 0, 0, 0], steps, src, probe=probe, ckpt=ckpt)


def inplane_film_2d(nx=64, ny=64, ntheta=2, nphi=3, dT=1.0):
    """In-plane conduction of a film (the verification problem (b) of Sec. 5 shaped): a square cell
    of 64 x 64 cells of 5 nm, periodic along x with a temperature difference of 1 K between the
    two periodic ends, diffusely reflecting top and bottom; 3 seeded bands with relaxation times
    2, 10 and 40 ps (seed 7 speeds and capacities), 48 directions.  The time step is half the
    transient workloads' (beta = 0.25) so that the limited scheme reaches a steady state."""
    C, v, _ = bands(7, 3)
    tau = np.array([2e-12, 1e-11, 4e-11])
    h = (5e-9, 5e-9, 5e-9)
    cfg = dict(name="inplane_film_2d_%dx%d_3x%d" % (nx, ny, 8 * ntheta * nphi), dim=2, n=(nx, ny, 1), h=h, nb=3,
               seed=7, quad=("octant", ntheta, nphi), bc=[PERIODIC, PERIODIC, DIFFUSE, DIFFUSE, PERIODIC, PERIODIC],
               Tw=[0.0] * 6, steps=20000, C=C, v=v, tau=tau, dt=cfl_time_step(h[:2], v, 0.25), source=None,
               jump=[dT, 0.0, 0.0])
    return cfg


def interface_2d(nx=256, ny=128, nb=40, ntheta=4, nphi=4):
    """Two materials side by side (an interface problem of Sec. 2.2 (v) shaped like the Ge-Si
    verification problem of Sec. 5): material A (seed 1002 bands) on 256 x 128 cells of 2 nm, its
    +x wall against the -x wall of material B (seed 2002 bands) on another 256 x 128 cells; 40
    bands and 128 directions on both sides; thermalizing outer x walls at T_ref, diffuse top and
    bottom; the hot spot's Gaussian source (sigma = 20 nm, 1e18 W/m^3) in A, 40 nm from the
    interface.  Band transmissions of the diffuse-mismatch form beta_AB = C_B / (C_A + C_B),
    beta_BA = C_A / (C_A + C_B) (they sum to one and keep a uniform temperature stationary).
    One time step: the smaller CFL step of the two."""
    h = (2e-9, 2e-9, 2e-9)
    quad = ("octant", ntheta, nphi)
    name = "interface_2d_2x%dx%d_%dx%d" % (nx, ny, nb, 8 * ntheta * nphi)
    src = dict(kind="gaussian", centre=((nx - 20) * h[0], 0.5 * ny * h[1]), sigma=20e-9, q0=1e18)
    A = _base(name + "_A", 2, (nx, ny, 1), h, nb, 1002, quad, [ISOTHERMAL, DIFFUSE, DIFFUSE, DIFFUSE, PERIODIC, PERIODIC],
              [0] * 6, 1000, src)
    B = _base(name + "_B", 2, (nx, ny, 1), h, nb, 2002, quad, [DIFFUSE, ISOTHERMAL, DIFFUSE, DIFFUSE, PERIODIC, PERIODIC],
              [0] * 6, 1000, None)
    A["dt"] = B["dt"] = min(A["dt"], B["dt"])
    return dict(name=name, A=A, B=B, wall_a=1, wall_b=0, beta_ab=B["C"] / (A["C"] + B["C"]),
                beta_ba=A["C"] / (A["C"] + B["C"]))


# gray silicon of the paper's verification problems (Sec. 5): one band
GRAY_SI = dict(C=1627600.0, v=2677.0, tau=39.9e-12)


def diffusive_film_1d(nx=100, h=40e-9, ntheta=16):
    """A gray-silicon film 4 um thick (100 cells of 40 nm, about 37 mean free paths) between
    thermalizing walls 0.5 K above and below T_ref, 16 Gauss-Legendre directions: the
    near-diffusive steady problem on which the sequential iterations of the steady solver slow
    down and the synthetic scheme of Sec. 3.5 is meant to help."""
    hh = (h, h, h)
    C, v, tau = (np.array([GRAY_SI[k]]) for k in ("C", "v", "tau"))
    return dict(name="diffusive_film_1d_%d_1x%d" % (nx, ntheta), dim=1, n=(nx, 1, 1), h=hh, nb=1, seed=0,
                quad=("gl1d", ntheta), bc=[ISOTHERMAL, ISOTHERMAL, PERIODIC, PERIODIC, PERIODIC, PERIODIC],
                Tw=[0.5, -0.5, 0, 0, 0, 0], steps=0, C=C, v=v, tau=tau, dt=cfl_time_step(hh[:1], v), source=None)


def ttg_1d(xi=1.0, nx=1000, ntheta=512, nb=1, A0=1.0, t_star=None):
    """Transient thermal grating (Sec. 4.2): one period L of T(x, 0) = A0 cos(2 pi x / L) with
    periodic ends, 1000 cells and 512 directions (GL in mu).  Gray silicon by default; the
    period follows from xi = 2 pi Kn = 2 pi v tau / L.  With nb > 1 the seeded non-gray bands
    (seed 1006) are used and L is fixed by xi on the capacity-weighted mean of v tau.  The run
    covers t* = t / tau up to 10 / xi (diffusive decay at small xi, ballistic at large), about
    3200 steps at the CFL time step for every xi."""
    if nb == 1:
        C, v, tau = (np.array([GRAY_SI[k]]) for k in ("C", "v", "tau"))
    else:
        C, v, tau = bands(1006, nb)
    vt = float(np.sum(C * v * tau) / np.sum(C))
    tau_ref = float(np.sum(C * tau) / np.sum(C))
    L = 2 * math.pi * vt / xi
    h = (L / nx, L / nx, L / nx)
    dt = cfl_time_step(h[:1], v)
    t_end = (10.0 / xi if t_star is None else t_star) * tau_ref
    steps = int(math.ceil(t_end / dt))
    cfg = dict(name="ttg_1d_%d_%dx%d_xi%g" % (nx, nb, ntheta, xi), dim=1, n=(nx, 1, 1), h=h, nb=nb, seed=1006,
               quad=("gl1d", ntheta), bc=[PERIODIC] * 6, Tw=[0.0] * 6, steps=steps, C=C, v=v, tau=tau, dt=dt,
               source=None, xi=xi, L=L, A0=A0, tau_ref=tau_ref)
    return cfg


def ttg_initial_temperature(cfg):
    """T(x, 0) - T_ref = A0 cos(2 pi x / L) at the cell centres, shape (nz, ny, nx)."""
    x = (np.arange(cfg["n"][0]) + 0.5) * cfg["h"][0]
    return (cfg["A0"] * np.cos(2 * math.pi * x / cfg["L"]))[None, None, :]


def grating_amplitude(cfg, T):
    """A = (2/N) sum_i T_i cos(2 pi x_i / L): the amplitude of the grating's mode in a field T."""
    x = (np.arange(cfg["n"][0]) + 0.5) * cfg["h"][0]
    return 2.0 / cfg["n"][0] * float(np.sum(np.asarray(T).reshape(-1) * np.cos(2 * math.pi * x / cfg["L"])))


def source_field(cfg):
    """Per-cell source Q_i (W/m^3) of a workload, float32 (nz, ny, nx), or None."""
    src = cfg.get("source")
    if src is None:
        return None
    if src["kind"] == "gaussian":
        return gaussian_spot(cfg["n"], cfg["h"], src["centre"], src["sigma"], src["q0"])
    return laser_source(cfg["n"], cfg["h"], src["centre"], src["sigma"], src["depth"], src["q0"])


def source_amplitudes(cfg, nsteps):
    """a(t_n) for n < nsteps, or None when the source is steady."""
    src = cfg.get("source")
    if src is None or "t0" not in src:
        return None
    return pulse_amplitudes(nsteps, cfg["dt"], src["t0"], src["sigma_t"])


def probe_weights(cfg):
    """J = mean of dT_L over the probe box: weights 1/|box| inside, 0 outside; (nz, ny, nx)."""
    nx, ny, nz = cfg["n"]
    p = cfg["probe"]
    wgt = np.zeros((nz, ny, nx))
    wgt[p["z"][0]:p["z"][1], p["y"][0]:p["y"][1], p["x"][0]:p["x"][1]] = 1.0
    return wgt / wgt.sum()
