"""Thin ctypes binding of the C ABI in ``include/bte.h`` (libbte_gb300.so).

Every function here only marshals arguments; all work of the explicit DOM transient step
(arXiv 2306.14181, Sec. 4) runs in the library's CUDA kernels.  There is no CPU fallback: if
the library is missing or cannot be loaded, ``load()`` raises.

Arrays: host data as numpy arrays, device data as CUDA torch tensors (passed by pointer,
``on_device = 1``).  State layout e[k][d][z][y][x].
"""
import ctypes as ct
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libbte_gb300.so")

BTE_OK, BTE_EINVAL, BTE_ENOMEM, BTE_ECUDA, BTE_ESTATE, BTE_ENONFINITE, BTE_ETIMEOUT, BTE_EUNSUPPORTED = range(8)
BTE_QUAD_GL1D_POLAR, BTE_QUAD_OCTANT, BTE_QUAD_EXPLICIT = 0, 1, 2
BTE_BC_ISOTHERMAL, BTE_BC_DIFFUSE, BTE_BC_SPECULAR, BTE_BC_PERIODIC, BTE_BC_INTERFACE = 0, 1, 2, 3, 4
BTE_STORE_F32, BTE_STORE_F16, BTE_STORE_BF16 = 0, 1, 2
BTE_LIM_FIRST_ORDER, BTE_LIM_MINMOD, BTE_LIM_VANALBADA = 0, 1, 2
BTE_ROUND_NEAREST, BTE_ROUND_STOCHASTIC = 0, 1
BTE_KERNEL_AUTO, BTE_KERNEL_GENERIC, BTE_KERNEL_TILED, BTE_KERNEL_PERSISTENT = 0, 1, 2, 3
BTE_SCHEME_SEQUENTIAL, BTE_SCHEME_SYNTHETIC = 0, 1

# every entry point include/bte.h declares
EXPORTS = ["bte_create", "bte_destroy", "bte_last_error", "bte_init_temperature", "bte_set_source", "bte_step",
           "bte_lattice_temperature", "bte_moments", "bte_energy", "bte_get_state", "bte_set_state",
           "bte_get_values", "bte_adjoint", "bte_adjoint_profile_read",
           "bte_get_info", "bte_get_quadrature", "bte_synchronize", "bte_profile", "bte_profile_read", "bte_energy_noalloc",
           "bte_set_wait_limit", "bte_residuals", "bte_run_steady", "bte_interface", "bte_step_pair",
           "bte_sis_iterate", "bte_run_steady_implicit", "bte_set_steady_scheme"]

_STATUS = {1: "EINVAL", 2: "ENOMEM", 3: "ECUDA", 4: "ESTATE", 5: "ENONFINITE", 6: "ETIMEOUT", 7: "EUNSUPPORTED"}


class BteError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("BTE_%s: %s" % (_STATUS.get(status, str(status)), msg))
        self.status = status


class bte_grid(ct.Structure):
    _fields_ = [("dim", ct.c_int), ("nx", ct.c_int), ("ny", ct.c_int), ("nz", ct.c_int),
                ("dx", ct.c_double), ("dy", ct.c_double), ("dz", ct.c_double), ("Tref", ct.c_double)]


class bte_bands(ct.Structure):
    _fields_ = [("nbands", ct.c_int), ("C", ct.POINTER(ct.c_double)), ("vabs", ct.POINTER(ct.c_double)),
                ("tau", ct.POINTER(ct.c_double))]


class bte_quadrature(ct.Structure):
    _fields_ = [("kind", ct.c_int), ("ntheta", ct.c_int), ("nphi", ct.c_int), ("ndirs", ct.c_int),
                ("s", ct.POINTER(ct.c_double)), ("w", ct.POINTER(ct.c_double))]


class bte_boundaries(ct.Structure):
    _fields_ = [("type", ct.c_int * 6), ("T_wall", ct.c_double * 6), ("dT_jump", ct.c_double * 3)]


class bte_options(ct.Structure):
    _fields_ = [("dt", ct.c_double), ("storage", ct.c_int), ("limiter", ct.c_int), ("T_scale", ct.c_double),
                ("rounding", ct.c_int), ("stream", ct.c_void_p), ("seed", ct.c_uint64), ("kernel", ct.c_int)]


class bte_info(ct.Structure):
    _fields_ = [("dim", ct.c_int), ("nx", ct.c_int), ("ny", ct.c_int), ("nz", ct.c_int), ("nbands", ct.c_int),
                ("ndirs", ct.c_int), ("ncell", ct.c_longlong), ("nelem", ct.c_longlong),
                ("state_bytes", ct.c_size_t), ("elem_bytes", ct.c_int), ("storage", ct.c_int),
                ("limiter", ct.c_int), ("kernel", ct.c_int), ("dt", ct.c_double), ("W", ct.c_double),
                ("step", ct.c_longlong), ("device_bytes", ct.c_size_t), ("launches_per_step", ct.c_int)]


_lib = None


def load():
    """Load libbte_gb300.so (raises if it is not built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError("libbte_gb300.so is not built; run `python -m paper_2306_14181_gb300.build`")
    lib = ct.CDLL(LIB_PATH)
    P = ct.c_void_p
    dp = ct.POINTER(ct.c_double)
    lib.bte_create.argtypes = [ct.POINTER(bte_grid), ct.POINTER(bte_bands), ct.POINTER(bte_quadrature),
                               ct.POINTER(bte_boundaries), ct.POINTER(bte_options), ct.POINTER(P)]
    lib.bte_destroy.argtypes = [P]
    lib.bte_destroy.restype = None
    lib.bte_last_error.argtypes = [P]
    lib.bte_last_error.restype = ct.c_char_p
    lib.bte_init_temperature.argtypes = [P, dp]
    lib.bte_set_source.argtypes = [P, P, ct.c_int, dp, ct.c_int]
    lib.bte_step.argtypes = [P, ct.c_int]
    lib.bte_lattice_temperature.argtypes = [P, dp]
    lib.bte_moments.argtypes = [P, dp, dp, dp]
    lib.bte_energy.argtypes = [P, dp, dp]
    lib.bte_energy_noalloc.argtypes = [P, dp, dp]
    lib.bte_get_state.argtypes = [P, P, ct.c_size_t, P, ct.c_int]
    lib.bte_set_state.argtypes = [P, P, ct.c_size_t, P, ct.c_int, ct.c_int]
    lib.bte_get_values.argtypes = [P, P, ct.c_int]
    lib.bte_adjoint.argtypes = [P, ct.c_int, ct.c_int, P, P, P, P]
    lib.bte_adjoint_profile_read.argtypes = [P, P, P, P, P]
    lib.bte_get_info.argtypes = [P, ct.POINTER(bte_info)]
    lib.bte_get_quadrature.argtypes = [P, dp, dp]
    lib.bte_synchronize.argtypes = [P]
    lib.bte_set_wait_limit.argtypes = [P, ct.c_longlong, ct.c_int]
    lib.bte_residuals.argtypes = [P, ct.c_int, dp, dp]
    lib.bte_run_steady.argtypes = [P, ct.c_longlong, ct.c_int, ct.c_double, ct.c_double,
                                   ct.POINTER(ct.c_longlong), dp, dp]
    lib.bte_sis_iterate.argtypes = [P, ct.c_int]
    lib.bte_set_steady_scheme.argtypes = [P, ct.c_int]
    lib.bte_run_steady_implicit.argtypes = [P, ct.c_longlong, ct.c_int, ct.c_double, ct.c_double,
                                            ct.POINTER(ct.c_longlong), dp, dp]
    lib.bte_interface.argtypes = [P, ct.c_int, P, ct.c_int, dp, dp]
    lib.bte_step_pair.argtypes = [P, P, ct.c_int]
    lib.bte_profile.argtypes = [P, ct.c_int]
    lib.bte_profile_read.argtypes = [P, dp, ct.POINTER(ct.c_longlong), dp, ct.POINTER(ct.c_longlong)]
    for name in EXPORTS:
        f = getattr(lib, name)
        if name not in ("bte_destroy", "bte_last_error"):
            f.restype = ct.c_int
    _lib = lib
    return lib


def _check(st, handle):
    if st != BTE_OK:
        msg = load().bte_last_error(handle)
        raise BteError(st, msg.decode() if msg else "")


def _dp(a):
    return None if a is None else a.ctypes.data_as(ct.POINTER(ct.c_double))


def _ptr(x):
    """(pointer, on_device) of a numpy array or a torch tensor."""
    if hasattr(x, "data_ptr"):
        return ct.c_void_p(x.data_ptr()), int(x.is_cuda)
    return ct.c_void_p(x.ctypes.data), 0


class Context:
    """Owner of one bte_ctx handle (destroyed with the object)."""

    def __init__(self, handle, keep):
        self.handle = handle
        self._keep = keep
        info = bte_get_info(self)
        self.shape = (info.nbands, info.ndirs, info.nz, info.ny, info.nx)
        self.info = info

    def __del__(self):
        if getattr(self, "handle", None):
            try:
                load().bte_destroy(self.handle)
            except Exception:
                pass
            self.handle = None


def _current_stream():
    try:
        import torch
        if torch.cuda.is_available():
            return ct.c_void_p(torch.cuda.current_stream().cuda_stream)
    except Exception:
        pass
    return ct.c_void_p(0)


def bte_create(dim, n, h, C, vabs, tau, quad, bc, T_wall, dt, storage=BTE_STORE_F32, limiter=BTE_LIM_VANALBADA,
               T_scale=1.0, rounding=BTE_ROUND_NEAREST, stream=None, seed=0, kernel=BTE_KERNEL_AUTO, Tref=300.0,
               dT_jump=None):
    """bte_create.  quad: ("gl1d", n) | ("octant", ntheta, nphi) | ("explicit", s[nd,3], w[nd]);
    dT_jump: temperature difference (K) across each periodic pair (None: none)."""
    lib = load()
    C = np.ascontiguousarray(C, dtype=np.float64)
    vabs = np.ascontiguousarray(vabs, dtype=np.float64)
    tau = np.ascontiguousarray(tau, dtype=np.float64)
    g = bte_grid(int(dim), int(n[0]), int(n[1]), int(n[2]), float(h[0]), float(h[1]), float(h[2]), float(Tref))
    b = bte_bands(C.size, _dp(C), _dp(vabs), _dp(tau))
    keep = [C, vabs, tau]
    if quad[0] == "gl1d":
        q = bte_quadrature(BTE_QUAD_GL1D_POLAR, int(quad[1]), 0, 0, None, None)
    elif quad[0] == "octant":
        q = bte_quadrature(BTE_QUAD_OCTANT, int(quad[1]), int(quad[2]), 0, None, None)
    else:
        s = np.ascontiguousarray(quad[1], dtype=np.float64).reshape(-1, 3)
        w = np.ascontiguousarray(quad[2], dtype=np.float64)
        keep += [s, w]
        q = bte_quadrature(BTE_QUAD_EXPLICIT, 0, 0, w.size, _dp(s), _dp(w))
    jmp = [0.0, 0.0, 0.0] if dT_jump is None else [float(x) for x in dT_jump]
    wl = bte_boundaries((ct.c_int * 6)(*[int(x) for x in bc]), (ct.c_double * 6)(*[float(x) for x in T_wall]),
                        (ct.c_double * 3)(*jmp))
    st = _current_stream() if stream is None else ct.c_void_p(stream)
    o = bte_options(float(dt), int(storage), int(limiter), float(T_scale), int(rounding), st, int(seed), int(kernel))
    h_ = ct.c_void_p()
    rc = lib.bte_create(ct.byref(g), ct.byref(b), ct.byref(q), ct.byref(wl), ct.byref(o), ct.byref(h_))
    _check(rc, None)
    return Context(h_, keep)


def bte_from_workload(cfg, **opts):
    """bte_create for a workload dict of ``paper_2306_14181_gb300.inputs``."""
    if cfg.get("jump") is not None:
        opts.setdefault("dT_jump", cfg["jump"])
    return bte_create(cfg["dim"], cfg["n"], cfg["h"], cfg["C"], cfg["v"], cfg["tau"], cfg["quad"], cfg["bc"],
                      cfg["Tw"], opts.pop("dt", cfg["dt"]), **opts)


def bte_destroy(ctx):
    if ctx.handle:
        load().bte_destroy(ctx.handle)
        ctx.handle = None


def bte_last_error(ctx=None):
    m = load().bte_last_error(ctx.handle if ctx is not None else None)
    return m.decode() if m else ""


def bte_init_temperature(ctx, dT0=None):
    a = None if dT0 is None else np.ascontiguousarray(dT0, dtype=np.float64).reshape(-1)
    _check(load().bte_init_temperature(ctx.handle, _dp(a)), ctx.handle)


def bte_set_source(ctx, Q, amp=None):
    """Q: numpy float32 (host) or CUDA float32 tensor (device), ncell values; None removes it."""
    if Q is None:
        _check(load().bte_set_source(ctx.handle, None, 0, None, 0), ctx.handle)
        return
    if not hasattr(Q, "data_ptr"):
        Q = np.ascontiguousarray(Q, dtype=np.float32).reshape(-1)
    p, dev = _ptr(Q)
    a = None if amp is None else np.ascontiguousarray(amp, dtype=np.float64)
    ctx._src = (Q, a)
    _check(load().bte_set_source(ctx.handle, p, dev, _dp(a), 0 if a is None else a.size), ctx.handle)


def bte_step(ctx, n=1):
    _check(load().bte_step(ctx.handle, int(n)), ctx.handle)


def bte_interface(ctx_a, wall_a, ctx_b, wall_b, beta_ab, beta_ba):
    """Couple wall wall_a of ctx_a (material A) with wall wall_b of ctx_b (material B) as a
    diffuse-mismatch interface; beta_ab[k] / beta_ba[k] are the band transmissions A->B / B->A
    (scalars are broadcast over the bands)."""
    nb = ctx_a.info.nbands
    bab = np.ascontiguousarray(np.broadcast_to(np.asarray(beta_ab, dtype=np.float64), (nb,)))
    bba = np.ascontiguousarray(np.broadcast_to(np.asarray(beta_ba, dtype=np.float64), (nb,)))
    _check(load().bte_interface(ctx_a.handle, int(wall_a), ctx_b.handle, int(wall_b), _dp(bab), _dp(bba)),
           ctx_a.handle)


def bte_step_pair(ctx_a, ctx_b, n=1):
    _check(load().bte_step_pair(ctx_a.handle, ctx_b.handle, int(n)), ctx_a.handle)


def bte_synchronize(ctx):
    _check(load().bte_synchronize(ctx.handle), ctx.handle)


def bte_set_wait_limit(ctx, limit_ns=0, stall_test=0):
    """Limit (ns) of the tiled forward kernel's bounded waits (0: the default 2 s); stall_test 1/2/3
    makes the consumers'/producer's/both first waits of the next launch wait on a barrier nothing
    completes (a failure-detection test)."""
    _check(load().bte_set_wait_limit(ctx.handle, int(limit_ns), int(stall_test)), ctx.handle)


def bte_residuals(ctx, nsteps=1):
    """Run nsteps steps; (eps_T, eps_q) of Algorithm 2 between the last two states."""
    eT, eq = ct.c_double(), ct.c_double()
    _check(load().bte_residuals(ctx.handle, int(nsteps), ct.byref(eT), ct.byref(eq)), ctx.handle)
    return eT.value, eq.value


def bte_run_steady(ctx, max_steps, check_every, tol_T, tol_q):
    """Step until eps_T < tol_T and eps_q < tol_q (checked every check_every steps) or max_steps:
    returns (steps run, eps_T, eps_q)."""
    n, eT, eq = ct.c_longlong(), ct.c_double(), ct.c_double()
    _check(load().bte_run_steady(ctx.handle, int(max_steps), int(check_every), float(tol_T), float(tol_q),
                                 ct.byref(n), ct.byref(eT), ct.byref(eq)), ctx.handle)
    return n.value, eT.value, eq.value


def bte_sis_iterate(ctx, n=1):
    """n iterations of the steady implicit DOM's sequential scheme."""
    _check(load().bte_sis_iterate(ctx.handle, int(n)), ctx.handle)


def bte_set_steady_scheme(ctx, scheme):
    """BTE_SCHEME_SEQUENTIAL or BTE_SCHEME_SYNTHETIC for the steady implicit iterations."""
    _check(load().bte_set_steady_scheme(ctx.handle, int(scheme)), ctx.handle)


def bte_run_steady_implicit(ctx, max_iters, check_every, tol_T, tol_q):
    """Implicit iterations until eps_T < tol_T and eps_q < tol_q (checked every check_every
    iterations) or max_iters: returns (iterations run, eps_T, eps_q)."""
    n, eT, eq = ct.c_longlong(), ct.c_double(), ct.c_double()
    _check(load().bte_run_steady_implicit(ctx.handle, int(max_iters), int(check_every), float(tol_T), float(tol_q),
                                          ct.byref(n), ct.byref(eT), ct.byref(eq)), ctx.handle)
    return n.value, eT.value, eq.value


def bte_lattice_temperature(ctx, out=None):
    nc = ctx.info.ncell
    out = np.empty(nc) if out is None else out
    _check(load().bte_lattice_temperature(ctx.handle, _dp(out)), ctx.handle)
    return out


def bte_moments(ctx):
    """(dT, dTL, q) as float64 arrays of shapes (nz,ny,nx), (nz,ny,nx), (3,nz,ny,nx)."""
    i = ctx.info
    g = (i.nz, i.ny, i.nx)
    T = np.empty(i.ncell)
    TL = np.empty(i.ncell)
    q = np.empty(3 * i.ncell)
    _check(load().bte_moments(ctx.handle, _dp(T), _dp(TL), _dp(q)), ctx.handle)
    return T.reshape(g), TL.reshape(g), q.reshape((3,) + g)


def bte_energy(ctx):
    E = np.zeros(1)
    F = np.zeros(6)
    _check(load().bte_energy(ctx.handle, _dp(E), _dp(F)), ctx.handle)
    return float(E[0]), F


def bte_energy_noalloc(ctx):
    """bte_energy's reductions without device allocation (for callers that may not allocate
    device memory after set-up); see include/bte.h for its size limit and concurrency rules."""
    E = np.zeros(1)
    F = np.zeros(6)
    _check(load().bte_energy_noalloc(ctx.handle, _dp(E), _dp(F)), ctx.handle)
    return float(E[0]), F


_NP_STORE = {BTE_STORE_F32: np.float32, BTE_STORE_F16: np.float16, BTE_STORE_BF16: np.uint16}


def bte_get_state(ctx, out=None, ref=None):
    """The stored state: numpy (float32, float16, or uint16 holding bfloat16 bits) by default,
    or into ``out`` (numpy or CUDA tensor) of state_bytes bytes.  With 16-bit storage the codes
    are departures from the reference field R: e = s_k (h + R / T_scale); ``ref`` (float32,
    ncell values, same memory space as ``out``) receives R when given."""
    i = ctx.info
    if out is None:
        out = np.empty(ctx.shape, dtype=_NP_STORE[i.storage])
    p, dev = _ptr(out)
    rp = _ptr(ref)[0] if ref is not None else None
    _check(load().bte_get_state(ctx.handle, p, i.state_bytes, rp, dev), ctx.handle)
    return out


def bte_set_state(ctx, src, ref=None, keep_step=False):
    """Load a state in the storage format; ``ref`` is the code reference R of 16-bit codes
    (None: R = 0, so a 16-bit state is e = s_k h)."""
    i = ctx.info
    if not hasattr(src, "data_ptr"):
        src = np.ascontiguousarray(src, dtype=_NP_STORE[i.storage])
    p, dev = _ptr(src)
    if ref is not None and not hasattr(ref, "data_ptr"):
        ref = np.ascontiguousarray(ref, dtype=np.float32)
    rp = _ptr(ref)[0] if ref is not None else None
    _check(load().bte_set_state(ctx.handle, p, i.state_bytes, rp, dev, int(bool(keep_step))), ctx.handle)


def bte_get_values(ctx, out=None):
    """The decoded state e as float32 (numpy of the state's shape, or into a CUDA tensor)."""
    if out is None:
        out = np.empty(ctx.shape, dtype=np.float32)
    p, dev = _ptr(out)
    _check(load().bte_get_values(ctx.handle, p, dev), ctx.handle)
    return out


def bte_adjoint(ctx, nsteps, probe, ckpt_every=0):
    """J = sum_i probe_i T_L,i after nsteps steps from the current state and its gradients:
    returns (J, dJ/dQ shaped (nz, ny, nx), dJ/dlog tau_k).  The context advances nsteps."""
    i = ctx.info
    probe = np.ascontiguousarray(probe, dtype=np.float64).reshape(-1)
    assert probe.size == i.ncell
    J = np.zeros(1)
    gQ = np.zeros(i.ncell)
    gt = np.zeros(i.nbands)
    _check(load().bte_adjoint(ctx.handle, int(nsteps), int(ckpt_every), _dp(probe), _dp(J), _dp(gQ), _dp(gt)),
           ctx.handle)
    return float(J[0]), gQ.reshape(i.nz, i.ny, i.nx), gt


def bte_adjoint_profile_read(ctx):
    """(adjoint-step ms, adjoint steps, forward ms, forward steps) of the last traced bte_adjoint."""
    a = np.zeros(1)
    f = np.zeros(1)
    na = ct.c_longlong()
    nf = ct.c_longlong()
    _check(load().bte_adjoint_profile_read(ctx.handle, _dp(a), ct.byref(na), _dp(f), ct.byref(nf)), ctx.handle)
    return float(a[0]), na.value, float(f[0]), nf.value


def bte_get_info(ctx):
    info = bte_info()
    _check(load().bte_get_info(ctx.handle, ct.byref(info)), ctx.handle)
    return info


def bte_get_quadrature(ctx):
    nd = ctx.info.ndirs
    s = np.empty(3 * nd)
    w = np.empty(nd)
    _check(load().bte_get_quadrature(ctx.handle, _dp(s), _dp(w)), ctx.handle)
    return s.reshape(nd, 3), w


def bte_profile(ctx, enable=True):
    _check(load().bte_profile(ctx.handle, int(bool(enable))), ctx.handle)


def bte_profile_read(ctx):
    """(forward ms, forward launches, finalize ms, finalize launches) since bte_profile(ctx, 1)."""
    f, g = ct.c_double(), ct.c_double()
    nf, ng = ct.c_longlong(), ct.c_longlong()
    _check(load().bte_profile_read(ctx.handle, ct.byref(f), ct.byref(nf), ct.byref(g), ct.byref(ng)), ctx.handle)
    return f.value, nf.value, g.value, ng.value
