"""ctypes front end of the FP64 oracle (``bte_oracle.c``).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

State layout: ``e[k][d][z][y][x]`` as a float64 array of shape (nb, nd, nz, ny, nx).
Boundary codes: 0 isothermal, 1 diffuse, 2 specular, 3 periodic; walls ordered
-x, +x, -y, +y, -z, +z.  Limiter codes: 0 first order, 1 minmod, 2 van Albada.
"""
import ctypes as ct
import math
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "bte_oracle.c")
_LIB = os.path.join(_HERE, "liboracle_bte.so")
_lock = threading.Lock()
_lib = None

BC_ISOTHERMAL, BC_DIFFUSE, BC_SPECULAR, BC_PERIODIC = 0, 1, 2, 3
LIM_FIRST_ORDER, LIM_MINMOD, LIM_VANALBADA = 0, 1, 2


def build_oracle(force=False):
    """Compile ``bte_oracle.c`` into ``liboracle_bte.so`` next to it (gcc, OpenMP)."""
    srcs = [_SRC, os.path.join(_HERE, "bte_oracle_adjoint.c")]
    srcs = [s for s in srcs if os.path.exists(s)]
    newest = max(os.path.getmtime(s) for s in srcs)
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= newest:
        return _LIB
    tmp = _LIB + ".tmp.%d" % os.getpid()
    cmd = ["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c99", "-o", tmp] + srcs + ["-lm"]
    subprocess.check_call(cmd)
    os.replace(tmp, _LIB)
    return _LIB


class _Prob(ct.Structure):
    _fields_ = [
        ("dim", ct.c_int), ("nx", ct.c_int), ("ny", ct.c_int), ("nz", ct.c_int),
        ("dx", ct.c_double), ("dy", ct.c_double), ("dz", ct.c_double),
        ("nb", ct.c_int), ("nd", ct.c_int),
        ("C", ct.POINTER(ct.c_double)), ("v", ct.POINTER(ct.c_double)), ("tau", ct.POINTER(ct.c_double)),
        ("s", ct.POINTER(ct.c_double)), ("w", ct.POINTER(ct.c_double)),
        ("mirror", ct.POINTER(ct.c_int)),
        ("bc", ct.c_int * 6), ("Tw", ct.c_double * 6),
        ("dt", ct.c_double), ("limiter", ct.c_int),
        ("jump", ct.c_double * 3),
    ]


def load_oracle():
    global _lib
    with _lock:
        if _lib is None:
            build_oracle()
            _lib = ct.CDLL(_LIB)
            dp = ct.POINTER(ct.c_double)
            fp = ct.POINTER(ct.c_float)
            pp = ct.POINTER(_Prob)
            _lib.orc_step.argtypes = [pp, dp, dp, fp, ct.c_double]
            _lib.orc_run.argtypes = [pp, dp, fp, dp, ct.c_int, ct.c_long, ct.c_int]
            _lib.orc_moments.argtypes = [pp, dp, dp, dp, dp]
            _lib.orc_lattice_temperature.argtypes = [pp, dp, dp]
            _lib.orc_energy.argtypes = [pp, dp, dp, dp]
            _lib.orc_step_points.argtypes = [pp, dp, fp, ct.c_double, ct.c_long, ct.POINTER(ct.c_long), dp]
            _lib.orc_step_tangent.argtypes = [pp, dp, dp, dp]
            _lib.orc_adjoint_step.argtypes = [pp, dp, dp, dp]
            _lib.orc_adjoint.argtypes = [pp, dp, fp, dp, ct.c_int, ct.c_long, ct.c_int, dp, dp, dp, dp, ct.c_int]
            _lib.orc_adjoint.restype = ct.c_int
            for f in (_lib.orc_interface_step, _lib.orc_interface_energy):
                f.restype = ct.c_int
            _lib.orc_interface_step.argtypes = [pp, dp, dp, fp, ct.c_double, ct.c_int, pp, dp, dp, fp, ct.c_double,
                                                ct.c_int, dp, dp]
            _lib.orc_sis_iteration.argtypes = [pp, dp, dp, fp, ct.c_double]
            _lib.orc_sis_iteration_tl.argtypes = [pp, dp, dp, dp, fp, ct.c_double]
            _lib.orc_interface_energy.argtypes = [pp, dp, ct.c_int, pp, dp, ct.c_int, dp, dp, dp, dp, dp, dp]
        return _lib


def _dp(a):
    return a.ctypes.data_as(ct.POINTER(ct.c_double))


def _fp(a):
    return None if a is None else a.ctypes.data_as(ct.POINTER(ct.c_float))


class Problem:
    """One discretised problem: grid, bands, quadrature, walls, time step and limiter."""

    def __init__(self, dim, n, h, C, v, tau, s, w, mirror, bc, Tw, dt, limiter=LIM_VANALBADA, jump=None):
        self.dim = int(dim)
        self.nx, self.ny, self.nz = (int(t) for t in n)
        self.dx, self.dy, self.dz = (float(t) for t in h)
        self.C = np.ascontiguousarray(C, dtype=np.float64)
        self.v = np.ascontiguousarray(v, dtype=np.float64)
        self.tau = np.ascontiguousarray(tau, dtype=np.float64)
        self.s = np.ascontiguousarray(s, dtype=np.float64).reshape(-1, 3)
        self.w = np.ascontiguousarray(w, dtype=np.float64)
        self.mirror = np.ascontiguousarray(mirror, dtype=np.int32).reshape(3, -1)
        self.nb, self.nd = self.C.size, self.w.size
        self.bc = [int(b) for b in bc]
        self.Tw = [float(t) for t in Tw]
        self.dt = float(dt)
        self.limiter = int(limiter)
        # temperature difference across each periodic pair (Sec. 2.2 (iv)); 0 on other axes
        self.jump = [float(t) for t in (jump if jump is not None else (0.0, 0.0, 0.0))]
        for a in range(3):
            assert self.jump[a] == 0.0 or self.bc[2 * a] == BC_PERIODIC, "a jump needs a periodic pair"
        self._lib = load_oracle()
        self._p = _Prob(self.dim, self.nx, self.ny, self.nz, self.dx, self.dy, self.dz, self.nb, self.nd,
                        _dp(self.C), _dp(self.v), _dp(self.tau), _dp(self.s), _dp(self.w),
                        self.mirror.ctypes.data_as(ct.POINTER(ct.c_int)),
                        (ct.c_int * 6)(*self.bc), (ct.c_double * 6)(*self.Tw), self.dt, self.limiter,
                        (ct.c_double * 3)(*self.jump))

    # -- sizes ---------------------------------------------------------------------------
    @property
    def shape(self):
        return (self.nb, self.nd, self.nz, self.ny, self.nx)

    @property
    def ncell(self):
        return self.nx * self.ny * self.nz

    @property
    def W(self):
        # sequential sum, the same order as the C code's total weight
        W = 0.0
        for x in self.w:
            W += float(x)
        return W

    def _src(self, Q):
        if Q is None:
            return None
        Q = np.ascontiguousarray(Q, dtype=np.float32).reshape(-1)
        assert Q.size == self.ncell
        return Q

    # -- state ---------------------------------------------------------------------------
    def equilibrium(self, dT):
        """e_{k,d,i} = C_k dT_i / W, the equilibrium energy density of Eq. (BTE_get_e0)."""
        dT = np.broadcast_to(np.asarray(dT, dtype=np.float64), (self.nz, self.ny, self.nx))
        e = self.C[:, None, None, None, None] * dT[None, None] / self.W
        return np.ascontiguousarray(np.broadcast_to(e, self.shape), dtype=np.float64)

    def step(self, e, Q=None, amp=1.0):
        e = np.ascontiguousarray(e, dtype=np.float64)
        out = np.empty_like(e)
        Qc = self._src(Q)
        self._lib.orc_step(ct.byref(self._p), _dp(e), _dp(out), _fp(Qc), float(amp))
        return out

    def run(self, e, nsteps, Q=None, amps=None, n0=0):
        """nsteps steps; amps[n] is the source amplitude at step n (None: 1; past the end: 0)."""
        e = np.array(e, dtype=np.float64, order="C", copy=True)
        Qc = self._src(Q)
        if amps is None:
            ap, na = None, 0
        else:
            amps = np.ascontiguousarray(amps, dtype=np.float64)
            ap, na = _dp(amps), amps.size
        self._lib.orc_run(ct.byref(self._p), _dp(e), _fp(Qc), ap, na, int(n0), int(nsteps))
        return e

    def lattice_temperature(self, e):
        e = np.ascontiguousarray(e, dtype=np.float64)
        TL = np.empty(self.ncell)
        self._lib.orc_lattice_temperature(ct.byref(self._p), _dp(e), _dp(TL))
        return TL.reshape(self.nz, self.ny, self.nx)

    def moments(self, e):
        """(T, T_L, q) of Eq. (getTQ) and Eq. (BTE_get_e0); q has shape (3, nz, ny, nx)."""
        e = np.ascontiguousarray(e, dtype=np.float64)
        T = np.empty(self.ncell)
        TL = np.empty(self.ncell)
        q = np.empty(3 * self.ncell)
        self._lib.orc_moments(ct.byref(self._p), _dp(e), _dp(T), _dp(TL), _dp(q))
        g = (self.nz, self.ny, self.nx)
        return T.reshape(g), TL.reshape(g), q.reshape((3,) + g)

    def energy(self, e):
        """(E_total, wall_flux[6]): the global energy and the outward wall heat flows."""
        e = np.ascontiguousarray(e, dtype=np.float64)
        E = np.zeros(1)
        F = np.zeros(6)
        self._lib.orc_energy(ct.byref(self._p), _dp(e), _dp(E), _dp(F))
        return float(E[0]), F

    def step_points(self, e, pts, Q=None, amp=1.0):
        """e^{n+1} at the given (k, d, cell) triples, from e^n."""
        e = np.ascontiguousarray(e, dtype=np.float64)
        pts = np.ascontiguousarray(pts, dtype=np.int64).reshape(-1, 3)
        out = np.empty(pts.shape[0])
        Qc = self._src(Q)
        self._lib.orc_step_points(ct.byref(self._p), _dp(e), _fp(Qc), float(amp), pts.shape[0],
                                  pts.ctypes.data_as(ct.POINTER(ct.c_long)), _dp(out))
        return out

    # -- discrete adjoint (exact transpose of the step; not in the paper) ----------------
    def step_tangent(self, e, de):
        """J(e) de: the step's derivative along de (forward mode, T_L coupling included)."""
        e = np.ascontiguousarray(e, dtype=np.float64)
        de = np.ascontiguousarray(de, dtype=np.float64)
        out = np.empty_like(e)
        self._lib.orc_step_tangent(ct.byref(self._p), _dp(e), _dp(de), _dp(out))
        return out

    def adjoint_step(self, e, lam):
        """J(e)^T lam (reverse mode)."""
        e = np.ascontiguousarray(e, dtype=np.float64)
        lam = np.ascontiguousarray(lam, dtype=np.float64)
        out = np.empty_like(e)
        self._lib.orc_adjoint_step(ct.byref(self._p), _dp(e), _dp(lam), _dp(out))
        return out

    def adjoint(self, e0, nsteps, probe, Q=None, amps=None, n0=0, ckpt=0):
        """J = sum_i probe_i T_L,i after nsteps steps from e0, with dJ/dQ (per cell; Q taken
        as 0 when None) and dJ/dlog tau_k.  ckpt > 0 keeps every ckpt-th state and recomputes
        the rest (bitwise the same result).  Returns (J, dJ_dQ, dJ_dlogtau)."""
        e0 = np.ascontiguousarray(e0, dtype=np.float64)
        probe = np.ascontiguousarray(probe, dtype=np.float64).reshape(-1)
        assert probe.size == self.ncell
        Qc = self._src(Q)
        if amps is None:
            ap, na = None, 0
        else:
            amps = np.ascontiguousarray(amps, dtype=np.float64)
            ap, na = _dp(amps), amps.size
        J = np.zeros(1)
        gQ = np.zeros(self.ncell)
        gt = np.zeros(self.nb)
        rc = self._lib.orc_adjoint(ct.byref(self._p), _dp(e0), _fp(Qc), ap, na, int(n0), int(nsteps), _dp(probe),
                                   _dp(J), _dp(gQ), _dp(gt), int(ckpt))
        if rc != 0:
            raise MemoryError("oracle adjoint: trajectory does not fit in memory")
        return float(J[0]), gQ.reshape(self.nz, self.ny, self.nx), gt

    def sis_iteration(self, e, Q=None, amp=1.0):
        """One sequential iteration of the steady implicit DOM (Sec. 3.3-3.5, Eq. disretized_BTE
        in delta form, first-order upwind on the left, the step's limited faces on the right,
        walls lagged by one iteration): e^{n+1} = e^n + De."""
        e = np.ascontiguousarray(e, dtype=np.float64)
        out = np.empty_like(e)
        self._lib.orc_sis_iteration(ct.byref(self._p), _dp(e), _dp(out), _fp(self._src(Q)), float(amp))
        return out

    def sis_iteration_tl(self, e, TL, Q=None, amp=1.0):
        """The sequential iteration with the equilibrium of a given lattice temperature TL."""
        e = np.ascontiguousarray(e, dtype=np.float64)
        TL = np.ascontiguousarray(np.broadcast_to(np.asarray(TL, dtype=np.float64), (self.nz, self.ny, self.nx)))
        out = np.empty_like(e)
        self._lib.orc_sis_iteration_tl(ct.byref(self._p), _dp(e), _dp(TL), _dp(out), _fp(self._src(Q)), float(amp))
        return out

    # -- synthetic iterative scheme (Sec. 3.5) ------------------------------------------------
    @property
    def k_bulk(self):
        """Bulk conductivity sum_k C_k v_k^2 tau_k / 3 (Sec. 3.5)."""
        return float(np.sum(self.C * self.v ** 2 * self.tau)) / 3.0

    def energy_residual(self, e, Q=None, amp=1.0):
        """r_i = sum_k sum_d w_d R_{k,d,i}: the energy the steady equation's right-hand side R
        (with e0 of T_L(e)) leaves in cell i per unit time and volume (W/m^3); R = (step(e) - e)/dt."""
        R = (self.step(e, Q, amp) - e) / self.dt
        return np.einsum("d,kdzyx->zyx", self.w, R)

    def laplacian(self):
        """The cell-centred 2*dim+1-point Laplacian (1/m^2) of a temperature correction on the
        grid, as a sparse matrix over the cells (x fastest), with the walls' conditions on the
        correction: a thermalizing wall holds the temperature (zero at the wall face: the ghost
        is minus the wall cell), reflecting walls pass no heat (the ghost equals the wall cell),
        periodic pairs wrap (the jump is in the state, not in the correction)."""
        import scipy.sparse as sp
        n = (self.nx, self.ny, self.nz)
        h = (self.dx, self.dy, self.dz)
        N = self.ncell
        rows, cols, vals = [], [], []
        for z in range(self.nz):
            for y in range(self.ny):
                for x in range(self.nx):
                    i = (z * self.ny + y) * self.nx + x
                    c = [x, y, z]
                    for a in range(self.dim):
                        w2 = 1.0 / (h[a] * h[a])
                        for side, step in ((0, -1), (1, 1)):
                            nb = list(c)
                            nb[a] += step
                            rows.append(i)
                            cols.append(i)
                            vals.append(-w2)
                            if 0 <= nb[a] < n[a]:
                                j = (nb[2] * self.ny + nb[1]) * self.nx + nb[0]
                                rows.append(i)
                                cols.append(j)
                                vals.append(w2)
                                continue
                            bc = self.bc[2 * a + side]
                            if bc == BC_PERIODIC:
                                nb[a] %= n[a]
                                j = (nb[2] * self.ny + nb[1]) * self.nx + nb[0]
                                rows.append(i)
                                cols.append(j)
                                vals.append(w2)
                            elif bc == BC_ISOTHERMAL:
                                rows.append(i)
                                cols.append(i)
                                vals.append(-w2)
                            else:
                                rows.append(i)
                                cols.append(i)
                                vals.append(w2)
        return sp.csr_matrix((vals, (rows, cols)), shape=(N, N))

    def synthetic_correction(self, r):
        """dT solving k_bulk L dT = -r (the macroscopic equation of Sec. 3.5 for the correction of
        T_L); with no thermalizing wall L is singular and dT is the mean-free least-squares
        solution of the mean-free r."""
        import scipy.sparse.linalg as spl
        if getattr(self, "_klap", None) is None:
            self._klap = (self.laplacian() * self.k_bulk).tocsc()
            self._klap_lu = (spl.splu(self._klap) if any(self.bc[w] == BC_ISOTHERMAL for w in range(2 * self.dim))
                             else None)
        L = self._klap
        b = -np.asarray(r, dtype=np.float64).reshape(-1)
        if self._klap_lu is not None:
            dT = self._klap_lu.solve(b)
        else:
            b = b - b.mean()
            dT = spl.lsqr(L, b, atol=1e-15, btol=1e-15, iter_lim=20 * self.ncell)[0]
            dT -= dT.mean()
        return dT.reshape(self.nz, self.ny, self.nx)

    def synthetic_iteration(self, e, TL, Q=None, amp=1.0):
        """One iteration of the synthetic scheme (Sec. 3.5, Steps 2-4): the sweep with e0 of TL,
        then the macroscopic equation for the lattice temperature of the next sweep.  The
        equation's right-hand side div q_nonFourier - sum Q, with the scheme's own face fluxes
        for q, is k_bulk L T_L(e) - r(e) (r: the energy residual), so the new lattice temperature
        is T_L(e) + dT with k_bulk L dT = -r(e).  Returns (e', TL')."""
        e1 = self.sis_iteration_tl(e, TL, Q, amp)
        dT = self.synthetic_correction(self.energy_residual(e1, Q, amp))
        return e1, self.lattice_temperature(e1) + dT

    def run_synthetic(self, e, max_iters, tol_T, tol_q, Q=None, Tref=300.0):
        """Synthetic iterations until the loop condition of Sec. 3.5 holds between consecutive
        states: (e, iterations, eps_T, eps_q)."""
        TL = self.lattice_temperature(e)
        eT = eq = math.inf
        n = 0
        while n < max_iters:
            e1, TL = self.synthetic_iteration(e, TL, Q)
            eT, eq = self.residuals(e, e1, Tref)
            e = e1
            n += 1
            if eT < tol_T and eq < tol_q:
                break
        return e, n, eT, eq

    def run_sis(self, e, max_iters, tol_T, tol_q, Q=None, Tref=300.0):
        """Sequential iterations until eps_T < tol_T and eps_q < tol_q between consecutive
        iterates (the loop condition of Sec. 3.5) or max_iters: (e, iterations, eps_T, eps_q)."""
        eT = eq = math.inf
        n = 0
        while n < max_iters:
            e1 = self.sis_iteration(e, Q)
            eT, eq = self.residuals(e, e1, Tref)
            e = e1
            n += 1
            if eT < tol_T and eq < tol_q:
                break
        return e, n, eT, eq

    def residuals(self, e_n, e_n1, Tref):
        """The loop condition of the transient solver (Sec. 4.1, Algorithm 2) between consecutive
        states: eps_T = sqrt(sum_i (T_i^n - T_i^{n+1})^2 / N) / T_max and eps_q the same for |q|,
        T and q of Eq. (getTQ); T_max is the largest absolute temperature Tref + T_i^{n+1} and
        |q|_max the largest |q_i^{n+1}|."""
        T0, _, q0 = self.moments(e_n)
        T1, _, q1 = self.moments(e_n1)
        N = T0.size
        qm0 = np.sqrt((q0 ** 2).sum(axis=0))
        qm1 = np.sqrt((q1 ** 2).sum(axis=0))
        num_T = math.sqrt(float(((T0 - T1) ** 2).sum()) / N)
        num_q = math.sqrt(float(((qm0 - qm1) ** 2).sum()) / N)
        Tmax = float(np.max(np.abs(Tref + T1)))
        qmax = float(np.max(qm1))
        eps_T = 0.0 if num_T == 0.0 else num_T / Tmax
        eps_q = 0.0 if num_q == 0.0 else num_q / qmax
        return eps_T, eps_q

    @property
    def cell_volume(self):
        L = [self.dx, self.dy, self.dz]
        return float(np.prod([L[a] if a < self.dim else 1.0 for a in range(3)]))


# -- interface between two materials (Sec. 2.2 (v)) -----------------------------------------
def _betas(b, nb):
    b = np.ascontiguousarray(np.broadcast_to(np.asarray(b, dtype=np.float64), (nb,)))
    assert np.all((b >= 0.0) & (b <= 1.0))
    return b


def interface_step(A, eA, wa, B, eB, wb, bAB, bBA, QA=None, QB=None, ampA=1.0, ampB=1.0):
    """One step of both materials of a diffuse-mismatch interface: wall ``wa`` of problem A
    faces wall ``wb`` of problem B (both DIFFUSE, same axis, opposite sides, same cells across);
    a band-k phonon crossing from A into B is transmitted with probability ``bAB[k]``, from B
    into A with ``bBA[k]``, and diffusely reflected otherwise.  Returns (eA', eB')."""
    eA = np.ascontiguousarray(eA, dtype=np.float64)
    eB = np.ascontiguousarray(eB, dtype=np.float64)
    oA, oB = np.empty_like(eA), np.empty_like(eB)
    bAB, bBA = _betas(bAB, A.nb), _betas(bBA, A.nb)
    rc = A._lib.orc_interface_step(ct.byref(A._p), _dp(eA), _dp(oA), _fp(A._src(QA)), float(ampA), int(wa),
                                   ct.byref(B._p), _dp(eB), _dp(oB), _fp(B._src(QB)), float(ampB), int(wb),
                                   _dp(bAB), _dp(bBA))
    if rc != 0:
        raise ValueError("walls do not form an interface")
    return oA, oB


def interface_run(A, eA, wa, B, eB, wb, bAB, bBA, nsteps, QA=None, QB=None):
    """nsteps interface steps from (eA, eB); returns the final pair."""
    for _ in range(nsteps):
        eA, eB = interface_step(A, eA, wa, B, eB, wb, bAB, bBA, QA, QB)
    return eA, eB


def interface_energy(A, eA, wa, B, eB, wb, bAB, bBA):
    """(E_A, flows_A[6], E_B, flows_B[6]): each side's energy and outward wall heat flows, the
    interface walls' flows being the heat crossing the interface."""
    eA = np.ascontiguousarray(eA, dtype=np.float64)
    eB = np.ascontiguousarray(eB, dtype=np.float64)
    bAB, bBA = _betas(bAB, A.nb), _betas(bBA, A.nb)
    EA, EB, FA, FB = np.zeros(1), np.zeros(1), np.zeros(6), np.zeros(6)
    rc = A._lib.orc_interface_energy(ct.byref(A._p), _dp(eA), int(wa), ct.byref(B._p), _dp(eB), int(wb), _dp(bAB),
                                     _dp(bBA), _dp(EA), _dp(FA), _dp(EB), _dp(FB))
    if rc != 0:
        raise ValueError("walls do not form an interface")
    return float(EA[0]), FA, float(EB[0]), FB
