"""Exact single-Fourier-mode solutions of the transient thermal grating (arXiv 2306.14181,
Sec. 4.2) for the explicit DOM step of ``bte_oracle.c``.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

A periodic 1-D problem started from T(x, 0) = A0 cos(q x) keeps the single spatial mode
e_{k,d}(x, t) = Re[ e_hat_{k,d}(t) exp(i q x) ]: every operator of the step is translation
invariant, so each mode evolves on its own.

- fully discrete, first-order face value: e_hat^{n+1} = G e_hat^n with the upwind symbol
  1 - |nu| (1 - exp(-i sg theta)), theta = q dx, the relaxation -dt/tau_k and the rank-one
  T_L coupling dt/tau_k C_k/W T_L_hat, T_L_hat = sum_{k,d} w_d e_hat/tau_k / sum_k C_k/tau_k
  (Eq. disretized_transientBTE, Eq. BTE_get_e0);
- semi-discrete (exact in space and time, discrete in angle): d e_hat/dt = M e_hat with
  M = -diag(i q v_k mu_d + 1/tau_k) + diag(1/tau_k) (C_k/W) col^T: the limit the scheme
  approaches as dx and dt go to zero.

The amplitude of the temperature mode is T_hat = sum_{k,d} w_d e_hat / sum_k C_k (Eq. getTQ).
"""
import numpy as np


def moment_row(P):
    """col[k*nd + d] = w_d / (tau_k D): T_L_hat = col . e_hat (Eq. BTE_get_e0)."""
    D = float(np.sum(P.C / P.tau))
    return np.concatenate([P.w / P.tau[k] / D for k in range(P.nb)])


def temperature_row(P):
    """row[k*nd + d] = w_d / sum_k C_k: T_hat = row . e_hat (Eq. getTQ)."""
    return np.tile(P.w, P.nb) / float(np.sum(P.C))


def discrete_first_order_matrix(P, theta):
    """G of one step of the first-order scheme for the mode exp(i theta j) (x axis)."""
    nb, nd = P.nb, P.nd
    col = moment_row(P)
    G = np.zeros((nb * nd, nb * nd), dtype=complex)
    for k in range(nb):
        for d in range(nd):
            r = k * nd + d
            nu = P.dt * P.v[k] * P.s[d, 0] / P.dx
            sg = 1.0 if nu > 0 else -1.0
            G[r, r] += 1.0 - abs(nu) * (1.0 - np.exp(-1j * sg * theta)) - P.dt / P.tau[k]
            G[r, :] += P.dt / P.tau[k] * (P.C[k] / P.W) * col
    return G


def semidiscrete_matrix(P, q):
    """M of d e_hat / dt = M e_hat for the mode exp(i q x) (x axis)."""
    nb, nd = P.nb, P.nd
    col = moment_row(P)
    M = np.zeros((nb * nd, nb * nd), dtype=complex)
    for k in range(nb):
        for d in range(nd):
            r = k * nd + d
            M[r, r] -= 1j * q * P.v[k] * P.s[d, 0] + 1.0 / P.tau[k]
            M[r, :] += (1.0 / P.tau[k]) * (P.C[k] / P.W) * col
    return M


def equilibrium_mode(P):
    """e_hat of the equilibrium at unit temperature amplitude: C_k / W in every direction."""
    return np.repeat(P.C / P.W, P.nd).astype(complex)


def semidiscrete_amplitudes(P, q, times):
    """T_hat(t) / T_hat(0) of the semi-discrete problem from the equilibrium mode, at `times`."""
    M = semidiscrete_matrix(P, q)
    lam, V = np.linalg.eig(M)
    c = np.linalg.solve(V, equilibrium_mode(P))
    row = temperature_row(P) @ V
    return np.array([np.real(row @ (np.exp(lam * t) * c)) for t in times])


def discrete_amplitudes(P, theta, steps):
    """T_hat(n) / T_hat(0) of the fully discrete first-order scheme, n in `steps` (increasing)."""
    G = discrete_first_order_matrix(P, theta)
    a = equilibrium_mode(P)
    row = temperature_row(P)
    out, n0 = [], 0
    for n in steps:
        a = np.linalg.matrix_power(G, n - n0) @ a
        n0 = n
        out.append(np.real(row @ a))
    return np.array(out)
