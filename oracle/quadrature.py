"""Directional discretisation for the oracle (arXiv 2306.14181, Sec. 3.2, Eq. directiondis).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

The paper samples the first octant with Gauss-Legendre nodes in the polar and the
azimuthal angle, weights each direction by ``w_theta * w_phi * sin(theta)`` and mirrors the
octant into all eight, giving ``N = 8 * Ntheta * Nphi`` directions.  The polar rule here is
Gauss-Legendre in ``mu = cos(theta)`` on [0, 1]; with ``dmu = sin(theta) dtheta`` the weight
``w_mu * w_phi`` is the same product the paper writes, and the angular integrals of
polynomials in ``s`` up to the rule's degree become exact (sum w = 4 pi,
sum w s s^T = 4 pi / 3 I).  ``paper_theta_rule`` keeps the literal reading (Gauss-Legendre in
theta with the ``sin(theta)`` factor) for comparison; it meets those identities only to
quadrature error.

For one-dimensional geometries the rule is Gauss-Legendre in ``mu`` on [-1, 1] with
``s = (mu, 0, 0)`` and ``w = 2 pi w_mu``.

Direction order (both rules): octant-major, ``d = octant * (Ntheta * Nphi) + j * Nphi + l``,
octant bit a set means component a is negative.  ``mirror[a][d]`` is the index of the
direction whose component a is negated (the specular partner across a wall normal to a).
"""
import numpy as np


def gauss_legendre(n, lo, hi):
    """Gauss-Legendre nodes and weights on [lo, hi] (numpy's rule, affinely mapped)."""
    x, w = np.polynomial.legendre.leggauss(n)
    half = 0.5 * (hi - lo)
    return lo + half * (x + 1.0), half * w


def _mirror_table(s):
    nd = s.shape[0]
    mirror = np.zeros((3, nd), dtype=np.int32)
    for a in range(3):
        for d in range(nd):
            t = s[d].copy()
            t[a] = -t[a]
            dist = np.abs(s - t).max(axis=1)
            j = int(np.argmin(dist))
            if dist[j] > 1e-12:
                raise ValueError("quadrature is not mirror symmetric")
            mirror[a, d] = j
    return mirror


def polar_1d(n_mu):
    """1-D rule: Gauss-Legendre in mu on [-1, 1], s = (mu, 0, 0), w = 2 pi w_mu."""
    mu, wmu = gauss_legendre(n_mu, -1.0, 1.0)
    # make the node set exactly symmetric (mu_j = -mu_{n-1-j})
    mu = 0.5 * (mu - mu[::-1])
    wmu = 0.5 * (wmu + wmu[::-1])
    s = np.zeros((n_mu, 3))
    s[:, 0] = mu
    w = 2.0 * np.pi * wmu
    return s, w, _mirror_table(s)


def octant_rule(ntheta, nphi, paper_theta_rule=False):
    """3-D rule of Sec. 3.2: octant product rule mirrored into eight octants."""
    if paper_theta_rule:
        th, wth = gauss_legendre(ntheta, 0.0, 0.5 * np.pi)
        mu = np.cos(th)
        sin_t = np.sin(th)
        wpol = wth * sin_t
    else:
        mu, wpol = gauss_legendre(ntheta, 0.0, 1.0)
        sin_t = np.sqrt(1.0 - mu * mu)
    phi, wphi = gauss_legendre(nphi, 0.0, 0.5 * np.pi)
    per = ntheta * nphi
    s = np.zeros((8 * per, 3))
    w = np.zeros(8 * per)
    for o in range(8):
        sg = np.array([-1.0 if (o >> a) & 1 else 1.0 for a in range(3)])
        for j in range(ntheta):
            for l in range(nphi):
                d = o * per + j * nphi + l
                s[d] = sg * np.array([sin_t[j] * np.cos(phi[l]), sin_t[j] * np.sin(phi[l]), mu[j]])
                w[d] = wpol[j] * wphi[l]
    return s, w, _mirror_table(s)
