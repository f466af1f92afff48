"""Mirror maps of the product rule for equivariance pins: the points of the rule (Sec. 3.2,
equally spaced azimuths, an even number of them) map onto each other when Omega_x (axis 0) or
Omega_y (axis 1) is negated; the map is found from the rule's own direction tables, so it does
not depend on where the azimuth is measured from."""
import numpy as np


def mirror_points(ox, oy, mu, axis):
    """perm[q] = the point whose direction is point q's with Omega_x (axis 0) or Omega_y negated."""
    sx, sy = (-1.0, 1.0) if axis == 0 else (1.0, -1.0)
    key = {(round(a, 12), round(b, 12), round(c, 12)): i for i, (a, b, c) in enumerate(zip(ox, oy, mu))}
    return np.array([key[(round(sx * a, 12) + 0.0, round(sy * b, 12) + 0.0, round(c, 12))]
                     for a, b, c in zip(ox, oy, mu)])


def mirror_basis(M, perm):
    """The orthogonal D with m(mirrored direction) = D m(direction) on the basis table M [Q x n]."""
    D = np.linalg.lstsq(M, M[perm], rcond=None)[0].T
    assert np.abs(M @ D.T - M[perm]).max() < 1e-12
    assert np.abs(D @ D.T - np.eye(M.shape[1])).max() < 1e-12
    return D


def mirror_xy(xy, axis):
    return xy * (np.array([-1.0, 1.0]) if axis == 0 else np.array([1.0, -1.0]))
