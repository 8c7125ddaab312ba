"""Closed-form dense matrices used to pin the oracle (tiny grids only).

Built directly from the formulas, without any FFT and without calling the
oracle's operators:
  * periodic band-limited second derivative on n points (the spectral
    differentiation matrix of trigonometric interpolation, written as the
    periodisation of the infinite-grid sinc kernel; separate even/odd forms),
  * the truncated decomposed 1-D operator of one axis: block-diagonal periodic
    blocks plus the t x t wrap-removal (minus) and transfer (plus) corner blocks
    (Sec. 3, Eq. LV_block, Figs. 3c and 5c),
  * the 3-D operator A_t = c (sum_d I x M_d x I + diag k^2).
"""
import numpy as np


def infinite_d2(m, h):
    m = np.asarray(m, dtype=np.float64)
    out = np.where(m == 0, -np.pi ** 2 / (3 * h * h), 0.0)
    nz = m != 0
    sign = np.where(np.mod(np.abs(m), 2) == 1, -1.0, 1.0)
    out[nz] = (-2.0 * sign[nz]) / (m[nz] ** 2 * h * h)
    return out


def periodic_d2_closed(n, h):
    """n x n periodic second-derivative matrix in closed form.

    even n: D(0) = -pi^2/(3h^2) - 2 pi^2/(3 n^2 h^2),
            D(m) = -2 pi^2 (-1)^m / (n^2 h^2 sin^2(pi m/n));
    odd n:  D(0) = -pi^2/(3h^2) + pi^2/(3 n^2 h^2),
            D(m) = -2 pi^2 (-1)^m cos(pi m/n) / (n^2 h^2 sin^2(pi m/n)).
    """
    i = np.arange(n)
    m = np.mod(i[:, None] - i[None, :], n)
    out = np.empty((n, n))
    zero = m == 0
    sign = np.where(m % 2 == 1, -1.0, 1.0)
    s = np.sin(np.pi * m / n)
    if n % 2 == 0:
        out[zero] = -np.pi ** 2 / (3 * h * h) - 2 * np.pi ** 2 / (3 * n * n * h * h)
        out[~zero] = (-2 * np.pi ** 2 * sign[~zero]) / (n * n * h * h * s[~zero] ** 2)
    else:
        out[zero] = -np.pi ** 2 / (3 * h * h) + np.pi ** 2 / (3 * n * n * h * h)
        cs = np.cos(np.pi * m / n)
        out[~zero] = (-2 * np.pi ** 2 * sign[~zero] * cs[~zero]) / (n * n * h * h * s[~zero] ** 2)
    return out


def correction_block_closed(t, h):
    a = np.arange(t)[:, None]
    b = np.arange(t)[None, :]
    return infinite_d2(t + b - a, h)


def axis_matrix(sizes, t, h, a_flag, periodic):
    """Truncated decomposed second-derivative operator of one axis (N x N)."""
    N = int(sum(sizes))
    offs = np.concatenate([[0], np.cumsum(sizes)[:-1]]).astype(int)
    S = len(sizes)
    M = np.zeros((N, N))
    for o, n in zip(offs, sizes):
        M[o:o + n, o:o + n] = periodic_d2_closed(n, h)
    if a_flag == 0:
        return M
    W = correction_block_closed(t, h)
    for s, (o, n) in enumerate(zip(offs, sizes)):
        if S > 1:
            left = s - 1 if s > 0 else (S - 1 if periodic else None)
            right = s + 1 if s < S - 1 else (0 if periodic else None)
        else:
            left = right = None
        M[o + n - t:o + n, o:o + t] -= W
        M[o:o + t, o + n - t:o + n] -= W.T
        if right is not None:
            orr = offs[right]
            M[o + n - t:o + n, orr:orr + t] += W
        if left is not None:
            ol, nl = offs[left], sizes[left]
            M[o:o + t, ol + nl - t:ol + nl] += W.T
    return M


def global_sinc_axis(N, h, periodic):
    """Undecomposed operator of one axis: periodic grid, or the infinite-grid kernel
    restricted to N points (no wrap-around)."""
    if periodic:
        return periodic_d2_closed(N, h)
    i = np.arange(N)
    return infinite_d2(i[:, None] - i[None, :], h)


def kron3(M0, M1, M2):
    n0, n1, n2 = M0.shape[0], M1.shape[0], M2.shape[0]
    return (np.kron(np.kron(M0, np.eye(n1)), np.eye(n2))
            + np.kron(np.kron(np.eye(n0), M1), np.eye(n2))
            + np.kron(np.kron(np.eye(n0), np.eye(n1)), M2))


def dense_A_truncated(shape, sizes, t, h, a_flags, periodic, k2, c):
    Ms = [axis_matrix(sizes[d], t, h, a_flags[d], periodic[d]) for d in range(3)]
    return c * (kron3(*Ms) + np.diag(np.asarray(k2).ravel()))


def dense_L(shape, sizes, h, k0sq, c):
    Ms = [axis_matrix(sizes[d], 0, h, 0, False) for d in range(3)]
    n = int(np.prod(shape))
    return c * (kron3(*Ms) + k0sq * np.eye(n))


def dense_A_global(shape, h, periodic, k2, c):
    Ms = [global_sinc_axis(shape[d], h, periodic[d]) for d in range(3)]
    return c * (kron3(*Ms) + np.diag(np.asarray(k2).ravel()))
