"""FP64 CPU oracle for the domain-decomposed modified Born series (MBS).

TEST INFRASTRUCTURE ONLY. Only the test suite, the package smoke check and the
CPU-baseline leg of the benchmark may import this module; the product path
never calls it and has no CPU fallback.

Plain, slow, written to be checked by eye against the paper (Mache & Vellekoop,
"Domain decomposition of the modified Born series approach for large-scale wave
propagation simulations"). Every quantity is complex128 / float64. The FFT is
this module's own (recursive mixed-radix Cooley-Tukey, direct sum for prime
lengths); numpy is used for array storage, elementwise arithmetic and small
matrix products only.

Grid conventions: arrays have shape (N0, N1, N2) in C order, axis 0 is the
slowest axis (the paper's x, the axis split in its large run, Sec. 4.3).

Readings where the paper is silent (each is also listed in the design notes):
  R1  k0^2 is the centre of the bounding box of {k^2(r)} in the complex plane.
  R2  ||A12|| in Eq. c_scale2 is the spectral norm of the unscaled t x t block W.
  R3  The off-diagonal blocks are built from the exact band-limited (sinc)
      second-derivative kernel of the infinite grid (Sec. 3, Fig. 4).
  R4  Truncation keeps only the t x t corner blocks (nearest images / neighbours).
  R5  x0 = 0; the residual of iteration n is taken before its update; the
      relative residual is ||r_n|| / ||r_0|| (Sec. 3.1).
  R6  Stop after the update in which eps_n < tol (strict).
  R8  Absorbing layers lie inside the grid: on each non-zero face width w the
      imaginary part of the index ramps linearly, adding kappa*(w - i)/w at
      depth i = 0..w-1 from the face; where faces meet the largest ramp applies
      (so corners do not raise ||k^2 - k0^2||_inf and with it the iteration
      count, Eq. c_scale).
  R9  A periodic, split axis transfers across the global seam (a_d = 2).
  R14 If the denominator of Eq. c_scale2 is zero, it is replaced by 0.05*max|k^2|.
Parity unpinned: none of the functions below (all are pinned by the tests).
"""
from __future__ import annotations

import math

import numpy as np

# ---------------------------------------------------------------------------
# Fourier transform (used for L as a fast convolution, Sec. 2, Eq. L-convolution)
# ---------------------------------------------------------------------------


def _smallest_prime_factor(n: int) -> int:
    p = 2
    while p * p <= n:
        if n % p == 0:
            return p
        p += 1
    return n


def dft_direct(x: np.ndarray, axis: int, sign: int) -> np.ndarray:
    """Direct O(N^2) DFT along ``axis``: X[q] = sum_m x[m] exp(sign*2*pi*i*m*q/N)."""
    n = x.shape[axis]
    m = np.arange(n)
    mat = np.exp(sign * 2j * np.pi * np.outer(m, m) / n)  # [m, q]
    xm = np.moveaxis(x, axis, -1)
    return np.moveaxis(xm @ mat, -1, axis)


def fft_axis(x: np.ndarray, axis: int, sign: int = -1) -> np.ndarray:
    """Unnormalised DFT along one axis by recursive decimation in time.

    With N = M*p (p the smallest prime factor): X[k + M q] =
    sum_r W_p^{rq} W_N^{rk} Y_r[k], where Y_r is the length-M DFT of x[p m + r].
    sign=-1 is the forward transform, sign=+1 the unnormalised inverse.
    """
    x = np.asarray(x, dtype=np.complex128)
    n = x.shape[axis]
    if n == 1:
        return x.copy()
    p = _smallest_prime_factor(n)
    if p == n:
        return dft_direct(x, axis, sign)
    m = n // p
    xm = np.moveaxis(x, axis, -1)
    sub = xm.reshape(xm.shape[:-1] + (m, p))          # sub[..., j, r] = x[p*j + r]
    y = fft_axis(sub, -2, sign)                        # y[..., k, r]
    k = np.arange(m)
    r = np.arange(p)
    y = y * np.exp(sign * 2j * np.pi * np.outer(k, r) / n)
    wp = np.exp(sign * 2j * np.pi * np.outer(r, r) / p)  # [r, q]
    z = y @ wp                                          # z[..., k, q] = X[k + m q]
    out = np.swapaxes(z, -1, -2).reshape(xm.shape)
    return np.moveaxis(out, -1, axis)


def fftn3(x: np.ndarray, sign: int = -1) -> np.ndarray:
    """Unnormalised 3-D DFT (forward for sign=-1)."""
    for ax in range(3):
        x = fft_axis(x, ax, sign)
    return x


def ifftn3(x: np.ndarray) -> np.ndarray:
    """Normalised inverse 3-D DFT (1/prod(n))."""
    return fftn3(x, +1) / float(np.prod(x.shape))


# ---------------------------------------------------------------------------
# Kernels of the Laplacian (Sec. 3, Fig. 4 and Eq. L-convolution)
# ---------------------------------------------------------------------------


def sinc_d2(m, h: float):
    """Band-limited second-derivative kernel on the infinite grid at distance m.

    D(0) = -pi^2/(3 h^2), D(m) = -2 (-1)^m / (m^2 h^2): the point response of the
    angular-spectrum Laplacian F^-1(-p^2)F when the grid is unbounded (Fig. 4a).
    """
    m = np.asarray(m, dtype=np.float64)
    out = np.empty_like(m)
    zero = m == 0
    out[zero] = -np.pi ** 2 / (3.0 * h * h)
    mm = m[~zero]
    out[~zero] = -2.0 * np.where(np.mod(np.abs(mm), 2) == 1, -1.0, 1.0) / (mm * mm * h * h)
    return out


def correction_block(t: int, h: float) -> np.ndarray:
    """Truncated t x t block W with W[a, b] = D(t + b - a) (distances 1 .. 2t-1).

    Row a is the a-th of the last t voxels of a subdomain, column b the b-th of
    the first t voxels of the next subdomain along the axis (Sec. 3, Figs. 4c, 5).
    """
    a = np.arange(t)[:, None]
    b = np.arange(t)[None, :]
    return sinc_d2(t + b - a, h)


def block_norm(w: np.ndarray) -> float:
    """Spectral norm (largest singular value) of W, as used in Eq. c_scale2."""
    if w.size == 0:
        return 0.0
    return float(np.linalg.svd(w, compute_uv=False)[0])


def frequencies_squared(n: int, h: float) -> np.ndarray:
    """|p|^2 along one axis of a subdomain of n voxels, in FFT order.

    p = 2 pi q / (n h) with q = k for 2k < n and q = k - n otherwise.
    """
    k = np.arange(n)
    q = np.where(2 * k < n, k, k - n).astype(np.float64)
    p = 2.0 * np.pi * q / (n * h)
    return p * p


# ---------------------------------------------------------------------------
# Problem set-up (Sec. 2, Eqs. helmholtz, LV, c_scale; Sec. 3.1, Eq. c_scale2)
# ---------------------------------------------------------------------------


def split_sizes(total: int, parts: int, explicit=None):
    """Subdomain sizes along an axis: near-equal, the first (total mod parts) one larger."""
    if explicit is not None:
        sizes = [int(v) for v in explicit]
        if len(sizes) != parts or sum(sizes) != total or min(sizes) < 1:
            raise ValueError("explicit subdomain sizes do not tile the axis")
        return sizes
    base, extra = divmod(total, parts)
    return [base + (1 if i < extra else 0) for i in range(parts)]


def absorbing_index(n: np.ndarray, widths, kappa: float) -> np.ndarray:
    """Refractive index with linear imaginary ramps on the boundary faces (reading R8).

    On a face of width w the ramp is (w - i)/w at depth i = 0..w-1 from the face;
    where layers of several faces meet, the largest ramp applies.
    """
    out = np.array(n, dtype=np.complex128)
    ramp3 = np.zeros(out.shape)
    for d in range(3):
        size = out.shape[d]
        ramp = np.zeros(size)
        lo, hi = widths[d]
        for i in range(min(lo, size)):
            ramp[i] = max(ramp[i], (lo - i) / lo)
        for i in range(min(hi, size)):
            ramp[size - 1 - i] = max(ramp[size - 1 - i], (hi - i) / hi)
        shape = [1, 1, 1]
        shape[d] = size
        ramp3 = np.maximum(ramp3, ramp.reshape(shape))
    return out + 1j * kappa * ramp3


def axis_flags(split, periodic):
    """a_d of Eq. c_scale2: 0 periodic and unsplit, 1 non-periodic unsplit, 2 split."""
    return [0 if (s == 1 and p) else (1 if s == 1 else 2) for s, p in zip(split, periodic)]


class Problem:
    """All derived quantities of one discretised problem, in float64/complex128."""

    def __init__(self, n, pixel, wavelength, widths=((0, 0),) * 3, split=(1, 1, 1),
                 periodic=(False, False, False), t=8, alpha=0.75, kappa=0.5,
                 split_sizes_=None):
        n = np.asarray(n)
        self.shape = tuple(int(s) for s in n.shape)
        assert len(self.shape) == 3
        self.h = float(pixel)
        self.wavelength = float(wavelength)
        self.split = tuple(int(s) for s in split)
        self.periodic = tuple(bool(p) for p in periodic)
        self.t = int(t)
        self.alpha = float(alpha)
        self.sizes = [split_sizes(self.shape[d], self.split[d],
                                  None if split_sizes_ is None else split_sizes_[d]) for d in range(3)]
        self.offsets = [list(np.concatenate([[0], np.cumsum(s)[:-1]]).astype(int)) for s in self.sizes]
        self.a = axis_flags(self.split, self.periodic)
        for d in range(3):
            if self.a[d] > 0 and min(self.sizes[d]) < self.t:
                raise ValueError("truncation t exceeds a subdomain size")
        # Eq. helmholtz: k(r) = 2 pi n(r) / lambda.
        self.n_eff = absorbing_index(n, widths, kappa)
        self.k2 = (2.0 * np.pi * self.n_eff / self.wavelength) ** 2
        # Reading R1: centre of the bounding box of k^2 in the complex plane.
        re, im = self.k2.real, self.k2.imag
        self.k0sq = complex(0.5 * (re.min() + re.max()), 0.5 * (im.min() + im.max()))
        self.contrast = float(np.abs(self.k2 - self.k0sq).max())
        self.W = correction_block(self.t, self.h)
        self.Wnorm = block_norm(self.W)
        denom = self.contrast + sum(self.a) * self.Wnorm
        if denom == 0.0:
            denom = 0.05 * float(np.abs(self.k2).max())  # reading R14
        # Eq. c_scale2 (reduces to Eq. c_scale when all a_d = 0).
        self.c = -0.95j / denom
        # Sec. 2: V = c(k^2 - k0^2); the medium factor of Eq. wavesim_iter is I - V.
        self.B = 1.0 - self.c * (self.k2 - self.k0sq)
        self.cW = self.c * self.W

    # -- subdomain helpers ---------------------------------------------------
    def boxes(self):
        """Yield (slices, sizes) of every subdomain (Sec. 3, block decomposition)."""
        for j0, (o0, n0) in enumerate(zip(self.offsets[0], self.sizes[0])):
            for j1, (o1, n1) in enumerate(zip(self.offsets[1], self.sizes[1])):
                for j2, (o2, n2) in enumerate(zip(self.offsets[2], self.sizes[2])):
                    yield (slice(o0, o0 + n0), slice(o1, o1 + n1), slice(o2, o2 + n2)), (n0, n1, n2)

    def neighbours(self, d, s):
        """Left and right neighbour index of subdomain s along axis d (None if none)."""
        S = self.split[d]
        if S == 1:
            return None, None
        left = s - 1 if s > 0 else (S - 1 if self.periodic[d] else None)
        right = s + 1 if s < S - 1 else (0 if self.periodic[d] else None)
        return left, right

    # -- operators ------------------------------------------------------------
    def apply_E(self, v: np.ndarray) -> np.ndarray:
        """Edge corrections E v, the off-diagonal part of V (Sec. 3.1, steps 1-5).

        For each axis d with a_d >= 1, each subdomain s and every pencil along d:
          P_s = c W  v_s[first t],   Q_s = c W^T v_s[last t]        (step 1)
          (E v)_s[last t]  += -P_s (wrap removal, step 4) + P_right(s) (step 5)
          (E v)_s[first t] += -Q_s (wrap removal, step 4) + Q_left(s)  (step 5)
        Contributions of different axes add (the Laplacian is a sum over axes).
        """
        v = np.asarray(v, dtype=np.complex128)
        out = np.zeros_like(v)
        t = self.t
        for d in range(3):
            if self.a[d] == 0:
                continue
            vm = np.moveaxis(v, d, 0)
            om = np.moveaxis(out, d, 0)
            S = self.split[d]
            P, Q = [], []
            for s in range(S):
                o, n = self.offsets[d][s], self.sizes[d][s]
                P.append(np.tensordot(self.cW, vm[o:o + t], axes=(1, 0)))
                Q.append(np.tensordot(self.cW.T, vm[o + n - t:o + n], axes=(1, 0)))
            for s in range(S):
                o, n = self.offsets[d][s], self.sizes[d][s]
                left, right = self.neighbours(d, s)
                om[o + n - t:o + n] -= P[s]
                om[o:o + t] -= Q[s]
                if right is not None:
                    om[o + n - t:o + n] += P[right]
                if left is not None:
                    om[o:o + t] += Q[left]
        return out

    def apply_V(self, v):
        """V v = c(k^2 - k0^2) v + E v (Sec. 3, Eq. LV_block)."""
        v = np.asarray(v, dtype=np.complex128)
        return self.c * (self.k2 - self.k0sq) * v + self.apply_E(v)

    def _per_subdomain(self, v, symbol):
        out = np.empty(v.shape, dtype=np.complex128)
        for sl, (n0, n1, n2) in self.boxes():
            p2 = (frequencies_squared(n0, self.h)[:, None, None]
                  + frequencies_squared(n1, self.h)[None, :, None]
                  + frequencies_squared(n2, self.h)[None, None, :])
            out[sl] = ifftn3(symbol(p2) * fftn3(v[sl]))
        return out

    def apply_L(self, v):
        """L v = c F^-1(k0^2 - |p|^2) F v on every subdomain (Eq. L-convolution, Sec. 3.1)."""
        v = np.asarray(v, dtype=np.complex128)
        return self._per_subdomain(v, lambda p2: self.c * (self.k0sq - p2))

    def propagate(self, v):
        """(L + I)^-1 v = F^-1 [1 / (c(k0^2 - |p|^2) + 1)] F v per subdomain (Sec. 2, Sec. 3.1)."""
        v = np.asarray(v, dtype=np.complex128)
        return self._per_subdomain(v, lambda p2: 1.0 / (self.c * (self.k0sq - p2) + 1.0))

    def apply_A(self, v):
        """A v = (L + V) v: the decomposed, truncated operator c(laplacian + k^2) (Eq. LV_block)."""
        return self.apply_L(v) + self.apply_V(v)

    def one_minus_V(self, v):
        """(I - V) v = B v - E v."""
        v = np.asarray(v, dtype=np.complex128)
        return self.B * v - self.apply_E(v)

    def preconditioned_residual(self, x, y):
        """Gamma^-1 (y - A x) with Gamma^-1 = (I - V)(L + I)^-1 (Sec. 2, Eq. richardson)."""
        x = np.asarray(x, dtype=np.complex128)
        y = np.asarray(y, dtype=np.complex128)
        return self.one_minus_V(self.propagate(y - self.apply_A(x)))

    def scaled_source(self, source):
        """y = -c S (Sec. 2, Eq. LV)."""
        return -self.c * np.asarray(source, dtype=np.complex128)

    # -- the iteration ---------------------------------------------------------
    def iteration(self, x, y):
        """One MBS step in the form of Eq. wavesim_iter.

        u = (I - V) x + y;  w = (L + I)^-1 u;  r = (I - V)(w - x) = Gamma^-1 (y - A x);
        returns (x + alpha r, ||r||_2^2).
        """
        u = self.one_minus_V(x) + y
        w = self.propagate(u)
        r = self.one_minus_V(w - x)
        return x + self.alpha * r, float(np.vdot(r, r).real)

    def solve(self, source, tol=1e-6, max_iter=10000, x0=None, callback=None):
        """Richardson iteration until eps_n = ||r_n||/||r_0|| < tol (Sec. 3.1, readings R5, R6).

        Returns (x, iterations, history of eps_n).
        """
        y = self.scaled_source(source)
        x = np.zeros(self.shape, dtype=np.complex128) if x0 is None else np.array(x0, dtype=np.complex128)
        history = []
        r0 = None
        for it in range(max_iter):
            x, rr = self.iteration(x, y)
            if r0 is None:
                r0 = rr
            eps = 0.0 if r0 == 0.0 else math.sqrt(rr / r0)
            history.append(eps)
            if callback is not None:
                callback(it, x, eps)
            if eps < tol:
                return x, it + 1, history
        return x, max_iter, history


def relative_l2(a, b) -> float:
    """||a - b||_2 / ||b||_2 (unsquared)."""
    a = np.asarray(a, dtype=np.complex128)
    b = np.asarray(b, dtype=np.complex128)
    nb = np.linalg.norm(b.ravel())
    return float(np.linalg.norm((a - b).ravel()) / (nb if nb > 0 else 1.0))
