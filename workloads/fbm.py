"""Seeded fractional Brownian motion (value noise) for synthetic terrain.

Octave ``k`` is lattice value noise at frequency ``2**k / wavelength`` with
amplitude ``2**(-hurst*k)``; the octave sum is normalised to [-1, 1] and
mapped to heights in ``[0, amplitude]``.  Lattice values come from an integer
hash of (lattice x, lattice y, seed, octave), so any point can be evaluated
independently and the field is identical on every machine up to the rounding
of a few multiplies.  Interpolation is bilinear with a quintic fade, which
keeps the field C2 so that its Laplacian (used by the curvature-refined
quadtree) is well defined.
"""

from __future__ import annotations

import numpy as np

_M1 = np.uint64(0x9E3779B97F4A7C15)
_M2 = np.uint64(0xC2B2AE3D27D4EB4F)
_M3 = np.uint64(0x165667B19E3779F9)
_F1 = np.uint64(0xFF51AFD7ED558CCD)
_F2 = np.uint64(0xC4CEB9FE1A85EC53)
_S33 = np.uint64(33)
_S11 = np.uint64(11)


def _hash01(ix: np.ndarray, iy: np.ndarray, salt: int) -> np.ndarray:
    """Hash integer lattice coordinates to uniform values in [-1, 1)."""
    with np.errstate(over="ignore"):
        return _hash01_impl(ix, iy, salt)


def _hash01_impl(ix, iy, salt: int) -> np.ndarray:
    ix, iy = np.broadcast_arrays(np.asarray(ix, dtype=np.int64),
                                 np.asarray(iy, dtype=np.int64))
    x = ix.astype(np.uint64) * _M1
    x ^= iy.astype(np.uint64) * _M2
    x ^= np.uint64(salt & 0xFFFFFFFF) * _M3
    x ^= x >> _S33
    x *= _F1
    x ^= x >> _S33
    x *= _F2
    x ^= x >> _S33
    return (x >> _S11).astype(np.float64) * (2.0 / 9007199254740992.0) - 1.0


def _fade(t: np.ndarray) -> np.ndarray:
    return t * t * t * (t * (t * 6.0 - 15.0) + 10.0)


class FBm:
    """Seeded fBm height field ``h(x, y)`` in metres, ``0 <= h <= amplitude``."""

    def __init__(self, seed: int, amplitude: float, wavelength: float,
                 octaves: int = 6, hurst: float = 0.8):
        self.seed = int(seed)
        self.amplitude = float(amplitude)
        self.wavelength = float(wavelength)
        self.octaves = int(octaves)
        self.hurst = float(hurst)
        amps = np.array([2.0 ** (-self.hurst * k) for k in range(self.octaves)])
        self._amps = amps / amps.sum()

    def _salt(self, k: int) -> int:
        return self.seed * 1000003 + k * 7919

    def __call__(self, x, y) -> np.ndarray:
        """Evaluate at arbitrary points (broadcast arrays, metres)."""
        x = np.asarray(x, dtype=np.float64)
        y = np.asarray(y, dtype=np.float64)
        x, y = np.broadcast_arrays(x, y)
        acc = np.zeros(x.shape, dtype=np.float64)
        for k in range(self.octaves):
            f = (2.0 ** k) / self.wavelength
            u, v = x * f, y * f
            iu, iv = np.floor(u), np.floor(v)
            su, sv = _fade(u - iu), _fade(v - iv)
            iu = iu.astype(np.int64)
            iv = iv.astype(np.int64)
            s = self._salt(k)
            n00 = _hash01(iu, iv, s)
            n10 = _hash01(iu + 1, iv, s)
            n01 = _hash01(iu, iv + 1, s)
            n11 = _hash01(iu + 1, iv + 1, s)
            n0 = n00 + (n10 - n00) * su
            n1 = n01 + (n11 - n01) * su
            acc += self._amps[k] * (n0 + (n1 - n0) * sv)
        return 0.5 * self.amplitude * (acc + 1.0)

    def _weights(self, coords: np.ndarray, f: float):
        """Sparse-as-dense interpolation matrix for one axis of a regular grid."""
        u = coords * f
        iu = np.floor(u)
        s = _fade(u - iu)
        iu = iu.astype(np.int64)
        lo = int(iu.min())
        hi = int(iu.max()) + 1
        w = np.zeros((coords.size, hi - lo + 1), dtype=np.float64)
        r = np.arange(coords.size)
        w[r, iu - lo] += 1.0 - s
        w[r, iu - lo + 1] += s
        return w, lo, hi

    def grid(self, xs, ys) -> np.ndarray:
        """Evaluate on the tensor grid ``xs`` x ``ys``; returns ``[len(ys), len(xs)]``.

        Value noise is separable on a regular grid, so each octave is the
        matrix product ``Wy @ L @ Wx.T`` of two interpolation matrices and the
        lattice values ``L``.
        """
        xs = np.asarray(xs, dtype=np.float64)
        ys = np.asarray(ys, dtype=np.float64)
        acc = np.zeros((ys.size, xs.size), dtype=np.float64)
        for k in range(self.octaves):
            f = (2.0 ** k) / self.wavelength
            wx, x0, x1 = self._weights(xs, f)
            wy, y0, y1 = self._weights(ys, f)
            lx = np.arange(x0, x1 + 1)
            ly = np.arange(y0, y1 + 1)
            lat = _hash01(lx[None, :], ly[:, None], self._salt(k))
            acc += self._amps[k] * (wy @ lat @ wx.T)
        return 0.5 * self.amplitude * (acc + 1.0)
