"""Pins for the oracle's smoothing kernels (Sec. 2.3 names cubic spline and
Wendland C2/C4/C6; W(r,h) = w(r/h)/h^3 with support radius h)."""
import math

import numpy as np
import pytest
from scipy.integrate import quad

import oracle

KERNELS = ["wc2", "wc4", "wc6", "m4"]


def _w(k, q):
    return float(oracle.kernel_eval(k, np.array([q]))[0][0])


def _dw(k, q):
    return float(oracle.kernel_eval(k, np.array([q]))[1][0])


@pytest.mark.parametrize("k", KERNELS)
def test_normalised_in_3d(k):
    # int W dV = 4 pi int_0^1 q^2 w(q) dq must be exactly 1 (kernel interpolation,
    # Sec. 2.3, reproduces a constant field).
    val, err = quad(lambda q: 4.0 * math.pi * q * q * _w(k, q), 0.0, 1.0,
                    points=[0.5], epsabs=1e-14, epsrel=1e-13, limit=200)
    assert abs(val - 1.0) < 1e-11


@pytest.mark.parametrize("k", KERNELS)
def test_derivative_matches_finite_difference(k):
    q = np.linspace(0.01, 0.99, 97)
    q = q[np.abs(q - 0.5) > 1e-3]  # the cubic spline's second derivative jumps at 1/2
    eps = 1e-6
    wp, _ = oracle.kernel_eval(k, q + eps)
    wm, _ = oracle.kernel_eval(k, q - eps)
    _, dw = oracle.kernel_eval(k, q)
    fd = (wp - wm) / (2 * eps)
    assert np.max(np.abs(fd - dw)) < 1e-6 * max(1.0, np.max(np.abs(dw)))


@pytest.mark.parametrize("k", KERNELS)
def test_compact_support_and_shape(k):
    q = np.linspace(0.0, 1.5, 301)
    w, dw = oracle.kernel_eval(k, q)
    assert np.all(w[q >= 1.0] == 0.0) and np.all(dw[q >= 1.0] == 0.0)
    # positive, monotonically decreasing inside the support, smooth at the edge
    assert np.all(w[q < 1.0] > 0.0)
    assert np.all(dw[(q > 0.0) & (q < 1.0)] < 0.0)
    assert _w(k, 1.0 - 1e-6) < 1e-9 and abs(_dw(k, 1.0 - 1e-6)) < 1e-5
    assert _dw(k, 0.0) == 0.0


@pytest.mark.parametrize("k", KERNELS)
def test_dW_dh_matches_finite_difference(k):
    # dW/dh = -(3 w + q w') / h^4, checked against W(r, h +- eps)
    r, h, eps = 0.37, 0.8, 1e-6

    def W(hh):
        return _w(k, r / hh) / hh ** 3

    fd = (W(h + eps) - W(h - eps)) / (2 * eps)
    q = r / h
    an = -(3 * _w(k, q) + q * _dw(k, q)) / h ** 4
    assert abs(fd - an) < 1e-7 * abs(an)
