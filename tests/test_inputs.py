"""Pins for the synthetic input generator (not the tracking method).

* the head solve reproduces the series-resistance closed form in 1-D;
* generated fields conserve volume per cell (cfg1 to 1e-12 m^3/s);
* the FFT Gaussian field has zero mean, unit variance and the exponential
  correlation e^{-1} at a lag of one correlation length.
"""
import math

import numpy as np
import pytest

from paper_2302_13590_gb300 import inputs as I


def test_head_solve_series_resistance():
    rng = np.random.default_rng(2)
    ncol = 12
    delr = rng.uniform(0.5, 2.0, ncol)
    K = rng.uniform(1e-5, 1e-3, ncol)
    ib = np.ones((1, 1, ncol), np.int8)
    ib[0, 0, 0] = ib[0, 0, -1] = -1
    head = np.zeros((1, 1, ncol))
    head[0, 0, 0], head[0, 0, -1] = 7.0, 2.0
    area = 1.3 * 0.7
    h, qx, qy, qz, it, res = I.solve_flow(1, 1, ncol, delr, np.array([1.3]), np.array([0.7]), K, ib, head,
                                          tol_abs=1e-20)
    R = sum((delr[j] / (2 * K[j]) + delr[j + 1] / (2 * K[j + 1])) / area for j in range(ncol - 1))
    Q = 5.0 / R
    np.testing.assert_allclose(qx[0, 0, 1:ncol], Q, rtol=1e-12)
    assert qx[0, 0, 0] == 0.0 and qx[0, 0, ncol] == 0.0
    assert np.all(qy == 0.0) and np.all(qz == 0.0)


def test_cfg1_mass_balance():
    f = I.cfg1_field()
    b = f.balance()
    assert np.abs(b).max() <= 1e-12
    # the well extracts 1e-3 m^3/s: net inflow into its cell balances it
    k, i, j = 0, 25, 25
    inflow = f.qx[k, i, j] - f.qx[k, i, j + 1] + f.qy[k, i, j] - f.qy[k, i + 1, j]
    assert inflow == pytest.approx(1e-3, rel=1e-9)
    assert f.ibound[0, 25, 25] == I.IB_SINK


def test_random_field_mass_balance():
    f = I.random_box_field(4, 5, 6, seed=3, lnk_var=2.0, n_wells=2, n_inactive=3)
    qs = np.abs(f.qx).max()
    assert np.abs(f.balance()).max() <= 1e-9 * qs


@pytest.mark.parametrize("lam", [(2.0, 6.0, 6.0), (1.0, 4.0, 8.0)])
def test_gaussian_field_statistics(lam):
    vals = []
    for s in range(4):
        y = I.gaussian_field((16, 96, 96), lam, seed=50 + s)
        vals.append(y)
    y = np.stack(vals)
    assert abs(y.mean()) < 0.15
    assert abs(y.var() - 1.0) < 0.15
    # correlation at a lag of one correlation length along each axis ~ e^{-1}
    for ax in range(3):
        L = int(round(lam[ax]))
        a = np.take(y, np.arange(0, y.shape[ax + 1] - L), axis=ax + 1)
        b = np.take(y, np.arange(L, y.shape[ax + 1]), axis=ax + 1)
        rho = float(np.mean(a * b) / np.sqrt(np.mean(a * a) * np.mean(b * b)))
        assert abs(rho - math.exp(-1.0)) < 0.1, (ax, rho)
