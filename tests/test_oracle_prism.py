"""Pins of the oracle's prism kernels against closed forms, limits and quadrature.

The paper does not print the prism formulas (Sec. 2.1 cites Haaz 1953, Li & Oldenburg
1998 and Rao & Babu 1991), so the oracle's closed forms are pinned here to facts that
do not come from those formulas: the point-source limits, additivity of the volume
integral, the infinite-slab (Bouguer) limit, Laplace's equation, Poisson's relation
between gravity and magnetic fields, and brute-force quadrature.
"""
import math

import numpy as np
import pytest

from oracle import prism

G_SI = 6.67430e-11


def test_gravity_point_mass_far_field():
    # cube of side a centred at (X, Y, Z) from the station; far away it acts as a point mass
    a = 50.0
    for X, Y, Z in [(3000.0, -2000.0, 4000.0), (-5000.0, 100.0, 1500.0)]:
        g = prism.gravity_gz(X - a / 2, X + a / 2, Y - a / 2, Y + a / 2, Z - a / 2, Z + a / 2)
        R = math.sqrt(X * X + Y * Y + Z * Z)
        point = G_SI * 1000.0 * a ** 3 * Z / R ** 3 * 1e5
        assert abs(g - point) / abs(point) < 1e-5


def test_gravity_sign_and_units():
    # a 1 g/cc cube right under the station attracts downwards (positive)
    g = prism.gravity_gz(-25.0, 25.0, -25.0, 25.0, 0.0, 50.0)
    assert g > 0
    # a slab-like wide prism tends to 2 pi G rho dz (Bouguer), in mGal
    L = 2.0e6
    dz = 50.0
    g = prism.gravity_gz(-L, L, -L, L, 100.0, 100.0 + dz)
    bouguer = 2 * math.pi * G_SI * 1000.0 * dz * 1e5
    assert abs(g - bouguer) / bouguer < 1e-4


def test_gravity_additivity():
    # the integral over a prism equals the sum over its 3x3x3 sub-prisms
    x = np.linspace(-70.0, 80.0, 4)
    y = np.linspace(-30.0, 120.0, 4)
    z = np.linspace(0.0, 150.0, 4)
    whole = prism.gravity_gz(x[0], x[-1], y[0], y[-1], z[0], z[-1])
    parts = sum(prism.gravity_gz(x[i], x[i + 1], y[j], y[j + 1], z[k], z[k + 1])
                for i in range(3) for j in range(3) for k in range(3))
    assert abs(whole - parts) <= 1e-12 * abs(whole)


def test_gravity_symmetry():
    # vertical attraction is even in x and in y (symmetric BTTB, Sec. 2.1)
    a = prism.gravity_gz(75.0, 125.0, -175.0, -125.0, 50.0, 100.0)
    b = prism.gravity_gz(-125.0, -75.0, -175.0, -125.0, 50.0, 100.0)
    c = prism.gravity_gz(75.0, 125.0, 125.0, 175.0, 50.0, 100.0)
    # corner sums cancel, so allow a few hundred ulps
    assert abs(a - b) <= 1e-12 * abs(a) and abs(a - c) <= 1e-12 * abs(a)


def test_gravity_quadrature():
    from scipy import integrate
    b = (-10.0, 15.0, -7.0, 9.0, 20.0, 35.0)
    num = integrate.tplquad(lambda zz, yy, xx: zz / (xx * xx + yy * yy + zz * zz) ** 1.5,
                            b[0], b[1], b[2], b[3], b[4], b[5], epsabs=1e-13, epsrel=1e-11)[0]
    assert abs(prism.gravity_unit(*b) - num) < 1e-9 * abs(num)


def test_tensor_quadrature():
    from scipy import integrate
    b = (-10.0, 15.0, -7.0, 9.0, 20.0, 35.0)

    def q(f):
        return integrate.tplquad(lambda zz, yy, xx: f(xx, yy, zz), b[0], b[1], b[2], b[3],
                                 b[4], b[5], epsabs=1e-13, epsrel=1e-10)[0]

    def r5(xx, yy, zz):
        return (xx * xx + yy * yy + zz * zz) ** 2.5

    num = [q(lambda xx, yy, zz: (2 * xx * xx - yy * yy - zz * zz) / r5(xx, yy, zz)),
           q(lambda xx, yy, zz: (2 * yy * yy - xx * xx - zz * zz) / r5(xx, yy, zz)),
           q(lambda xx, yy, zz: (2 * zz * zz - xx * xx - yy * yy) / r5(xx, yy, zz)),
           q(lambda xx, yy, zz: 3 * xx * yy / r5(xx, yy, zz)),
           q(lambda xx, yy, zz: 3 * xx * zz / r5(xx, yy, zz)),
           q(lambda xx, yy, zz: 3 * yy * zz / r5(xx, yy, zz))]
    got = prism.gradient_tensor(*b)
    for n_, g_ in zip(num, got):
        assert abs(n_ - g_) < 1e-8 * max(abs(n_), 1e-3)


def test_magnetic_dipole_far_field():
    a = 50.0
    for inc, dec in [(50.0, 10.0), (90.0, 0.0), (30.0, -40.0)]:
        f = np.array(prism.field_direction(inc, dec))
        for X, Y, Z in [(2500.0, 1800.0, 3000.0), (-4000.0, 900.0, 1200.0)]:
            dt = prism.magnetic_dt(X - a / 2, X + a / 2, Y - a / 2, Y + a / 2,
                                   Z - a / 2, Z + a / 2, inc, dec)
            R = np.array([X, Y, Z])
            Rn = np.linalg.norm(R)
            c = f @ R / Rn
            dip = prism.FIELD_NT * a ** 3 * (3 * c * c - 1) / (4 * math.pi * Rn ** 3)
            assert abs(dt - dip) < 1e-4 * abs(dip)


def test_magnetic_poisson_relation():
    # with a vertical field, dT = F/(4 pi) * d/dz_station of Int z/R^3 dV
    b = [75.0, 125.0, -175.0, -125.0, 50.0, 100.0]
    h = 1e-3
    up = prism.gravity_unit(b[0], b[1], b[2], b[3], b[4] + h, b[5] + h)
    dn = prism.gravity_unit(b[0], b[1], b[2], b[3], b[4] - h, b[5] - h)
    dgdz = (dn - up) / (2 * h)            # station moving down by h shortens z offsets
    dt = prism.magnetic_dt(*b, 90.0, 0.0)
    assert abs(dt - prism.FIELD_NT / (4 * math.pi) * dgdz) < 1e-6 * abs(dt)


def test_magnetic_laplace_trace():
    b = (-40.0, 10.0, 60.0, 110.0, 0.0, 50.0)
    s = sum(prism.magnetic_dt(*b, inc, dec) for inc, dec in [(0.0, 0.0), (0.0, 90.0), (90.0, 0.0)])
    ref = abs(prism.magnetic_dt(*b, 90.0, 0.0))
    assert abs(s) < 1e-12 * ref


def test_magnetic_additivity_and_slab():
    x = np.linspace(-70.0, 80.0, 4)
    y = np.linspace(-30.0, 120.0, 4)
    z = np.linspace(0.0, 150.0, 4)
    whole = prism.magnetic_dt(x[0], x[-1], y[0], y[-1], z[0], z[-1], 50.0, 10.0)
    parts = sum(prism.magnetic_dt(x[i], x[i + 1], y[j], y[j + 1], z[k], z[k + 1], 50.0, 10.0)
                for i in range(3) for j in range(3) for k in range(3))
    assert abs(whole - parts) <= 1e-11 * abs(whole)
    # a laterally infinite uniformly magnetised layer has no external field
    L = 1.0e7
    slab = prism.magnetic_dt(-L, L, -L, L, 100.0, 150.0, 50.0, 10.0)
    assert abs(slab) < 1e-5 * abs(whole)


@pytest.mark.parametrize("inc,dec", [(50.0, 10.0), (35.0, 60.0)])
def test_magnetic_not_symmetric(inc, dec):
    # magnetic blocks are BTTB but not symmetric in general (Sec. 2.1)
    a = prism.magnetic_dt(75.0, 125.0, -175.0, -125.0, 50.0, 100.0, inc, dec)
    b = prism.magnetic_dt(-125.0, -75.0, 125.0, 175.0, 50.0, 100.0, inc, dec)
    assert abs(a - b) > 1e-6 * abs(a)


def _mp_exact_gravity(b):
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 40

    def F(x, y, z):
        r = mp.sqrt(x * x + y * y + z * z)
        return x * mp.log(y + r) + y * mp.log(x + r) - z * mp.atan2(x * y, z * r)
    s = 0
    for i, x in enumerate(b[0:2]):
        for j, y in enumerate(b[2:4]):
            for k, z in enumerate(b[4:6]):
                s += (-1) ** (i + j + k) * F(mp.mpf(x), mp.mpf(y), mp.mpf(z))
    return float(s) * prism.GRAV_SCALE


def _mp_exact_magnetic(b, inc, dec):
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 40
    T = [mp.mpf(0)] * 6
    for i, x in enumerate(b[0:2]):
        for j, y in enumerate(b[2:4]):
            for k, z in enumerate(b[4:6]):
                x, y, z = mp.mpf(x), mp.mpf(y), mp.mpf(z)
                r = mp.sqrt(x * x + y * y + z * z)
                c = -(-1) ** (i + j + k)
                T[0] -= c * mp.atan(y * z / (x * r))
                T[1] -= c * mp.atan(x * z / (y * r))
                T[2] -= c * mp.atan2(x * y, z * r)
                T[3] += c * mp.log(z + r)
                T[4] += c * mp.log(y + r)
                T[5] += c * mp.log(x + r)
    fx, fy, fz = [mp.mpf(v) for v in prism.field_direction(inc, dec)]
    q = fx * fx * T[0] + fy * fy * T[1] + fz * fz * T[2] + 2 * (fx * fy * T[3] + fx * fz * T[4]
                                                                 + fy * fz * T[5])
    return float(q) * prism.FIELD_NT / (4 * math.pi)


@pytest.mark.parametrize("D", [0.5, 1.7, 1.95, 2.05, 2.6, 3.5, 4.1, 5.0, 7.9, 9.0, 40.0, 150.0])
def test_cell_entries_accurate_at_every_distance(D):
    # the hybrid closed-form / quadrature entries agree with 40-digit evaluations
    worst_g = worst_m = 0.0
    for ang in (0.1, 0.7, 1.3):
        for zc in (25.0, 125.0):
            cx = D * 50 * math.cos(ang) + 12.5
            cy = D * 50 * math.sin(ang) * 0.7 - 12.5
            b = (cx - 25, cx + 25, cy - 25, cy + 25, zc - 25, zc + 25)
            eg = _mp_exact_gravity(b)
            em = _mp_exact_magnetic(b, 50.0, 10.0)
            worst_g = max(worst_g, abs(prism.gravity_cell(*b) - eg) / abs(eg))
            worst_m = max(worst_m, abs(prism.magnetic_cell(*b, 50.0, 10.0) - em) / abs(em))
    assert worst_g < 2e-13 and worst_m < 2e-13, (worst_g, worst_m)


def test_closed_form_loses_digits_far_away():
    # documents why far entries use quadrature: 150 cells away the corner sum is poor
    b = (7475.0, 7525.0, -2275.0, -2225.0, 0.0, 50.0)
    eg = _mp_exact_gravity(b)
    assert abs(prism.gravity_gz(*b) - eg) / eg > 1e-9
    assert abs(prism.gravity_cell(*b) - eg) / eg < 1e-14
