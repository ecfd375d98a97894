"""Prism kernels of the forward model (Sec. 2.1, Eq. (2)): FP64 closed forms.

TEST INFRASTRUCTURE ONLY: this file belongs to the CPU oracle.  Only ``tests/``,
``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline leg may import it; the
product path never does.

The paper cites Haaz (1953) / Li & Oldenburg (1998) for the gravity kernel and Rao &
Babu (1991) for the magnetic kernel without printing either (Sec. 2.1).  Both are the
volume integrals of a point-source kernel over a right rectangular prism:

* gravity: vertical attraction ``g_z = gamma*rho * Int z / R^3 dV`` (z positive down),
  integrated in closed form with the antiderivative
  ``F = x ln(y + R) + y ln(x + R) - z atan2(x y, z R)`` summed over the eight corners
  with sign ``(-1)^(i+j+k)`` (lower corner index 0);
* magnetic: total-field anomaly of a uniformly induced prism (no remanence, no
  self-demagnetisation), ``dT = (kappa F / 4 pi) * sum_ab f_a f_b T_ab`` with
  ``T_ab = Int d_a d_b (1/R) dV`` (the prism's gravity-gradient tensor, Poisson's
  relation), whose corner antiderivatives are ``-atan(yz/(xR))`` (xx), ``ln(z+R)``
  (xy), ``ln(y+R)`` (xz) and the cyclic forms.  ``f`` is the unit vector of the
  inducing field (x north, y east, z down): ``(cos I cos D, cos I sin D, sin I)``.

Coordinates passed in are corner offsets ``cell corner - station`` in metres.  Units:
gravity in mGal per g/cc, magnetic in nT per SI susceptibility.

Numerical evaluation (the paper is silent on it): the closed forms sum eight corner
terms of size ~R log R whose total is ~V/R^2 (gravity) or ~V/R^3 (magnetic), so they
lose about (R/L)^3 ulps to cancellation at distance R from a cell of size L (7e-7
relative error at 150 cells).  The cell entries used for G (``gravity_cell``,
``magnetic_cell``) therefore take the closed form only within 2 L of the station and
otherwise integrate the point-source kernel by tensor Gauss-Legendre quadrature: 14
points per axis for 2 L <= D < 4 L, 8 for 4 L <= D < 8 L and 6 beyond (D = distance
from the station to the cell centre, L = the longest cell side).  Against 40-digit
evaluations of the closed form this keeps every entry within ~1e-13 relative.
"""
from __future__ import annotations

import numpy as np

GAMMA = 6.67430e-11          # m^3 kg^-1 s^-2
GCC_TO_KGM3 = 1000.0         # g/cc -> kg/m^3
MS2_TO_MGAL = 1.0e5          # m/s^2 -> mGal
GRAV_SCALE = GAMMA * GCC_TO_KGM3 * MS2_TO_MGAL
FIELD_NT = 50000.0           # inducing field strength (nT); the paper does not state it


def _log_plus(a, rest2, r):
    """ln(a + r) with r = sqrt(a^2 + rest2), stable when a < 0 (no cancellation)."""
    a = np.asarray(a, dtype=np.float64)
    out = np.empty(np.broadcast(a, rest2, r).shape)
    a_b, rest_b, r_b = np.broadcast_arrays(a, rest2, r)
    pos = a_b >= 0
    out[pos] = np.log(a_b[pos] + r_b[pos])
    neg = ~pos
    out[neg] = np.log(rest_b[neg] / (r_b[neg] - a_b[neg]))
    return out


def _corners(x1, x2, y1, y2, z1, z2):
    """Yield (x, y, z, sign) for the eight corners, sign = (-1)^(i+j+k)."""
    for i, x in enumerate((x1, x2)):
        for j, y in enumerate((y1, y2)):
            for k, z in enumerate((z1, z2)):
                yield (np.asarray(x, np.float64), np.asarray(y, np.float64),
                       np.asarray(z, np.float64), (-1.0) ** (i + j + k))


def gravity_unit(x1, x2, y1, y2, z1, z2):
    """Int z/R^3 dV over the prism (metres), station at the origin, z down."""
    total = 0.0
    for x, y, z, s in _corners(x1, x2, y1, y2, z1, z2):
        r = np.sqrt(x * x + y * y + z * z)
        f = (x * _log_plus(y, x * x + z * z, r) + y * _log_plus(x, y * y + z * z, r)
             - z * np.arctan2(x * y, z * r))
        total = total + s * f
    return total


def gravity_gz(x1, x2, y1, y2, z1, z2):
    """Vertical attraction in mGal of a 1 g/cc prism (corner offsets in metres)."""
    return GRAV_SCALE * gravity_unit(x1, x2, y1, y2, z1, z2)


def gradient_tensor(x1, x2, y1, y2, z1, z2):
    """(Txx, Tyy, Tzz, Txy, Txz, Tyz) = Int d_a d_b (1/R) dV, dimensionless."""
    txx = tyy = tzz = txy = txz = tyz = 0.0
    for x, y, z, s in _corners(x1, x2, y1, y2, z1, z2):
        r = np.sqrt(x * x + y * y + z * z)
        # corner sign for the upper-limit-positive convention is -(-1)^(i+j+k)
        c = -s
        # x and y corner offsets are never zero (stations sit over cell centres);
        # z >= 0, so atan2 gives the z -> 0+ limit of atan(xy/(zR)).
        txx = txx - c * np.arctan(y * z / (x * r))
        tyy = tyy - c * np.arctan(x * z / (y * r))
        tzz = tzz - c * np.arctan2(x * y, z * r)
        txy = txy + c * _log_plus(z, x * x + y * y, r)
        txz = txz + c * _log_plus(y, x * x + z * z, r)
        tyz = tyz + c * _log_plus(x, y * y + z * z, r)
    return txx, tyy, tzz, txy, txz, tyz


def field_direction(inc_deg: float, dec_deg: float):
    """Unit vector of the inducing field, x north, y east, z down."""
    i = np.deg2rad(inc_deg)
    d = np.deg2rad(dec_deg)
    return np.cos(i) * np.cos(d), np.cos(i) * np.sin(d), np.sin(i)


def magnetic_dt(x1, x2, y1, y2, z1, z2, inc_deg: float, dec_deg: float,
                field_nt: float = FIELD_NT):
    """Total-field anomaly (nT) of a prism of unit SI susceptibility, induced only."""
    fx, fy, fz = field_direction(inc_deg, dec_deg)
    txx, tyy, tzz, txy, txz, tyz = gradient_tensor(x1, x2, y1, y2, z1, z2)
    quad = (fx * fx * txx + fy * fy * tyy + fz * fz * tzz
            + 2.0 * (fx * fy * txy + fx * fz * txz + fy * fz * tyz))
    return field_nt / (4.0 * np.pi) * quad


# --- cell entries: closed form near the station, Gauss-Legendre quadrature far -------
NEAR = 2.0
MID = 4.0
FAR = 8.0


def _gauss_points(n: int):
    t, w = np.polynomial.legendre.leggauss(n)
    return t, w


def _quadrature(x1, x2, y1, y2, z1, z2, n, integrand):
    """Tensor Gauss-Legendre rule with n points per axis over each prism (arrays)."""
    t, w = _gauss_points(n)
    cx, hx = 0.5 * (x1 + x2), 0.5 * (x2 - x1)
    cy, hy = 0.5 * (y1 + y2), 0.5 * (y2 - y1)
    cz, hz = 0.5 * (z1 + z2), 0.5 * (z2 - z1)
    total = 0.0
    for i in range(n):
        x = cx + hx * t[i]
        for j in range(n):
            y = cy + hy * t[j]
            wij = w[i] * w[j]
            for k in range(n):
                z = cz + hz * t[k]
                total = total + (wij * w[k]) * integrand(x, y, z)
    return total * hx * hy * hz


def _hybrid(x1, x2, y1, y2, z1, z2, closed, integrand):
    x1, x2, y1, y2, z1, z2 = np.broadcast_arrays(*[np.asarray(v, np.float64)
                                                   for v in (x1, x2, y1, y2, z1, z2)])
    cx, cy, cz = 0.5 * (x1 + x2), 0.5 * (y1 + y2), 0.5 * (z1 + z2)
    L = np.maximum(np.maximum(x2 - x1, y2 - y1), z2 - z1)
    D = np.sqrt(cx * cx + cy * cy + cz * cz)
    out = np.empty(x1.shape)
    groups = [(D < NEAR * L, None), ((D >= NEAR * L) & (D < MID * L), 14),
              ((D >= MID * L) & (D < FAR * L), 8), (D >= FAR * L, 6)]
    for mask, n in groups:
        if not np.any(mask):
            continue
        args = [v[mask] for v in (x1, x2, y1, y2, z1, z2)]
        out[mask] = closed(*args) if n is None else _quadrature(*args, n, integrand)
    return out if out.shape else float(out)


def gravity_cell(x1, x2, y1, y2, z1, z2):
    """Entry of G for gravity (mGal per g/cc): Int z/R^3 dV, accurate at any distance."""
    def f(x, y, z):
        r2 = x * x + y * y + z * z
        return z / (r2 * np.sqrt(r2))
    return GRAV_SCALE * _hybrid(x1, x2, y1, y2, z1, z2, gravity_unit, f)


def magnetic_cell(x1, x2, y1, y2, z1, z2, inc_deg: float, dec_deg: float,
                  field_nt: float = FIELD_NT):
    """Entry of G for the total-field anomaly (nT per SI), accurate at any distance."""
    fx, fy, fz = field_direction(inc_deg, dec_deg)

    def closed(*b):
        txx, tyy, tzz, txy, txz, tyz = gradient_tensor(*b)
        return (fx * fx * txx + fy * fy * tyy + fz * fz * tzz
                + 2.0 * (fx * fy * txy + fx * fz * txz + fy * fz * tyz))

    def f(x, y, z):
        r2 = x * x + y * y + z * z
        fr = fx * x + fy * y + fz * z
        return (3.0 * fr * fr - r2) / (r2 * r2 * np.sqrt(r2))
    return field_nt / (4.0 * np.pi) * _hybrid(x1, x2, y1, y2, z1, z2, closed, f)
