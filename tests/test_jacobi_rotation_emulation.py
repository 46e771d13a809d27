"""The rotations of the cluster solve's Jacobi (Alg. 5, "SVD of D" via K = D D^T),
emulated in float32 and float64: the half-angle form with refined reciprocal square
roots, and the one-reciprocal small-angle form t = (a_pq / x)(1 - (a_pq / x)^2),
c = 1 - t^2 / 2, s = t c used when |a_pq| <= g |x| (x = a_qq - a_pp; g = 2^-7 in FP32,
2^-14 in FP64).  Checked: c^2 + s^2 = 1 to the bound the small form claims (3 g^4 / 4
plus rounding), and the rotated off-diagonal entry is annihilated to O(t^3) of |a_pq|.
The checks pin the design constants; the GPU parity tests cover the kernel.  CPU only.
"""
import numpy as np
import pytest


def rotation_small(app, aqq, apq, dt):
    one = dt(1)
    u = dt(apq) * (one / dt(aqq - app))
    t = dt(u * (one - u * u))
    c = dt(one - dt(0.5) * t * t)
    return c, dt(t * c)


def rotation_exact(app, aqq, apq):
    # tan(phi): the smaller root of t^2 + 2 theta t - 1 = 0, theta = (a_qq - a_pp) / (2 a_pq)
    theta = (aqq - app) / (2.0 * apq)
    t = np.sign(theta) / (abs(theta) + np.sqrt(theta * theta + 1.0))
    c = 1.0 / np.sqrt(1.0 + t * t)
    return c, t * c


def offdiag_after(app, aqq, apq, c, s):
    # (J^T A J)(p, q) for J = [[c, s], [-s, c]]
    return (c * c - s * s) * apq + c * s * (app - aqq)


@pytest.mark.parametrize("dt,g,unit", [(np.float32, 2.0 ** -7, 2.0 ** -24),
                                       (np.float64, 2.0 ** -14, 2.0 ** -53)])
def test_small_angle_rotation_orthogonal_and_annihilating(dt, g, unit):
    rng = np.random.default_rng(5)
    for _ in range(2000):
        x = float(rng.uniform(0.1, 10.0) * rng.choice([-1.0, 1.0]))
        app = float(rng.standard_normal())
        aqq = app + x
        apq = float(rng.uniform(-1.0, 1.0)) * g * abs(x)
        c, s = rotation_small(dt(app), dt(aqq), dt(apq), dt)
        # c^2 + s^2 - 1 = -3 t^4 / 4 + O(t^6), t <= g, plus a few roundings
        dev = abs(float(c) ** 2 + float(s) ** 2 - 1.0)
        assert dev <= 0.75 * g ** 4 + 8 * unit
        # against the exact rotation: the angle agrees to O(t^4) relative, so the
        # off-diagonal left behind is O(t^3) |a_pq| plus rounding
        ce, se = rotation_exact(app, aqq, apq)
        assert abs(float(s) - se) <= 2 * g ** 3 * abs(se) + 8 * unit
        left = abs(offdiag_after(app, aqq, apq, float(c), float(s)))
        assert left <= (4 * g ** 2 + 64 * unit) * abs(apq) + 16 * unit * abs(x)


def test_small_angle_bound_fails_beyond_its_threshold():
    # at t = 2^-4 the first-order cosine is off by 3 t^4 / 4 ~ 1.1e-5, far above FP32
    # rounding: the threshold 2^-7 is what keeps the small form orthogonal in FP32
    t = 2.0 ** -4
    c = 1.0 - 0.5 * t * t
    s = t * c
    assert abs(c * c + s * s - 1.0) > 1e-5
