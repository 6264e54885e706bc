"""Pins for the derived channels of the oracle (Sec. 4.5 Vel2D, Sec. 3.2 splat radius): the
projected velocity against central differences of the screen map along v, the angle and
magnitude against its components' definition, and the splat radius against the pixel distance
between a point on the optical axis and a point r above it."""
import numpy as np

import nrv_inputs as I
import oracle


def _screen(view, p):
    M = np.asarray(view.viewproj, np.float64).reshape(4, 4)
    c = M @ np.append(p, 1.0)
    return np.array([(c[0] / c[3] + 1) * view.width / 2, (1 - c[1] / c[3]) * view.height / 2])


def _one_point_key(idx, view):
    k = np.full((view.height, view.width), np.uint64(0xFFFFFFFFFFFFFFFF))
    k[3, 5] = np.uint64(idx)
    return k


def test_vel2d_matches_finite_differences_of_the_screen_map():
    view = I.make_view((0.3, 0.9, 2.5), (0.5, 0.4, 0.5), 640, 360)
    rng = np.random.default_rng(1)
    for _ in range(20):
        p = rng.uniform(0, 1, 3).astype(np.float32)
        v = rng.standard_normal(3).astype(np.float32)
        xyz = p[None]
        attr = np.zeros((1, 4), np.uint32)
        attr[0, 1:4] = v.view(np.uint32)
        key = _one_point_key(0, view)
        got = {f: oracle.derived_channel(key, xyz, attr, view, f, 1)[3, 5]
               for f in (oracle.VEL2D_X, oracle.VEL2D_Y, oracle.VEL2D_ANGLE, oracle.VEL2D_MAG)}
        h = 1e-6
        fd = (_screen(view, p.astype(np.float64) + h * v) - _screen(view, p.astype(np.float64) - h * v)) / (2 * h)
        np.testing.assert_allclose([got[oracle.VEL2D_X], got[oracle.VEL2D_Y]], fd, rtol=1e-6, atol=1e-6)
        assert abs(got[oracle.VEL2D_MAG] - np.hypot(*fd)) <= 1e-6 * max(1.0, np.hypot(*fd))
        assert abs(np.cos(got[oracle.VEL2D_ANGLE]) * got[oracle.VEL2D_MAG] - fd[0]) <= 1e-5 * max(1.0, abs(fd[0]))
        assert abs(np.sin(got[oracle.VEL2D_ANGLE]) * got[oracle.VEL2D_MAG] - fd[1]) <= 1e-5 * max(1.0, abs(fd[1]))
    # empty pixels are NaN
    assert np.isnan(oracle.derived_channel(key, xyz, attr, view, oracle.VEL2D_X, 1)[0, 0])


def test_splat_radius_on_the_optical_axis():
    eye, target = np.array([0.2, 0.1, 3.0]), np.array([0.2, 0.1, 0.0])
    view = I.make_view(tuple(eye), tuple(target), 800, 600)
    for depth, r in ((1.0, 0.01), (2.5, 0.003), (0.7, 0.02)):
        p = (eye + (target - eye) / np.linalg.norm(target - eye) * depth).astype(np.float32)
        attr = np.array([[np.float32(r).view(np.uint32)]], np.uint32)
        got = oracle.derived_channel(_one_point_key(0, view), p[None], attr, view,
                                     oracle.SPLAT_RADIUS, 0)[3, 5]
        # a point r above p (camera up is +y here) lands r_px pixels above p on screen
        d = np.linalg.norm(_screen(view, p.astype(np.float64) + np.array([0, r, 0])) -
                           _screen(view, p.astype(np.float64)))
        assert abs(got - d) <= 1e-5 * d, (got, d)
        # and it scales as 1 / depth
        assert abs(got * depth - r * 300 / np.tan(np.radians(I.FOVY_DEG) / 2)) <= 1e-4 * got * depth
