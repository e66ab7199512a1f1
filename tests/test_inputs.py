"""Seeded input generators (CPU): the scalings keep every window's points in
the domains the library checks (the box [-1/4, 1/4)^d of Sec. 3.1, and the
ball |x| <= 1/4 - eps_b/2 that outer boundary smoothing needs)."""
import numpy as np

from paper_2504_00480_gb300 import inputs


def test_minmax_scale_stays_in_the_box():
    X = inputs.minmax_scale(np.random.default_rng(0).standard_normal((5000, 6)) * 7.0 + 3.0)
    assert X.min() >= inputs.LO and X.max() <= inputs.HI
    assert -0.25 <= X.min() and X.max() < 0.25
    np.testing.assert_allclose(X.min(axis=0), inputs.LO)
    np.testing.assert_allclose(X.max(axis=0), inputs.HI)


def test_ball_scale_reaches_the_radius_per_window():
    W = [[0, 1, 2], [3, 4], [5]]
    X = inputs.minmax_scale(np.random.default_rng(1).standard_normal((4000, 6)))
    Y = inputs.ball_scale(X, W, 0.1875)
    for w in W:
        norms = np.sqrt((Y[:, w] ** 2).sum(axis=1))
        assert abs(norms.max() - 0.1875) < 1e-15
        # one factor per window: the shape of the window's point cloud is kept
        ratio = Y[:, w] / np.where(X[:, w] == 0, 1, X[:, w])
        nz = X[:, w] != 0
        assert np.ptp(ratio[nz]) < 1e-12
    # rounding to float32 with a margin keeps the points inside the ball
    Z = inputs.to_precision(inputs.ball_scale(X, W, 0.999 * 0.1875), np.float32).astype(np.float64)
    for w in W:
        assert np.sqrt((Z[:, w] ** 2).sum(axis=1)).max() <= 0.1875


def test_generators_are_seeded():
    a = inputs.nlml_grad(n=2000, R=4)
    b = inputs.nlml_grad(n=2000, R=4)
    np.testing.assert_array_equal(a.X, b.X)
    np.testing.assert_array_equal(a.V, b.V)
