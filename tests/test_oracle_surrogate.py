"""Pins of the surrogate oracle (CPU): the convolution equals a library
cross-correlation, the analytic gradients equal central finite differences,
and the coarse channels / cell averages / interpolation reduce to their
definitions on hand-made cases."""
import numpy as np
import pytest

from oracle import surrogate as S


def _tiny_params(seed=3):
    rng = np.random.default_rng(seed)
    dims = [(3, 4, 5), (4, 4, 3), (4, 4, 3), (4, 1, 3)]
    return [(rng.normal(0, 0.5, (o, c, k, k)), rng.normal(0, 0.1, o)) for c, o, k in dims]


def test_conv_equals_scipy_correlate():
    from scipy.signal import correlate
    rng = np.random.default_rng(1)
    X = rng.normal(size=(3, 11, 9))
    W = rng.normal(size=(2, 3, 5, 5))
    b = rng.normal(size=2)
    Z = S.conv_valid(X, W, b)
    for o in range(2):
        ref = sum(correlate(X[c], W[o, c], mode="valid") for c in range(3)) + b[o]
        np.testing.assert_allclose(Z[o], ref, rtol=1e-12, atol=1e-12)


def test_forward_shapes_and_receptive_field():
    ps = S.init_params(0)
    X = np.random.default_rng(0).random((3, 26, 30))
    Y, _ = S.forward(ps, X)
    assert Y.shape == (26 - 2 * S.HALO, 30 - 2 * S.HALO)
    # an output depends on inputs within HALO cells only
    X3 = X.copy()
    X3[:, 25, 29] += 5.0                     # far corner: outside output (0, 0)'s window
    Y3, _ = S.forward(ps, X3)
    assert Y3[0, 0] == Y[0, 0]


@pytest.mark.parametrize("li", [0, 1, 2, 3])
def test_gradients_match_central_differences(li):
    ps = _tiny_params()
    rng = np.random.default_rng(7)
    X = rng.normal(size=(3, 14, 13))
    T = rng.normal(size=(14 - 2 * S.HALO, 13 - 2 * S.HALO))
    L, grads = S.loss_and_grad(ps, X, T)
    W, b = ps[li]
    eps = 1e-6
    for idx in [(0, 0, 0, 0), tuple(np.array(W.shape) - 1), (0, W.shape[1] // 2, 1, 2)]:
        Wp = W.copy(); Wp[idx] += eps
        Wm = W.copy(); Wm[idx] -= eps
        pp = list(ps); pp[li] = (Wp, b)
        pm = list(ps); pm[li] = (Wm, b)
        num = (S.loss_and_grad(pp, X, T)[0] - S.loss_and_grad(pm, X, T)[0]) / (2 * eps)
        assert grads[li][0][idx] == pytest.approx(num, rel=1e-5, abs=1e-9)
    bp = b.copy(); bp[0] += eps
    bm = b.copy(); bm[0] -= eps
    pp = list(ps); pp[li] = (W, bp)
    pm = list(ps); pm[li] = (W, bm)
    num = (S.loss_and_grad(pp, X, T)[0] - S.loss_and_grad(pm, X, T)[0]) / (2 * eps)
    assert grads[li][1][0] == pytest.approx(num, rel=1e-5, abs=1e-9)


def test_coarse_channels_cell_average_and_upsampling():
    xy = np.array([[0, 0], [3, 2], [7, 7], [8, 1]])
    heading = np.array([1, 3, 6, 0])
    X = S.coarse_channels(16, 8, 4, xy, heading)
    assert X.shape == (3, 2, 4)
    assert X[0, 0, 0] == 2 / 16 and X[0, 1, 1] == 1 / 16 and X[0, 0, 2] == 1 / 16
    assert X[1, 0, 0] == 1 / 16 and X[2, 0, 0] == 1 / 16
    assert X[1, 1, 1] == pytest.approx(-(2 ** -0.5) / 16)
    F = np.arange(64.0).reshape(8, 8)
    np.testing.assert_array_equal(S.cell_average(F, 4), [[13.5, 17.5], [45.5, 49.5]])
    # interpolating a constant gives the constant; a linear ramp stays linear
    np.testing.assert_allclose(S.upsample(np.full((3, 4), 2.5), 4), 2.5)
    ramp = np.tile(np.arange(4.0), (3, 1))
    up = S.upsample(ramp, 4, periodic=False)
    np.testing.assert_allclose(up[5, 6:10], (np.arange(6, 10) + 0.5) / 4 - 0.5)


def test_untapered_near_field_equals_the_model_field_at_radius_rn():
    """With r_in >= rn the near part is the model's pedestrian field with the
    influence radius set to rn (the C oracle, independent code)."""
    import oracle as O
    import scenegen as SG
    sc = SG.random_scene(23, 19, 40, r=4, seed=7, periodic_x=1, exits=("south",),
                         goal_mode="mixed", heading_mode="random")
    m = O.model(sc, r=4)
    occ, bad = O.occupancy(m, sc.cell, sc.xy)
    assert bad == 0
    Fp, _ = O.field(m, sc.cell, occ, sc.heading, parts=2)
    Fn = S.tapered_near_field(sc.W, sc.H, sc.xy, sc.heading, 4, 10.0, m.kP, m.aP, m.gamma,
                              periodic_x=1, periodic_y=0)
    np.testing.assert_allclose(Fn, Fp, rtol=1e-12, atol=1e-12)


def test_taper_of_a_single_pedestrian():
    """One pedestrian heading east: full kernel inside r_in, half of it at
    the taper's midpoint, nothing at or beyond rn."""
    rn, r_in = 6, 2.0
    F = S.tapered_near_field(21, 21, [(10, 10)], [1], rn, r_in, 2.0, -0.5, 0.5)
    K = lambda dx, dy: 2.0 * np.hypot(dx, dy) ** -0.5 * (1 + 0.5 * dx / np.hypot(dx, dy))
    assert F[10, 12] == pytest.approx(K(2, 0), rel=1e-14)        # d = 2 = r_in
    assert F[10, 14] == pytest.approx(0.5 * K(4, 0), rel=1e-14)  # d = 4, midpoint
    assert F[10, 16] == 0.0 and F[16, 16] == 0.0                 # d = 6 and 8.5
    assert F[13, 13] == pytest.approx(S.taper_weight(np.hypot(3, 3), r_in, rn) * K(3, 3), rel=1e-14)
    assert 0.0 < S.taper_weight(5.0, r_in, rn) < 0.5 < S.taper_weight(3.0, r_in, rn) < 1.0
