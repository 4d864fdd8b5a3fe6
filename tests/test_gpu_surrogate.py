"""The learned field surrogate on the GPU against its FP64 oracle: BF16
gradients within the BF16 bound, the assembled surrogate field against the
oracle's composition, training that lowers the loss, and a trained network
that beats both its untrained start and the near-field truncation it
corrects (the method without the network)."""
import numpy as np
import pytest

import oracle as O
import paper_1803_04782_gb300 as sfm
import scenegen as SG
from oracle import surrogate as OS
from paper_1803_04782_gb300 import build as B

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    B.build()
    sfm.lib()


def bf16(a):
    """Round to the nearest BF16 (ties to even), returned as float64."""
    u = np.ascontiguousarray(a, np.float32).view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def _rounded_params(seed=0, scale=1.0):
    ps = OS.init_params(seed)
    return [(bf16(W * scale), bf16(b)) for W, b in ps]


def test_gradients_match_the_oracle_within_bf16_bound():
    rng = np.random.default_rng(11)
    params = _rounded_params(3)
    params = [(W, bf16(rng.normal(0, 0.05, b.shape))) for W, b in params]
    X = bf16(rng.random((3, 30, 34)) * 0.3)
    T = rng.normal(0, 1.0, (30 - 2 * OS.HALO, 34 - 2 * OS.HALO))
    L_o, g_o = OS.loss_and_grad(params, X, T)
    with sfm.Surrogate(params=sfm.flatten_params(params)) as s:
        L_g, g_flat = s.grad(X, T)
    assert L_g == pytest.approx(L_o, rel=2e-2)
    g_g = sfm.unflatten_params(g_flat)
    for li, ((gw_o, gb_o), (gw_g, gb_g)) in enumerate(zip(g_o, g_g)):
        for a, b in ((gw_o, gw_g), (gb_o, gb_g)):
            a, b = a.ravel(), b.ravel()
            rel = np.linalg.norm(a - b) / max(np.linalg.norm(a), 1e-30)
            cos = float(a @ b / max(np.linalg.norm(a) * np.linalg.norm(b), 1e-30))
            assert rel <= 2e-2, (li, rel)
            assert cos >= 0.999, (li, cos)


def test_surrogate_field_matches_the_oracle_composition():
    sc = SG.random_scene(96, 64, 700, r=12, seed=31, periodic_x=1, periodic_y=1, ring=False,
                         exits=(), goal_mode="fixed", heading_mode="random")
    s_, rn, scale = 8, 2, 5.0
    params = _rounded_params(4, scale=0.5)
    # oracle: exact near field (radius rn) + static field, plus the network's
    # far part on the coarse channels, interpolated to every su
    m = O.model(sc, r=rn)
    occ, _ = O.occupancy(m, sc.cell, sc.xy)
    Fn, Sn = O.field(m, sc.cell, occ, sc.heading)
    X = OS.coarse_channels(sc.W, sc.H, s_, sc.xy, sc.heading)
    Xp = np.pad(X, ((0, 0), (OS.HALO, OS.HALO), (OS.HALO, OS.HALO)), mode="wrap")
    Y, _ = OS.forward(params, bf16(Xp))
    F_orc = Fn + scale * OS.upsample(Y, s_, periodic=True)
    with sfm.Sim(sc) as sim, sfm.Surrogate(coarsen=s_, near_radius=rn, target_scale=scale,
                                           params=sfm.flatten_params(params)) as sur:
        F = sur.field(sim).astype(np.float64)
    far = scale * np.abs(OS.upsample(Y, s_))
    tol = 1e-5 * Sn + 2e-2 * far.max() + 1e-6
    assert (np.abs(F - F_orc) <= tol).all(), float(np.max(np.abs(F - F_orc) - tol))


def _canvas(side, seed):
    return SG.training_canvas(side=side, r=40, seed=seed)


def test_training_lowers_loss_and_beats_the_untrained_net_and_truncation():
    train = _canvas(768, 61)
    test = _canvas(768, 62)
    init = sfm.flatten_params(_rounded_params(0))
    with sfm.Sim(train) as tsim, sfm.Sim(test) as esim, \
            sfm.Surrogate(coarsen=8, near_radius=3, target_scale=20.0, lr=2e-3,
                          params=init) as sur:
        before = sur.eval(esim)
        curve = sur.train(tsim, 150)
        assert curve[-10:].mean() < 0.3 * curve[:3].mean(), curve[[0, 1, 2, -3, -2, -1]]
        after = sur.eval(esim)
        # the method without the network: near field only (zero network output)
        zero = np.zeros_like(init)
        sur.set_params(zero)
        trunc = sur.eval(esim)
    assert after["field_rel_err"] < 0.5 * before["field_rel_err"], (before, after)
    assert after["field_rel_err"] < 0.5 * trunc["field_rel_err"], (trunc, after)
    assert after["flip_rate"] < trunc["flip_rate"], (trunc, after)
