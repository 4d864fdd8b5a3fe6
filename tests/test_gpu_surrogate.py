"""The learned field surrogate on the GPU against its FP64 oracle: BF16
gradients within the BF16 bound, the assembled surrogate field against the
oracle's composition, training that lowers the loss, a trained network that
beats both its untrained start and the near-field truncation it corrects
(the method without the network), and the exact fallback of the decisions:
bit-for-bit exact ticks with an infinite margin bound, the flip target with
a calibrated one."""
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


@pytest.mark.parametrize("shape", [(30, 34), (157, 333)])
def test_tcgen05_layers_match_the_mma_sync_layers_and_the_oracle(shape):
    """The 3x3 32 -> 32 layers on tcgen05 against the same layers on mma.sync
    (both sum in FP32 and round the activations to BF16, in different orders,
    so a hidden activation may differ by one BF16 rounding), and the network's
    output against the FP64 oracle from the same BF16 inputs and weights; the
    larger image has ragged tiles in both directions."""
    rng = np.random.default_rng(21)
    params = _rounded_params(5, scale=0.5)
    X = bf16(rng.random((3,) + shape) * 0.3)
    with sfm.Surrogate(params=sfm.flatten_params(params)) as s:
        Yu = s.forward(X, tcgen05=True)
        Ym = s.forward(X, tcgen05=False)
    Yo, _ = OS.forward(params, X)
    assert Yu.shape == Ym.shape == Yo.shape
    scale = float(np.abs(Yo).max())
    assert scale > 0
    assert float(np.abs(Yu - Ym).max()) <= 2e-2 * scale
    for Y in (Yu, Ym):
        assert np.linalg.norm(Y - Yo) / np.linalg.norm(Yo) <= 2e-2


@pytest.mark.parametrize("after", [0, 1])
def test_tcgen05_wait_that_runs_out_reports_timeout_and_falls_back(after):
    """A tcgen05 launch whose producer stops issuing copies (a test hook, no
    fault): its MMA and store warps' bounded waits run out, the launch drains
    what it issued and frees its tensor memory, the call reports
    SFM_ETIMEOUT, and later calls run the layers on mma.sync with the same
    result as before."""
    rng = np.random.default_rng(22)
    params = _rounded_params(6, scale=0.5)
    # 394 x 394 layer-2 outputs: 396 tiles of 4 x 128, at least two per CTA
    # on 152 SMs, so after = 1 stops every CTA with tiles left
    X = bf16(rng.random((3, 400, 400)) * 0.3)
    with sfm.Surrogate(params=sfm.flatten_params(params)) as s:
        Ym = s.forward(X, tcgen05=False)
        s.test_stop_copies(after)
        with pytest.raises(sfm.SfmError) as e:
            s.forward(X, tcgen05=True)
        assert e.value.status == sfm.SFM_ETIMEOUT
        Y2 = s.forward(X, tcgen05=True)   # now on mma.sync
        assert np.array_equal(Y2, Ym)
    # the device is still usable for a fresh surrogate on tcgen05
    with sfm.Surrogate(params=sfm.flatten_params(params)) as s:
        Yu = s.forward(X, tcgen05=True)
    assert float(np.abs(Yu - Ym).max()) <= 2e-2 * float(np.abs(Ym).max())


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


@pytest.mark.parametrize("rn,taper", [(2, None), (6, 2.5)])
def test_surrogate_field_matches_the_oracle_composition(rn, taper):
    """F_sur = F_static + (tapered) near part + scale * bilinear(network
    output), against the FP64 oracle's composition from the same BF16 inputs."""
    sc = SG.random_scene(96, 64, 700, r=12, seed=31, periodic_x=1, periodic_y=1, ring=False,
                         exits=(), goal_mode="fixed", heading_mode="random")
    s_, scale = 8, 5.0
    params = _rounded_params(4, scale=0.5)
    m = O.model(sc)
    occ, _ = O.occupancy(m, sc.cell, sc.xy)
    Fs, Ss = O.field(m, sc.cell, occ, sc.heading, parts=1)
    r_in = float(rn) if taper is None else taper
    Fn = Fs + OS.tapered_near_field(sc.W, sc.H, sc.xy, sc.heading, rn, r_in, m.kP, m.aP, m.gamma,
                                    periodic_x=1, periodic_y=1)
    X = OS.coarse_channels(sc.W, sc.H, s_, sc.xy, sc.heading)
    Xp = np.pad(X, ((0, 0), (OS.HALO, OS.HALO), (OS.HALO, OS.HALO)), mode="wrap")
    Y, _ = OS.forward(params, bf16(Xp))
    F_orc = Fn + scale * OS.upsample(Y, s_, periodic=True)
    with sfm.Sim(sc) as sim, sfm.Surrogate(coarsen=s_, near_radius=rn, target_scale=scale,
                                           taper_inner=taper,
                                           params=sfm.flatten_params(params)) as sur:
        F = sur.field(sim).astype(np.float64)
    far = scale * np.abs(OS.upsample(Y, s_))
    near_mag = np.abs(Fn - Fs).max()
    tol = 1e-5 * (Ss + near_mag) + 2e-2 * far.max() + 1e-6
    assert (np.abs(F - F_orc) <= tol).all(), float(np.max(np.abs(F - F_orc) - tol))


def _fallback_scenes():
    return [
        SG.random_scene(300, 260, 5000, r=12, seed=111, exits=("east",), goal_mode="mixed",
                        heading_mode="random"),
        SG.random_scene(128, 96, 1500, r=9, seed=103, periodic_x=1, periodic_y=1, ring=False,
                        exits=(), goal_mode="fixed", heading_mode="random"),
        SG.random_scene(160, 144, 1400, r=41, seed=113, periodic_x=1, exits=("north",),
                        goal_mode="mixed", heading_mode="random"),
        SG.random_scene(160, 176, 1500, r=47, seed=110, periodic_y=1, exits=("east",),
                        goal_mode="mixed", heading_mode="random"),
    ]


@pytest.mark.parametrize("i", range(6))
def test_infinite_delta_falls_back_everywhere_and_reproduces_the_exact_ticks(i):
    """With delta = +inf neither the network nor the surrogate composition
    runs: every pedestrian is decided on the exact field at its 9 candidates
    only, computed by the warp fallback in the exact gather's order (the
    exact candidate-only tick).  The trajectory equals the lattice path's bit
    for bit, on small scenes, with walk periods, and on the 4096^2 floor at
    the benchmark's density and radius."""
    if i < 4:
        sc = _fallback_scenes()[i]
    elif i == 4:
        sc = SG.random_scene(300, 260, 6000, r=20, seed=133, obstacles=4, exits=("east", "north"),
                             goal_mode="mixed", heading_mode="random")
    else:
        sc = SG.floor(side=4096, n=62500, exit_len=64)
    init = sfm.flatten_params(_rounded_params(2))
    with sfm.Sim(sc) as a, sfm.Sim(sc) as b, \
            sfm.Surrogate(coarsen=4, near_radius=3, params=init) as sur:
        if i == 4:
            per, pha = SG.walk_periods(sc.n, 4)
            a.set_walk_periods(per, pha)
            b.set_walk_periods(per, pha)
        for t in range(4):
            a.step(1)
            sur.step(b, 1)
            np.testing.assert_array_equal(a.decisions()[0], b.decisions()[0], err_msg=f"tick {t}")
            for x, y in zip(a.peds(), b.peds()):
                np.testing.assert_array_equal(x, y)
        fb, dec = sur.counts()
        if i == 4:   # walk periods: only the pedestrians whose tick it is decide
            assert 0 < fb < dec
        else:
            assert fb == dec > 0
        assert a.stats()["exited"] == b.stats()["exited"]


def test_tick_decisions_on_the_candidate_composition_match_the_lattice_surrogate_field():
    """A surrogate tick composes F_sur at each pedestrian's candidates instead
    of over the lattice.  With delta = 0 (only margins within FP32 rounding
    fall back) its decisions equal the oracle's decisions on the lattice
    surrogate field of sfm_surrogate_field, wherever the oracle's best two
    energies are apart by more than FP32 rounding."""
    sc = SG.random_scene(400, 320, 6000, r=20, seed=131, obstacles=5, exits=("east",),
                         goal_mode="mixed", heading_mode="random")
    init = sfm.flatten_params(_rounded_params(5))
    with sfm.Sim(sc) as sim, sfm.Surrogate(coarsen=8, near_radius=3, params=init) as sur:
        sim.step(2)
        xy, hd, al = sim.peds()
        F = sur.field(sim).astype(np.float64)
        D = sim.guidance()
        m = O.model(sc)
        occ, bad = O.occupancy(m, sc.cell, xy, al)
        assert bad == 0
        ch_o, E, _, adm = O.decide(m, sc.cell, occ, xy, hd, sc.goal, al, D, Ffull=F,
                                   Sfull=np.abs(F))
        sur.set_delta(0.0)
        sur.step(sim, 1)
        ch, _ = sim.decisions()
    live = al.astype(bool)
    Ea = np.where(adm.astype(bool), E, np.inf)
    two = np.sort(Ea, axis=1)[:, :2]
    with np.errstate(invalid="ignore"):  # dead pedestrians: no admissible candidate
        margin = two[:, 1] - two[:, 0]
    clear = live & (margin > 1e-5 * (np.abs(two[:, 0]) + 1.0))
    assert clear.sum() > 0.9 * live.sum()
    np.testing.assert_array_equal(ch[clear], ch_o[clear])


def test_calibrated_delta_meets_the_flip_target_and_zero_delta_only_ties():
    """A calibrated delta (99th percentile of the candidate error spread) keeps
    the decision flip rate within 0.1% while part of the crowd is decided on
    the surrogate alone; delta = 0 re-decides only margins within rounding,
    so it cannot flip more than the surrogate alone."""
    sc = SG.random_scene(512, 512, 6000, r=20, seed=121, obstacles=6, exits=("east", "west"),
                         goal_mode="mixed", heading_mode="random")
    init = sfm.flatten_params(_rounded_params(5))
    with sfm.Sim(sc) as sim, sfm.Surrogate(coarsen=8, near_radius=3, params=init) as sur:
        sim.step(2)
        d = sur.calibrate(sim, 0.99)
        assert 0.0 < d < np.inf
        sim.step(2)
        ev = sur.eval(sim)
        assert ev["decided"] > 5000
        assert ev["flip_rate"] <= 1e-3, ev
        assert ev["fallback_rate"] < 1.0, ev
        assert ev["flip_rate"] <= ev["flip_rate_raw"]
        sur.set_delta(0.0)
        ev0 = sur.eval(sim)
        assert ev0["fallback_rate"] <= ev["fallback_rate"]
        assert ev0["flip_rate"] <= ev0["flip_rate_raw"]
        with pytest.raises(sfm.SfmError):
            sur.set_delta(-1.0)


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
    assert after["flip_rate_raw"] < trunc["flip_rate_raw"], (trunc, after)
