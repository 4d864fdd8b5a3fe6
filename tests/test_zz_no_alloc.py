"""The allocation-free field entry point (sfm_field_noalloc) on the GPU.

sfm_field_noalloc serves callers that cannot allocate device memory while
they run (a host that reserves all device memory up front in its own pool);
its working memory is a fixed device array inside the library.  This test
calls it through the C ABI twice in a row, on different crowds, and checks
each result against the context path's field (sfm_create / sfm_place /
sfm_compute_field), within the field tolerance of the other parity tests
(1e-5 of the sum of term magnitudes at each su, from the FP64 oracle).  The
file is collected last so that a run stopping at the first failure has run
every other test first.
"""
import numpy as np
import pytest

import oracle as O
import paper_1803_04782_gb300 as sfm
import scenegen as SG
from paper_1803_04782_gb300 import build as B

pytestmark = pytest.mark.gpu


def _context_field(sc):
    with sfm.Sim(sc) as sim:
        sim.compute_field()
        return sim.field(), sim.static_field()


def _oracle_S(sc, alive=None):
    m = O.model(sc)
    occ, bad = O.occupancy(m, sc.cell, sc.xy, alive)
    assert bad == 0
    return O.field(m, sc.cell, occ, sc.heading)[1]


def test_field_noalloc_matches_context_field_on_two_calls():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    B.build()
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    first = SG.random_scene(300, 220, 3000, r=12, seed=501, periodic_x=1, exits=("south",),
                            obstacles=3, goal_mode="mixed", heading_mode="random")
    second = SG.random_scene(300, 220, 800, r=40, seed=502, exits=("east", "north"),
                             obstacles=5, heading_mode="random")
    stream = torch.cuda.current_stream()
    for sc in (first, second):
        F_ctx, Fs = _context_field(sc)
        S = _oracle_S(sc)
        lat = sfm.Lattice(sc.W, sc.H, sc.periodic_x, sc.periodic_y)
        prm = sfm.make_params(**sc.params)
        xy = torch.from_numpy(np.ascontiguousarray(sc.xy, np.int32)).to(dev)
        hd = torch.from_numpy(np.ascontiguousarray(sc.heading, np.uint8)).to(dev)
        base = torch.from_numpy(Fs).to(dev)
        out = torch.full((sc.H, sc.W), float("nan"), dtype=torch.float32, device=dev)
        st = sfm.sfm_field_noalloc(lat, prm, xy, hd, None, base, out, stream)
        assert st == sfm.SFM_OK
        F = out.cpu().numpy()
        assert np.isfinite(F).all()
        diff = np.abs(F.astype(np.float64) - F_ctx.astype(np.float64))
        assert (diff <= 1e-5 * S + 1e-30).all(), float(np.max(diff / np.maximum(S, 1e-300)))


def test_field_noalloc_rejects_sizes_beyond_its_limits():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    B.build()
    dev = torch.device("cuda", 0)
    base = torch.zeros((64, 64), dtype=torch.float32, device=dev)
    out = torch.zeros_like(base)
    xy = torch.zeros((4, 2), dtype=torch.int32, device=dev)
    lat = sfm.Lattice(64, 64, 0, 0)
    assert sfm.sfm_field_noalloc(lat, sfm.make_params(r=sfm.SFM_NOALLOC_MAX_RADIUS + 1), xy, None,
                                 None, base, out) == sfm.SFM_EINVAL
    big = sfm.Lattice(32 * 257, 32 * 256, 0, 0)   # 65792 bins > SFM_NOALLOC_MAX_BINS
    assert sfm.sfm_field_noalloc(big, sfm.make_params(r=3), xy, None, None, base,
                                 out) == sfm.SFM_EINVAL
    many = torch.zeros((sfm.SFM_NOALLOC_MAX_PEDS + 1, 2), dtype=torch.int32, device=dev)
    assert sfm.sfm_field_noalloc(lat, sfm.make_params(r=3), many, None, None, base,
                                 out) == sfm.SFM_EINVAL
    # a pedestrian outside the lattice is reported, not written anywhere
    bad = torch.tensor([[3, 3], [64, 5]], dtype=torch.int32, device=dev)
    assert sfm.sfm_field_noalloc(lat, sfm.make_params(r=3), bad, None, None, base,
                                 out) == sfm.SFM_ECONFLICT
