"""The allocation-free field entry point (sfm_field_noalloc) on the GPU.

sfm_field_noalloc serves callers that cannot allocate device memory while
they run (a host that reserves all device memory up front in its own pool);
its working memory is a fixed device array inside the library.  This test
calls it through the C ABI three times in a row, on different crowds, and
checks each result against the context path's field (sfm_create / sfm_place /
sfm_compute_field) and the FP64 oracle's, within the field tolerance of the
other parity tests (1e-5 of the sum of term magnitudes at each su), and that
the device's free memory is the same before and after a call once its
kernels are loaded.  The file is collected last so that a run stopping at
the first failure has run every other test first.
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


def _oracle_field(sc, alive=None):
    m = O.model(sc)
    occ, bad = O.occupancy(m, sc.cell, sc.xy, alive)
    assert bad == 0
    return O.field(m, sc.cell, occ, sc.heading)


def _noalloc(torch, dev, sc, stream, Fs):
    lat = sfm.Lattice(sc.W, sc.H, sc.periodic_x, sc.periodic_y)
    prm = sfm.make_params(**sc.params)
    xy = torch.from_numpy(np.ascontiguousarray(sc.xy, np.int32)).to(dev)
    hd = torch.from_numpy(np.ascontiguousarray(sc.heading, np.uint8)).to(dev)
    base = torch.from_numpy(Fs).to(dev)
    out = torch.full((sc.H, sc.W), float("nan"), dtype=torch.float32, device=dev)
    return lat, prm, xy, hd, base, out


def test_field_noalloc_matches_context_field_on_calls_in_a_row():
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
    # a third crowd on the first lattice, radius and kernels: its call runs
    # only kernels the first call already loaded, so the device's free memory
    # must not change across it
    third = SG.random_scene(300, 220, 2500, r=12, seed=503, periodic_x=1, exits=("south",),
                            obstacles=3, goal_mode="mixed", heading_mode="random")
    stream = torch.cuda.current_stream()
    for k, sc in enumerate((first, second, third)):
        F_ctx, Fs = _context_field(sc)
        Fo, S = _oracle_field(sc)
        lat, prm, xy, hd, base, out = _noalloc(torch, dev, sc, stream, Fs)
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info(dev)[0]
        st = sfm.sfm_field_noalloc(lat, prm, xy, hd, None, base, out, stream)
        torch.cuda.synchronize()
        free1 = torch.cuda.mem_get_info(dev)[0]
        assert st == sfm.SFM_OK
        if k == 2:
            assert free1 == free0, f"device free memory changed by {free0 - free1} bytes"
        F = out.cpu().numpy()
        assert np.isfinite(F).all()
        # against the existing entry point (context path) and the FP64 oracle
        tol = 1e-5 * S + 1e-30
        diff = np.abs(F.astype(np.float64) - F_ctx.astype(np.float64))
        assert (diff <= tol).all(), float(np.max(diff / np.maximum(S, 1e-300)))
        diff_o = np.abs(F.astype(np.float64) - Fo)
        assert (diff_o <= tol).all(), float(np.max(diff_o / np.maximum(S, 1e-300)))


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
    big_base = torch.zeros((big.H, big.W), dtype=torch.float32, device=dev)
    assert sfm.sfm_field_noalloc(big, sfm.make_params(r=3), xy, None, None, big_base,
                                 torch.empty_like(big_base)) == sfm.SFM_EINVAL
    del big_base
    many = torch.zeros((sfm.SFM_NOALLOC_MAX_PEDS + 1, 2), dtype=torch.int32, device=dev)
    assert sfm.sfm_field_noalloc(lat, sfm.make_params(r=3), many, None, None, base,
                                 out) == sfm.SFM_EINVAL
    # arguments the bare C pointers cannot describe are refused by the binding
    for bad_args in (
            dict(xy=xy.cpu()),                                  # host memory
            dict(xy=xy.to(torch.int64)),                        # wrong dtype
            dict(xy=xy.reshape(-1)),                            # wrong shape
            dict(heading=torch.zeros(3, dtype=torch.uint8, device=dev)),  # short
            dict(heading=torch.zeros(4, dtype=torch.int32, device=dev)),  # dtype
            dict(alive=torch.zeros(5, dtype=torch.uint8, device=dev)),    # long
            dict(base=base[:32]),                               # too few su
            dict(field=torch.zeros((64, 64), dtype=torch.float64, device=dev)),
            dict(field=out.cpu())):
        kw = dict(xy=xy, heading=None, alive=None, base=base, field=out)
        kw.update(bad_args)
        with pytest.raises(ValueError):
            sfm.sfm_field_noalloc(lat, sfm.make_params(r=3), **kw)
    # a pedestrian outside the lattice is reported, not written anywhere
    bad = torch.tensor([[3, 3], [64, 5]], dtype=torch.int32, device=dev)
    assert sfm.sfm_field_noalloc(lat, sfm.make_params(r=3), bad, None, None, base,
                                 out) == sfm.SFM_ECONFLICT
