"""Host-side checks of the C ABI (no GPU needed): the library builds, loads,
exports every entry point include/sfm.h declares, and the binding's struct
layouts match the header's."""
import ctypes as C
import os
import re
import subprocess

import pytest

import paper_1803_04782_gb300 as sfm
from paper_1803_04782_gb300 import build as B

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "sfm.h")


@pytest.fixture(scope="module")
def libpath():
    return B.build()


def _declared():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(sfm_[a-z_]+)\s*\(", src)))


def test_library_exports_every_declared_entry_point(libpath):
    names = _declared()
    assert len(names) >= 18
    L = C.CDLL(libpath)
    for n in names:
        assert hasattr(L, n), n
    assert sorted(sfm.EXPORTS) == names
    out = subprocess.run(["nm", "-D", "--defined-only", libpath], capture_output=True, text=True)
    exported = set(re.findall(r" T (sfm_\w+)", out.stdout))
    assert exported == set(names)


def test_binding_loads_and_reports_version(libpath):
    assert sfm.lib() is not None
    assert sfm.sfm_abi_version() == 5


def test_struct_layouts_match_header(tmp_path):
    prog = tmp_path / "layout.c"
    prog.write_text(
        '#include <stdio.h>\n#include <stddef.h>\n#include "sfm.h"\n'
        "int main(void){printf(\"%zu %zu %zu %zu %zu %zu %zu\\n\", sizeof(sfm_lattice),"
        " sizeof(sfm_params), offsetof(sfm_params, seed), offsetof(sfm_params, hbm_budget_bytes),"
        " sizeof(sfm_stats_t), offsetof(sfm_stats_t, error_flags),"
        " offsetof(sfm_stats_t, device_bytes)); return 0;}\n")
    exe = tmp_path / "layout"
    subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), str(prog), "-o", str(exe)])
    got = [int(v) for v in subprocess.check_output([str(exe)]).split()]
    want = [C.sizeof(sfm.Lattice), C.sizeof(sfm.Params), sfm.Params.seed.offset,
            sfm.Params.hbm_budget_bytes.offset, C.sizeof(sfm.Stats),
            sfm.Stats.error_flags.offset, sfm.Stats.device_bytes.offset]
    assert got == want


def test_surrogate_struct_layouts_match_header(tmp_path):
    prog = tmp_path / "slayout.c"
    prog.write_text(
        '#include <stdio.h>\n#include <stddef.h>\n#include "sfm.h"\n'
        "int main(void){printf(\"%zu %zu %zu %zu %zu\\n\", sizeof(sfm_surrogate_cfg),"
        " offsetof(sfm_surrogate_cfg, taper_inner), sizeof(sfm_surrogate_report),"
        " offsetof(sfm_surrogate_report, delta), offsetof(sfm_surrogate_report, decided));"
        " return 0;}\n")
    exe = tmp_path / "slayout"
    subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), str(prog), "-o", str(exe)])
    got = [int(v) for v in subprocess.check_output([str(exe)]).split()]
    want = [C.sizeof(sfm.SurrogateCfg), sfm.SurrogateCfg.taper_inner.offset,
            C.sizeof(sfm.SurrogateReport), sfm.SurrogateReport.delta.offset,
            sfm.SurrogateReport.decided.offset]
    assert got == want


def test_params_helper_round_trips():
    p = sfm.make_params(r=40, seed=2**64 - 1, hbm_budget_bytes=5 << 30)
    assert p.r == 40 and p.seed == 2**64 - 1 and p.hbm_budget_bytes == 5 << 30
    assert p.kP == 1.0 and p.aP == -0.5 and p.kE == -1.0


def test_create_rejects_bad_arguments_before_touching_the_gpu():
    import numpy as np
    cell = np.zeros((10, 10), np.uint8)
    cases = [
        (dict(W=2, H=10), dict(r=1), "3x3"),
        (dict(W=10, H=10), dict(r=65), "radius"),
        (dict(W=10, H=10, periodic_x=1), dict(r=5), "2r+1"),
        (dict(W=10, H=10), dict(r=2, bin=16), "bin"),
    ]
    for lat, prm, msg in cases:
        L = sfm.Lattice(lat["W"], lat["H"], lat.get("periodic_x", 0), 0)
        with pytest.raises(sfm.SfmError) as e:
            sfm.sfm_create(L, cell, sfm.make_params(**prm))
        assert e.value.status == sfm.SFM_EINVAL
        assert msg in str(e.value)


def test_resident_bytes_and_band_budget():
    lat = sfm.Lattice(100, 77, 0, 0)
    assert sfm.sfm_resident_bytes(lat) == 100 * 77 * 13 + 128 * 77
    lat = sfm.Lattice(16384, 16384, 0, 0)
    assert sfm.sfm_resident_bytes(lat) == 16384 * 16384 * 14
    assert sfm.band_budget(16384, 16384, 4096) == 16384 * 16384 * 14 + 4 * 16384 * (4096 + 33)


def test_snapshot_calls_reject_null_without_a_gpu():
    import ctypes as C
    n = C.c_size_t(0)
    assert sfm.lib().sfm_snapshot(None, None, C.byref(n)) == sfm.SFM_EINVAL
    assert sfm.lib().sfm_restore(None, None, 0) == sfm.SFM_EINVAL


def test_create_refuses_a_budget_too_small_before_allocating():
    """Failure injection on the host: an HBM budget below the resident arrays,
    or leaving room for fewer than 32 field rows, is SFM_EBUDGET."""
    import numpy as np
    cell = np.zeros((200, 300), np.uint8)
    L = sfm.Lattice(300, 200, 0, 0)
    resident = sfm.sfm_resident_bytes(L)
    for budget, msg in ((resident - 1, "resident arrays"),
                        (resident + 4 * 300 * 20, "fewer than 32 field rows")):
        with pytest.raises(sfm.SfmError) as e:
            sfm.sfm_create(L, cell, sfm.make_params(r=3, hbm_budget_bytes=budget))
        assert e.value.status == sfm.SFM_EBUDGET
        assert msg in str(e.value)
