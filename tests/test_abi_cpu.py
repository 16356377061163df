"""CPU-side checks of the C ABI: the library builds and loads, exports every
function include/nb.h declares, and the host-only calls validate arguments.
No kernel runs here."""
import ctypes
import os
import re
import shutil

import pytest

from paper_1506_00716_gb300 import build as nbbuild
from paper_1506_00716_gb300 import nb
from paper_1506_00716_gb300 import waterbox as wb

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "nb.h")


def _declared():
    txt = open(HEADER).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(nb_[a-z_]+)\s*\(", txt)))


@pytest.fixture(scope="module")
def lib():
    if shutil.which(nbbuild.NVCC) is None and not os.path.exists(nbbuild.LIB):
        pytest.skip("nvcc not available")
    nbbuild.build()
    return nb.load()


def test_exports_every_declared_function(lib):
    declared = _declared()
    assert len(declared) >= 19
    assert sorted(nb.EXPORTS) == declared
    for name in declared:
        assert getattr(lib, name) is not None


def test_params_struct_layout_matches_header():
    # double rc, rlist; int coul; double eps_r, eps_rf, ewald_beta, fcoul; int ntypes; 2 pointers
    assert ctypes.sizeof(nb.nb_params) == 8 * 2 + 8 + 8 * 4 + 8 + 8 * 2
    assert ctypes.sizeof(nb.nb_list_info) == 5 * 8


def test_footprint_validates_arguments(lib):
    p = wb.params_rf()
    box = [3.0, 3.0, 3.0]
    assert nb.nb_sys_footprint(p, 1944, box) > 1944 * 56
    with pytest.raises(nb.NbError) as e:
        nb.nb_sys_footprint(p, 0, box)
    assert e.value.status == 1
    with pytest.raises(nb.NbError) as e:
        nb.nb_sys_footprint(p, 100, [2.0, 3.0, 3.0])  # edge < 2 * rlist
    assert e.value.status == 2
    bad = wb.params_rf()
    bad.rlist = 0.9  # below rc
    with pytest.raises(nb.NbError) as e:
        nb.nb_sys_footprint(bad, 100, box)
    assert e.value.status == 1
    bad = wb.params_rf()
    bad.ntypes = 65
    with pytest.raises(nb.NbError):
        nb.nb_sys_footprint(bad, 100, box)


def test_footprint_grows_with_atoms(lib):
    p = wb.params_rf()
    small = nb.nb_sys_footprint(p, 24000, [6.21] * 3)
    large = nb.nb_sys_footprint(p, 3_000_000, [31.0] * 3)
    assert 100 * small < large < 200 * small
