"""CPU-side checks of the C ABI: the library builds and loads, exports every
function include/nb.h declares, and the host-only calls validate arguments.
No kernel runs here."""
import ctypes
import os
import re
import shutil
import subprocess

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


def test_params_struct_layout_matches_header(tmp_path):
    """The binding's structs have the C compiler's layout of include/nb.h."""
    src = tmp_path / "layout.c"
    src.write_text(
        '#include <stddef.h>\n#include <stdio.h>\n#include "nb.h"\n'
        "#define F(s, m) printf(#s \" \" #m \" %zu\\n\", offsetof(s, m))\n"
        "int main(void) {\n"
        '  printf("nb_params size %zu\\n", sizeof(nb_params));\n'
        "  F(nb_params, rc); F(nb_params, rlist); F(nb_params, coul); F(nb_params, eps_r);\n"
        "  F(nb_params, eps_rf); F(nb_params, ewald_beta); F(nb_params, fcoul); F(nb_params, ntypes);\n"
        "  F(nb_params, c6); F(nb_params, c12); F(nb_params, modifiers);\n"
        '  printf("nb_tuning size %zu\\n", sizeof(nb_tuning));\n'
        '  printf("nb_request_stats size %zu\\n", sizeof(nb_request_stats));\n'
        '  printf("nb_list_info size %zu\\n", sizeof(nb_list_info));\n'
        '  printf("nb_pme_params size %zu\\n", sizeof(nb_pme_params));\n'
        "  F(nb_pme_params, grid); F(nb_pme_params, order);\n"
        "  return 0;\n}\n")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    got = {" ".join(line.split()[:2]): int(line.split()[2]) for line in out if line.strip()}
    assert got["nb_params size"] == ctypes.sizeof(nb.nb_params)
    for name, _ in nb.nb_params._fields_:
        assert got[f"nb_params {name}"] == getattr(nb.nb_params, name).offset, name
    assert got["nb_tuning size"] == ctypes.sizeof(nb.nb_tuning)
    assert got["nb_request_stats size"] == ctypes.sizeof(nb.nb_request_stats)
    assert got["nb_list_info size"] == ctypes.sizeof(nb.nb_list_info) == 6 * 8
    assert got["nb_pme_params size"] == ctypes.sizeof(nb.nb_pme_params) == 16
    assert got["nb_pme_params order"] == nb.nb_pme_params.order.offset


def test_modifiers_are_validated(lib):
    box = [3.0, 3.0, 3.0]
    ok = [(wb.COUL_RF, nb.NB_MOD_LJ_SHIFT | nb.NB_MOD_RF_EXCL),
          (wb.COUL_EWALD, nb.NB_MOD_LJ_SHIFT | nb.NB_MOD_EWALD_SHIFT)]
    for coul, mods in ok:
        assert nb.nb_sys_footprint(wb.Params(coul=coul, modifiers=mods), 1944, box) > 0
    bad = [(wb.COUL_RF, nb.NB_MOD_EWALD_SHIFT), (wb.COUL_EWALD, nb.NB_MOD_RF_EXCL), (wb.COUL_RF, 8)]
    for coul, mods in bad:
        with pytest.raises(nb.NbError) as e:
            nb.nb_sys_footprint(wb.Params(coul=coul, modifiers=mods), 1944, box)
        assert e.value.status == 1  # NB_ERR_ARG


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


def test_null_handles_are_refused_without_device_work(lib):
    """The list exports and the tuning calls refuse a NULL handle with
    NB_ERR_ARG before touching the device (here, where there is none)."""
    n = ctypes.c_longlong()
    assert lib.nb_pairlist_export(None, None, None, None, None, ctypes.byref(n)) == 1
    assert lib.nb_pairlist_export_slots(None, None, None, None, None, ctypes.byref(n)) == 1
    t = nb.nb_tuning(32, 3, 0, 0, 4)
    assert lib.nb_ctx_set_tuning(None, ctypes.byref(t)) == 1
    assert lib.nb_ctx_get_tuning(None, ctypes.byref(t)) == 1
