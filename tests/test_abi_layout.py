"""Host side of the C ABI, no GPU: the ctypes structures of the Python binding have the layout
the C compiler gives the structures of include/mpmrom.h (size and every field offset), and
the create calls reject invalid configurations with MPM_EINVAL and a message before they touch
the device."""
import ctypes as C
import os
import shutil
import subprocess

import pytest

from paper_2109_12390_gb300 import _abi

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

STRUCTS = [("mpm_config", _abi.MpmConfig), ("decoder_desc", _abi.DecoderDesc), ("rom_config", _abi.RomConfig),
           ("snapshot_desc", _abi.SnapshotDesc), ("train_config", _abi.TrainConfig)]


@pytest.fixture(scope="module")
def c_layout(tmp_path_factory):
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    d = tmp_path_factory.mktemp("layout")
    lines = ["#include <stddef.h>", "#include <stdio.h>", '#include "mpmrom.h"', "int main(void) {"]
    for cname, py in STRUCTS:
        lines.append(f'  printf("{cname} . %zu\\n", sizeof({cname}));')
        for fname, _ in py._fields_:
            lines.append(f'  printf("{cname} {fname} %zu\\n", offsetof({cname}, {fname}));')
    lines += ["  return 0;", "}"]
    src = d / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = d / "layout"
    subprocess.run([cc, "-std=c11", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"), str(src), "-o",
                    str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout
    table = {}
    for line in out.splitlines():
        s, f, v = line.split()
        table[(s, f)] = int(v)
    return table


@pytest.mark.parametrize("cname,py", STRUCTS, ids=[s for s, _ in STRUCTS])
def test_ctypes_layout_matches_header(c_layout, cname, py):
    assert C.sizeof(py) == c_layout[(cname, ".")]
    for fname, _ in py._fields_:
        assert getattr(py, fname).offset == c_layout[(cname, fname)], fname


def test_header_field_sets_match():
    """Every field of each header struct is bound (a field missing from ctypes would shift
    nothing if it were last, so compare the field lists parsed from the header too)."""
    import re
    txt = open(os.path.join(ROOT, "include", "mpmrom.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    for cname, py in STRUCTS:
        body = re.search(r"typedef struct %s \{(.*?)\} %s;" % (cname, cname), txt, re.S).group(1)
        fields = [re.search(r"([A-Za-z_][A-Za-z0-9_]*)\s*(\[\d+\])?$", decl.strip()).group(1)
                  for decl in body.split(";") if decl.strip()]
        assert fields == [f for f, _ in py._fields_], cname


@pytest.fixture(scope="module")
def lib():
    from paper_2109_12390_gb300.build import build
    build()
    return _abi.lib()


def _mpm_cfg(**kw):
    E = (C.c_float * 1)(1e4)
    nu = (C.c_float * 1)(0.3)
    off = (C.c_int64 * 2)(0, 64)
    cfg = _abi.MpmConfig(dim=2, n_grid=64, dx=1 / 64, dt=1e-4, bc=0, bc_width=3, material=0, transfer=0,
                         rho=1.0, p_vol=1e-4, n_inst=1, E=E, nu=nu, inst_offsets=off)
    for k, v in kw.items():
        setattr(cfg, k, v)
    return cfg, (E, nu, off)


@pytest.mark.parametrize("field,value,needle", [
    ("dim", 4, "dim"), ("n_grid", 60, "n_grid"), ("dt", 0.0, "dt"), ("material", 9, "material"),
    ("transfer", 5, "transfer"), ("polar_eft", 2, "polar_eft"), ("bc_width", -1, "bc_width"),
])
def test_mpm_init_rejects_invalid_config(lib, field, value, needle):
    cfg, keep = _mpm_cfg(**{field: value})
    out = C.c_void_p()
    st = lib.mpm_init(C.byref(cfg), C.byref(out))
    assert st == _abi.MPM_EINVAL and not out.value
    assert needle in lib.mpm_last_error().decode()


def test_mpm_init_rejects_decreasing_offsets_and_plastic_bounds(lib):
    cfg, keep = _mpm_cfg()
    keep[2][1] = 0
    out = C.c_void_p()
    assert lib.mpm_init(C.byref(cfg), C.byref(out)) == _abi.MPM_EINVAL
    cfg, keep = _mpm_cfg(material=2, plastic_compression=1.5, plastic_stretch=0.01)
    assert lib.mpm_init(C.byref(cfg), C.byref(out)) == _abi.MPM_EINVAL
    assert "plastic" in lib.mpm_last_error().decode()



@pytest.mark.parametrize("E,nu", [(0.0, 0.3), (1e4, 0.5), (1e4, -1.0), (float("nan"), 0.3)])
def test_mpm_init_rejects_invalid_material_before_allocating(lib, E, nu):
    cfg, keep = _mpm_cfg()
    keep[0][0], keep[1][0] = E, nu
    out = C.c_void_p()
    assert lib.mpm_init(C.byref(cfg), C.byref(out)) == _abi.MPM_EINVAL and not out.value
    assert "E must be" in lib.mpm_last_error().decode()


@pytest.mark.parametrize("desc,needle", [
    (dict(d=4, r=8, width=128, n_hidden=3, activation=0), "d must be"),
    (dict(d=2, r=40, width=128, n_hidden=3, activation=0), "d + r"),
    (dict(d=2, r=8, width=64, n_hidden=3, activation=0), "width"),
    (dict(d=2, r=8, width=128, n_hidden=7, activation=0), "hidden"),
    (dict(d=2, r=8, width=128, n_hidden=3, activation=3), "activation"),
])
def test_decoder_create_rejects_invalid_desc(lib, desc, needle):
    out = C.c_void_p()
    st = lib.decoder_create(C.byref(_abi.DecoderDesc(**desc)), C.byref(out))
    assert st == _abi.MPM_EINVAL and not out.value
    assert needle in lib.mpm_last_error().decode()


def test_null_arguments_are_rejected(lib):
    out = C.c_void_p()
    assert lib.mpm_init(None, C.byref(out)) == _abi.MPM_EINVAL
    assert lib.decoder_create(None, C.byref(out)) == _abi.MPM_EINVAL
    assert lib.rom_create(C.byref(_abi.RomConfig()), None, None, 0, C.byref(out)) == _abi.MPM_EINVAL
    assert lib.trainer_create(None, None, None, None, C.byref(out)) == _abi.MPM_EINVAL
    assert "null" in lib.mpm_last_error().decode()
