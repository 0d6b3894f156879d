"""CPU checks of the C ABI: the library builds for sm_103a, loads, and exports
every symbol include/icrs.h declares; struct layouts match the header."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def libmod():
    from paper_2510_02639_gb300 import build as B
    B.build()
    from paper_2510_02639_gb300 import icrs
    return icrs


def declared_functions():
    src = open(os.path.join(ROOT, "include", "icrs.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(icrs_[a-z0-9_]+)\s*\(", src)))


def test_header_symbols_exported(libmod):
    names = declared_functions()
    assert names, "no functions found in the header"
    assert set(names) == set(libmod.EXPORTED)
    for n in names:
        assert hasattr(libmod.lib, n), n


def test_struct_layouts(libmod, tmp_path):
    """The binding's ctypes structs have the header's field offsets and sizes
    (a C program compiled against include/icrs.h prints them)."""
    import subprocess
    inc = os.path.join(ROOT, "include")
    src = tmp_path / "layout.c"
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "icrs.h"', "int main(void) {"]
    for st, cls in (("icrs_params", libmod.IcrsParams), ("icrs_grid", libmod.IcrsGrid)):
        lines.append(f'printf("{st} size %zu\\n", sizeof({st}));')
        for f, _ in cls._fields_:
            lines.append(f'printf("{st} {f} %zu\\n", offsetof({st}, {f}));')
    lines += ["return 0;", "}"]
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", inc, str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    got = {tuple(l.split()[:2]): int(l.split()[2]) for l in out if l.strip()}
    for st, cls in (("icrs_params", libmod.IcrsParams), ("icrs_grid", libmod.IcrsGrid)):
        assert got[(st, "size")] == ctypes.sizeof(cls), st
        for f, _ in cls._fields_:
            assert got[(st, f)] == getattr(cls, f).offset, (st, f)
    assert ctypes.sizeof(libmod.IcrsParams) == libmod.PARAMS_DTYPE.itemsize == 23 * 8
    g = libmod.make_grid()
    assert (g.n_r, g.n_theta, g.n_limb, g.n_bins_r, g.n_bins_theta) == (64, 256, 500, 32, 128)
    assert abs(g.delta_c - 0.02) < 1e-15 and abs(g.margin - 0.05) < 1e-15


def test_strerror_and_version(libmod):
    assert libmod.lib.icrs_abi_version() == 3
    for c in range(5):
        assert libmod.lib.icrs_strerror(c)


def test_invalid_arguments_rejected_without_gpu(libmod):
    # argument checks run before any CUDA call
    g = libmod.make_grid(n_r=0)
    rc = libmod.lib.icrs_magnification(ctypes.c_void_p(1), 1, ctypes.c_void_p(1), 1,
                                       ctypes.byref(g), ctypes.c_void_p(1), None, None)
    assert rc == libmod.ICRS_EINVAL
    g = libmod.make_grid()
    rc = libmod.lib.icrs_magnification(None, 1, None, 1, ctypes.byref(g), None, None, None)
    assert rc == libmod.ICRS_EINVAL
    # empty problem: nothing to do
    rc = libmod.lib.icrs_magnification(ctypes.c_void_p(1), 0, ctypes.c_void_p(1), 5,
                                       ctypes.byref(g), ctypes.c_void_p(1), None, None)
    assert rc == libmod.ICRS_OK


def test_product_path_has_no_oracle_import():
    pkg = os.path.join(ROOT, "paper_2510_02639_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
                txt = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in txt and "from oracle" not in txt, f
                assert "icrs_oracle" not in txt, f


def header_defines():
    src = open(os.path.join(ROOT, "include", "icrs.h")).read()
    d = {k: v for k, v in re.findall(r"#define\s+(ICRS_[A-Z0-9_]+)\s+([0-9.eE+-]+)u?\b", src)}
    d.update({k: str(1 << int(n)) for k, n in re.findall(r"#define\s+(ICRS_[A-Z0-9_]+)\s+\(1u << (\d+)\)", src)})
    return d


def test_status_bits_and_constants_agree(libmod):
    """The binding's and the oracle's status bits, MLP sizes and roughness
    threshold carry the header's values (each side defines its own)."""
    from oracle import mlp as M
    d = header_defines()
    for name in ("NONCONV", "IMGCOUNT", "SECTCAP", "EDGE", "NAN", "OVERFLOW", "LIMB", "ROUGH", "SPOT", "PROFILE"):
        assert int(d["ICRS_ST_" + name]) == getattr(libmod, "ST_" + name), name
    assert int(d["ICRS_ST_LIMB"]) == M.ST_LIMB and int(d["ICRS_ST_ROUGH"]) == M.ST_ROUGH
    assert int(d["ICRS_ST_SPOT"]) == M.ST_SPOT and int(d["ICRS_ST_PROFILE"]) == M.ST_PROFILE
    assert float(d["ICRS_ROUGH_MAX"]) == M.ROUGH_MAX
    assert int(d["ICRS_MLP_NPARAM"]) == libmod.MLP_NPARAM == M.N_PARAMS
    assert int(d["ICRS_MLP_PACK_BYTES"]) == libmod.MLP_PACK_BYTES
