"""Host-side checks of the C ABI (no GPU needed): the library builds for
sm_103a, loads, exports every entry point declared in include/goc.h, and the
ctypes mirror of each struct has the size and field offsets of the C header."""
import ctypes
import os
import re
import subprocess

import pytest

import paper_2607_15362_b300 as goc
from paper_2607_15362_b300 import _abi

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "goc.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(goc_[a-z_]+)\s*\(", text)))


def test_library_exports_every_declared_entry_point():
    lib = goc.lib()
    names = declared_functions()
    assert len(names) >= 20
    for n in names:
        assert hasattr(lib, n), n
    assert set(names) == set(_abi.SIGNATURES), set(names) ^ set(_abi.SIGNATURES)


def test_library_is_built_for_sm_103a():
    import importlib
    b = importlib.import_module("paper_2607_15362_b300.build")
    assert "arch=compute_103a,code=sm_103a" in b.NVCC_FLAGS
    assert os.path.exists(goc.build())


@pytest.mark.parametrize("name,cls", [("goc_grid", _abi.GocGrid), ("goc_map", _abi.GocMap),
                                      ("goc_flow", _abi.GocFlow), ("goc_mhd", _abi.GocMhd),
                                      ("goc_exec", _abi.GocExec)])
def test_ctypes_structs_match_the_header(tmp_path, name, cls):
    fields = [f[0] for f in cls._fields_]
    src = tmp_path / "probe.c"
    body = "\n".join(f'printf("%zu ", offsetof({name}, {f}));' for f in fields)
    src.write_text(f'#include <stdio.h>\n#include <stddef.h>\n#include "{HEADER}"\n'
                   f'int main(void){{ printf("%zu ", sizeof({name})); {body} return 0; }}\n')
    exe = tmp_path / "probe"
    subprocess.run(["gcc", "-o", str(exe), str(src)], check=True)
    got = [int(x) for x in subprocess.run([str(exe)], capture_output=True, text=True).stdout.split()]
    want = [ctypes.sizeof(cls)] + [getattr(cls, f).offset for f in fields]
    assert got == want


def test_errors_are_reported_without_a_device_call():
    """Invalid arguments are rejected on the host with a message."""
    lib = goc.lib()
    g, m, f, h = goc.structs_from_spec({"nx": 2, "ny": 8, "walls": {"W": {"u": 0}, "E": {"u": 0},
                                                                     "S": None, "N": None}})
    out = ctypes.c_void_p()
    st = lib.goc_create(ctypes.byref(g), ctypes.byref(m), ctypes.byref(f), ctypes.byref(h), None, ctypes.byref(out))
    assert st == _abi.GOC_EINVAL
    assert b"3 nodes" in lib.goc_last_error()
    assert lib.goc_step(None, 1) == _abi.GOC_EINVAL
    lib.goc_destroy(None)


def test_standard_scheme_rejects_stretched_maps_without_a_gpu():
    """goc_create validates scheme 1 before touching the device."""
    import goc_inputs as gi
    from paper_2607_15362_b300.lattice import structs_from_spec, _exec

    prob = gi.Problem("cavity", 16, 16, {"kind": "tanh2", "beta": 1.5}, {"kind": "uniform"}, {"Re": 10.0, "u_lid": 0.05})
    spec = prob.lattice_spec(0.01)
    spec["gi"] = 0
    g, m, f, h = structs_from_spec(spec)
    e = _exec("fp32", None, 100, "stochastic", "standard")
    out = ctypes.c_void_p()
    st = _abi.lib().goc_create(ctypes.byref(g), ctypes.byref(m), ctypes.byref(f), ctypes.byref(h),
                               ctypes.byref(e), ctypes.byref(out))
    assert st == _abi.GOC_EINVAL and not out.value
    assert b"uniform maps" in _abi.lib().goc_last_error()
    spec2 = gi.Problem("cavity", 16, 16, {"kind": "uniform"}, {"kind": "uniform"}, {"Re": 10.0, "u_lid": 0.05}).lattice_spec(1 / 3)
    g, m, f, h = structs_from_spec(spec2)          # gi defaults to 1
    st = _abi.lib().goc_create(ctypes.byref(g), ctypes.byref(m), ctypes.byref(f), ctypes.byref(h),
                               ctypes.byref(e), ctypes.byref(out))
    assert st == _abi.GOC_EINVAL and b"gi_correction" in _abi.lib().goc_last_error()
