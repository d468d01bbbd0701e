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


def test_in_place_streaming_is_refused_outside_its_scope_without_a_gpu():
    """goc_exec.streaming = 1 takes scheme 0 and a straight grid (any
    storage, with or without the MIE); anything else is GOC_EUNSUPPORTED
    before the device is touched, and an unknown value GOC_EINVAL."""
    import goc_inputs as gi
    from paper_2607_15362_b300.lattice import structs_from_spec, _exec

    prob = gi.Problem("cavity", 16, 16, {"kind": "tanh2", "beta": 1.5}, {"kind": "uniform"}, {"Re": 10.0, "u_lid": 0.05})
    spec = prob.lattice_spec(0.01)
    tc = gi.taylor_couette(n1=16, n2=5, r_in=6.0, sectors=9.0, Re=20.0, u_in=1.0, u_out=1.5)
    cases = [(spec, dict(scheme="goc_srt")), (spec, dict(scheme="goc_raw")),
             (tc.lattice_spec(0.01), {}), (tc.lattice_spec(0.01), dict(storage="fp16"))]
    for sp, kw in cases:
        g, m, f, h = structs_from_spec(sp)
        e = _exec(kw.get("storage", "fp32"), None, 100, "stochastic", kw.get("scheme", "goc"), streaming="in_place")
        out = ctypes.c_void_p()
        st = _abi.lib().goc_create(ctypes.byref(g), ctypes.byref(m), ctypes.byref(f), ctypes.byref(h),
                                   ctypes.byref(e), ctypes.byref(out))
        assert st == _abi.GOC_EUNSUPPORTED and not out.value, (kw, st)
        assert b"in-place streaming" in _abi.lib().goc_last_error()
    g, m, f, h = structs_from_spec(spec)
    e = _exec("fp32", None, 100, streaming="in_place")   # slabs and batches keep two buffers
    out = ctypes.c_void_p()
    st = _abi.lib().goc_create_slab(ctypes.byref(g), ctypes.byref(m), ctypes.byref(f), ctypes.byref(h),
                                    ctypes.byref(e), 0, 8, ctypes.byref(out))
    assert st == _abi.GOC_EUNSUPPORTED and not out.value
    st = _abi.lib().goc_batch_create(1 << 30, 4, ctypes.byref(e), ctypes.byref(out))
    assert st == _abi.GOC_EUNSUPPORTED and not out.value
    assert b"two population buffers" in _abi.lib().goc_last_error()
    e = _exec("fp32", None, 100)
    e.streaming = 2
    out = ctypes.c_void_p()
    st = _abi.lib().goc_create(ctypes.byref(g), ctypes.byref(m), ctypes.byref(f), ctypes.byref(h),
                               ctypes.byref(e), ctypes.byref(out))
    assert st == _abi.GOC_EINVAL and b"streaming" in _abi.lib().goc_last_error()


@pytest.mark.parametrize("map1,map2,walls,needle", [
    ({"kind": "tanh1", "beta": 0.0}, {"kind": "uniform"}, "WE", b"one-wall tanh beta"),
    ({"kind": "sinh", "mu": 3.0, "yc": 1.2}, {"kind": "uniform"}, "WE", b"yc"),
    ({"kind": "sinh", "mu": 0.0, "yc": 0.5}, {"kind": "uniform"}, "WE", b"mu"),
    ({"kind": "tanh1", "beta": 2.0}, {"kind": "uniform"}, "", b"periodic axis"),
    ({"kind": "uniform"}, {"kind": "annulus", "r_in": 2.0, "r_out": 10.0, "sectors": 6.0}, "WE", b"xi1 (radial)"),
    ({"kind": "annulus", "r_in": 2.0, "r_out": 10.0, "sectors": 6.0}, {"kind": "uniform"}, "WESN", b"periodic S/N"),
    ({"kind": "annulus", "r_in": 10.0, "r_out": 2.0, "sectors": 6.0}, {"kind": "uniform"}, "WE", b"r_inner < r_outer"),
])
def test_map_parameters_are_validated_without_a_gpu(map1, map2, walls, needle):
    """goc_metric_info rejects bad map parameters (one-wall tanh, interior
    point, annulus) on the host, before any device call."""
    w = {s: ({"u": 0.0} if s in walls else None) for s in "WESN"}
    spec = {"nx": 12, "ny": 10, "map1": map1, "map2": map2, "walls": w}
    g, m, f, h = goc.structs_from_spec(spec)
    q, cs2 = ctypes.c_double(), ctypes.c_double()
    st = _abi.lib().goc_metric_info(ctypes.byref(g), ctypes.byref(m), ctypes.byref(q), ctypes.byref(cs2))
    assert st == _abi.GOC_EINVAL
    assert needle in _abi.lib().goc_last_error()


def test_oversized_lattices_are_rejected_without_a_gpu():
    """nx * ny above 2^31 or ny above 65535 (the launch grid limit of the
    one-off kernels) is refused with a message, before any allocation."""
    for nx, ny in ((70000, 70000), (8, 70000)):
        spec = {"nx": nx, "ny": ny, "walls": {"W": None, "E": None, "S": None, "N": None}}
        g, m, f, h = goc.structs_from_spec(spec)
        q, cs2 = ctypes.c_double(), ctypes.c_double()
        st = _abi.lib().goc_metric_info(ctypes.byref(g), ctypes.byref(m), ctypes.byref(q), ctypes.byref(cs2))
        assert st == _abi.GOC_EINVAL
        assert b"too large" in _abi.lib().goc_last_error()


def test_node_table_map_is_validated_and_sized_on_the_host():
    """A TABLE map needs both host arrays, h1, h2 > 0 at every node and along
    the wall sides; goc_metric_info then returns q = the smallest h without a
    device call."""
    import numpy as np
    import goc_inputs as gi
    p = gi.spiral_cavity(12, 10)
    spec = p.lattice_spec(0.1)
    g, m, f, h = goc.structs_from_spec(spec)
    q, cs2 = ctypes.c_double(), ctypes.c_double()
    assert _abi.lib().goc_metric_info(ctypes.byref(g), ctypes.byref(m), ctypes.byref(q), ctypes.byref(cs2)) == 0
    assert q.value == pytest.approx(float(np.min(p.metric["h1"])), rel=1e-15)
    assert cs2.value == pytest.approx(q.value ** 2 / 3, rel=1e-15)
    bad = dict(p.metric, h2=p.metric["h2"].copy())
    bad["h2"][3, 4] = 0.0
    spec["metric"] = bad
    g, m, f, h = goc.structs_from_spec(spec)
    assert _abi.lib().goc_metric_info(ctypes.byref(g), ctypes.byref(m), ctypes.byref(q), ctypes.byref(cs2)) == _abi.GOC_EINVAL
    assert b"h1, h2" in _abi.lib().goc_last_error()
    m.table = None
    assert _abi.lib().goc_metric_info(ctypes.byref(g), ctypes.byref(m), ctypes.byref(q), ctypes.byref(cs2)) == _abi.GOC_EINVAL
    assert b"needs table" in _abi.lib().goc_last_error()
    g, m, f, h = goc.structs_from_spec({"nx": 12, "ny": 10, "map2": {"kind": "table"},
                                        "walls": {"W": None, "E": None, "S": None, "N": None}})
    assert _abi.lib().goc_metric_info(ctypes.byref(g), ctypes.byref(m), ctypes.byref(q), ctypes.byref(cs2)) == _abi.GOC_EINVAL
    assert b"kind[0]" in _abi.lib().goc_last_error()


def _build_c_example(tmp_path):
    pkg = os.path.dirname(goc.build())
    exe = tmp_path / "cavity"
    subprocess.run(["gcc", "-O2", "-std=c11", "-I", os.path.join(ROOT, "include"), "-o", str(exe),
                    os.path.join(ROOT, "tests", "c_abi", "cavity.c"), "-L", pkg, "-lgoc", f"-Wl,-rpath,{pkg}"],
                   check=True)
    return exe


def test_a_c_program_builds_against_the_library(tmp_path):
    """tests/c_abi/cavity.c uses only include/goc.h and links against
    libgoc.so with a plain C compiler (no C++ or CUDA toolchain)."""
    assert _build_c_example(tmp_path).exists()


@pytest.mark.gpu
def test_a_c_program_drives_the_library_like_the_binding(tmp_path):
    """The same 64 x 48 cavity run from C and from the Python binding gives
    the same fields (the binding only marshals arguments)."""
    import numpy as np
    exe = _build_c_example(tmp_path)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split()
    su, sv, mass, rmax = (float(x) for x in out)
    spec = {"nx": 64, "ny": 48, "map1": {"kind": "tanh2", "beta": 1.2}, "map2": {"kind": "tanh2", "beta": 1.4},
            "walls": {"W": {"u": 0.0}, "E": {"u": 0.0}, "S": {"u": 0.0}, "N": {"u": 0.01}},
            "rho0": 1.0, "nu": 0.02, "gi": 1}
    L = goc.Lattice(spec)
    L.step(500)
    rho, u1, u2, _, _ = L.moments()
    assert float(u1.sum()) == pytest.approx(su, rel=1e-12, abs=1e-15)
    assert float(u2.sum()) == pytest.approx(sv, rel=1e-12, abs=1e-15)
    assert float(rho.max()) == pytest.approx(rmax, rel=1e-14)
    assert L.mass() == pytest.approx(mass, rel=1e-14)
    L.close()


@pytest.mark.parametrize("where", ["nu", "fext", "wall_u", "beta", "b_init"])
def test_non_finite_parameters_are_refused_on_the_host(where):
    """A NaN or infinite parameter (a corrupted request) is refused with
    GOC_EINVAL before any device call, wherever it sits."""
    spec = {"nx": 16, "ny": 12, "map2": {"kind": "tanh2", "beta": 1.0},
            "walls": {"W": None, "E": None, "S": {"u": 0.0}, "N": {"u": 0.01}}, "nu": 0.1,
            "mhd": {"tau_m": 1.0, "B_init": (0.0, 0.01)}}
    g, m, f, h = goc.structs_from_spec(spec)
    bad = float("nan")
    if where == "nu":
        f.nu = bad
    elif where == "fext":
        f.fext[1] = float("inf")
    elif where == "wall_u":
        g.wall_u[3] = bad
    elif where == "beta":
        m.beta[1] = bad
    else:
        h.b_init[0] = bad
    out = ctypes.c_void_p()
    st = _abi.lib().goc_create(ctypes.byref(g), ctypes.byref(m), ctypes.byref(f), ctypes.byref(h), None,
                               ctypes.byref(out))
    assert st == _abi.GOC_EINVAL and not out.value
    assert b"finite" in _abi.lib().goc_last_error()


def test_bench_reference_arm_prints_one_contract_line():
    """bench.py --impl reference (the FP64 oracle on the host cores) prints one
    JSON line with the contract's keys, on the same workload options as the
    main line."""
    import json
    import sys
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                          "--warmup", "3", "--cavity-n", "32", "--ref-steps-per-step", "1", "--grid", "annulus"],
                         capture_output=True, text=True, check=True, cwd=ROOT).stdout.strip().splitlines()
    line = json.loads(out[-1])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
              "vs_baseline", "dtype", "data", "config", "impl", "cpu_baseline", "e2e"):
        assert k in line, k
    assert line["impl"] == "reference" and line["value"] > 0 and line["config"]["workload"].startswith("taylor_couette")
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["cpu_baseline"]["kind"] == "oracle"
