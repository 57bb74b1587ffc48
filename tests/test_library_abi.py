"""The C ABI library builds, loads without a GPU and exports every symbol the
public header declares; the Python binding mirrors the header's structs."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = []
    for fn in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if fn.endswith(".h"):
            text = open(os.path.join(ROOT, "include", fn)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names += re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\*?\s*(hif_[a-z_0-9]+)\s*\(", text, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    from paper_1307_2666_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    names = _declared()
    for required in ["hif_factor", "hif_apply", "hif_solve", "hif_solve_transpose", "hif_destroy",
                     "hif_apply_transpose", "hif_matvec", "hif_solve_refined", "hif_stats"]:
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    for name in _declared():
        assert hasattr(lib, name), name


def _declared_signatures():
    """name -> list of parameter type strings, from the header's prototypes."""
    text = ""
    for fn in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if fn.endswith(".h"):
            text += re.sub(r"/\*.*?\*/", "", open(os.path.join(ROOT, "include", fn)).read(), flags=re.S)
    out = {}
    for m in re.finditer(r"^\s*((?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\*?)\s*(hif_[a-z_0-9]+)\s*\(([^)]*)\)\s*;",
                         text, flags=re.M):
        params = [p.strip() for p in " ".join(m.group(3).split()).split(",") if p.strip()]
        out[m.group(2)] = (" ".join(m.group(1).split()), [] if params == ["void"] else params)
    return out


def _ctypes_kind(t):
    # the C type a ctypes argtype stands for, coarsely: pointer, 8-byte integer,
    # 4-byte integer, double, float
    import ctypes as C
    if t in (C.c_void_p, C.c_char_p) or (isinstance(t, type) and issubclass(t, C._Pointer)):
        return "ptr"
    return {C.c_int64: "i64", C.c_uint64: "i64", C.c_int: "i32", C.c_int32: "i32", C.c_double: "f64",
            C.c_float: "f32"}[t]


def _c_kind(p):
    if "*" in p:
        return "ptr"
    base = p.split()[0] if p.split()[0] != "const" else p.split()[1]
    return {"int64_t": "i64", "uint64_t": "i64", "int": "i32", "int32_t": "i32", "double": "f64", "float": "f32",
            "hif_handle": "ptr", "hif_status": "i32"}[base]


def test_binding_signatures_match_header():
    # every exported call takes, in the binding, as many arguments of the same
    # kinds (pointer, 64-bit or 32-bit integer, double, float) as the header declares
    from paper_1307_2666_gb300 import hif
    import ctypes as C
    sigs = _declared_signatures()
    assert set(sigs) == set(_declared())
    ret = {"hif_status": C.c_int, "const char*": C.c_char_p, "const char *": C.c_char_p, "uint64_t": C.c_uint64}
    for name, (rtype, params) in sigs.items():
        restype, argtypes = hif.EXPORTS[name]
        assert restype is ret[rtype], (name, rtype)
        assert len(argtypes) == len(params), (name, params)
        assert [_ctypes_kind(t) for t in argtypes] == [_c_kind(p) for p in params], (name, params)


def test_binding_covers_header(lib):
    from paper_1307_2666_gb300 import hif
    for name in _declared():
        assert name in hif.EXPORTS, name


def test_struct_layouts_match_header(lib):
    from paper_1307_2666_gb300 import hif
    # hif_options_default fills every field; defaults from the header comment
    o = hif.hif_options_default(2)
    assert (o.dim, o.leaf_occupancy, o.second_kind, o.precision, o.fractional_levels) == (2, 64, 1, 0, 1)
    assert o.proxy_points == 64 and o.proxy_radius == 1.5 and o.fp32_tol_floor == 2.0 ** -17
    assert o.direct_precision == 2 and o.use_graphs == 1 and o.autotune == 1 and o.symmetric == 1 and o.ldl == 1
    o3 = hif.hif_options_default(3)
    assert o3.proxy_points == 512


def test_ctypes_layouts_match_c_compiler(tmp_path):
    # compile a probe against the header and compare sizes / offsets
    import subprocess
    from paper_1307_2666_gb300 import hif
    src = tmp_path / "probe.c"
    src.write_text('''#include <stdio.h>
#include <stddef.h>
#include "hif.h"
int main(void){printf("%zu %zu %zu %zu %zu %zu %zu %zu %zu %zu %zu %zu %zu %zu %zu %zu %zu %zu %zu\\n", sizeof(hif_options),
 offsetof(hif_options, proxy_radius),
 offsetof(hif_options, stream), offsetof(hif_options, direct_precision), offsetof(hif_options, autotune),
 offsetof(hif_options, symmetric), offsetof(hif_options, ldl), offsetof(hif_options, wavenumber),
 sizeof(hif_stats_t), offsetof(hif_stats_t, kinds), offsetof(hif_stats_t, flops),
 offsetof(hif_stats_t, top_size), offsetof(hif_stats_t, ldl_fallbacks),
 sizeof(hif_profile_entry), offsetof(hif_profile_entry, bytes),
 sizeof(hif_gemm_problem), offsetof(hif_gemm_problem, m), offsetof(hif_gemm_problem, alpha),
 offsetof(hif_gemm_problem, beta)); return 0;}''')
    exe = tmp_path / "probe"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = [int(v) for v in subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split()]
    O, S, E, G = hif.hif_options, hif.hif_stats_t, hif.hif_profile_entry, hif.hif_gemm_problem
    want = [ctypes.sizeof(O), O.proxy_radius.offset, O.stream.offset, O.direct_precision.offset, O.autotune.offset,
            O.symmetric.offset, O.ldl.offset, O.wavenumber.offset, ctypes.sizeof(S), S.kinds.offset, S.flops.offset, S.top_size.offset,
            S.ldl_fallbacks.offset, ctypes.sizeof(E), E.bytes.offset, ctypes.sizeof(G), G.m.offset, G.alpha.offset,
            G.beta.offset]
    assert got == want


def test_status_strings_and_argument_errors(lib):
    from paper_1307_2666_gb300 import hif
    L = hif.load()
    assert L.hif_status_string(0) == b"HIF_OK"
    assert b"EINVAL" in L.hif_status_string(1)
    # invalid arguments are rejected before any device work (no GPU needed)
    h = ctypes.c_void_p()
    assert L.hif_factor(None, 10, None, None, None, None, 0, 1e-6, None, ctypes.byref(h)) == hif.HIF_EINVAL
    assert h.value is None
    assert L.hif_options_default(4, None) == hif.HIF_EINVAL
    assert L.hif_destroy(None) == hif.HIF_OK
    assert L.hif_apply(None, None, None, 1, 1) == hif.HIF_EINVAL
    norms = (ctypes.c_double * 3)()
    its = (ctypes.c_int * 3)()
    assert L.hif_error_estimates(None, None, 1e-2, 10, norms, its) == hif.HIF_EINVAL
    cnt = ctypes.c_int64(-1)
    assert L.hif_eliminated_dofs(None, 0, None, 0, ctypes.byref(cnt)) == hif.HIF_EINVAL
    assert L.hif_adjoint_gradients(None, None, None, 1, 1, None, None, None) == hif.HIF_EINVAL
    assert L.hif_matvec_digits(None, 0, 6, None, None, 1, 1) == hif.HIF_EINVAL
    assert b"classes must be 4, 5, 6 or 8" in L.hif_last_error()
    # a symmetric option outside {0, 1} is rejected before any device work
    o = hif.hif_options_default(2)
    o.symmetric = 2
    pts = np.zeros((4, 2))
    one = np.ones(4)
    assert L.hif_factor(pts.ctypes.data, 4, one.ctypes.data, one.ctypes.data, one.ctypes.data, one.ctypes.data,
                        0, 1e-6, ctypes.byref(o), ctypes.byref(h)) == hif.HIF_EINVAL
    assert h.value is None
