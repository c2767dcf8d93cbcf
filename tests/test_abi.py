"""The C ABI library loads, exports every entry point include/lamp.h declares, and
rejects invalid arguments on the host before touching a GPU (CPU-only tests)."""
import ctypes
import re
from pathlib import Path

import pytest

ROOT = Path(__file__).resolve().parents[1]


@pytest.fixture(scope="module")
def L():
    from paper_2511_11359_gb300 import build as b

    b.build()
    import paper_2511_11359_gb300 as L

    return L


def header_functions():
    src = (ROOT / "include" / "lamp.h").read_text()
    return re.findall(r"LAMP_API\s+[\w\s\*]+?\b(lamp_\w+)\s*\(", src)


def test_header_lists_expected_functions(L):
    names = header_functions()
    assert len(names) == len(set(names)) >= 13
    assert set(names) == set(L.EXPORTED_SYMBOLS)


def test_every_declared_symbol_is_exported(L):
    lib = ctypes.CDLL(str(L.library_path))
    for name in header_functions():
        assert hasattr(lib, name), name


def test_params_default(L):
    p = L.default_params()
    assert (p.eta, p.tau1, p.tau2, p.alpha, p.beta, p.tol) == (0.0, 0.0, 0.0, 0.01, 1.1, 1e-6)
    assert p.max_iter == 100000 and p.check_every == 50 and p.prec == L.PREC_FP32 and p.K == 0.0
    assert p.gap_tol == 0.0 and p.gap_every == 0 and p.infeas_only == 0


def _prob(L, **kw):
    pr = L._Problem()
    pr.n, pr.m, pr.d, pr.kind = 8, 9, 2, L.COST_SQEUCLID
    pr.x, pr.y, pr.r, pr.c = 0x1000, 0x2000, 0x3000, 0x4000  # never dereferenced: validation fails first
    pr.cost_scale = 1.0
    for k, v in kw.items():
        setattr(pr, k, v)
    return pr


BAD = [
    ({"n": 0}, {}), ({"m": -1}, {}), ({"d": 0}, {}), ({"d": 65}, {}), ({"kind": 7}, {}), ({"x": 0}, {}),
    ({"r": 0}, {}), ({"kind": 0, "C": 0, "ldc": 9}, {}), ({"kind": 0, "C": 0x10, "ldc": 3}, {}),
    ({"cost_scale": float("nan")}, {}),
    ({}, {"eta": -1.0}), ({}, {"alpha": 0.0}), ({}, {"beta": -0.1}), ({}, {"tau1": -1.0}),
    ({}, {"tau1": 2.0, "eta": 1.0}), ({}, {"check_every": 0}), ({}, {"max_iter": -5}), ({}, {"prec": 9}),
    ({}, {"K": -1.0}), ({}, {"tol": float("nan")}), ({}, {"eta": float("inf")}),
    # tensor cores only for the dot-form costs (LAMP_COST_L1 = 2, LAMP_COST_LINF = 3, DENSE = 0)
    ({"kind": 2}, {"prec": 1}), ({"kind": 3}, {"prec": 1}), ({"kind": 0, "C": 0x10, "ldc": 9}, {"prec": 1}),
    ({"n": 1 << 32}, {}), ({"m": (1 << 31) + 1}, {}), ({}, {"check_every": 100001}),
    ({"cost_scale": float("inf")}, {}), ({}, {"alpha": float("nan")}), ({}, {"K": float("inf")}),
    # primal-dual gap termination and the eta > 0 rule switch
    ({}, {"gap_tol": -1e-9}), ({}, {"gap_tol": float("nan")}), ({}, {"gap_tol": float("inf")}),
    ({}, {"gap_every": -1}), ({}, {"infeas_only": 2}),
]


@pytest.mark.parametrize("pkw,akw", BAD)
def test_invalid_arguments_rejected_on_host(L, pkw, akw):
    pr = _prob(L, **pkw)
    pa = L.default_params(**akw)
    h = ctypes.c_void_p()
    code = L.lib.lamp_create(ctypes.byref(h), ctypes.byref(pr), ctypes.byref(pa), None)
    assert code == L.LAMP_E_INVALID
    assert h.value is None
    assert L.lib.lamp_last_error(None)


def test_null_context_calls(L):
    assert L.lib.lamp_solve(None, None) == L.LAMP_E_INVALID
    assert L.lib.lamp_iterate(None, 1) == L.LAMP_E_INVALID
    assert L.lib.lamp_grad(None, None, None) == L.LAMP_E_INVALID
    assert L.lib.lamp_launches_per_iteration(None) == 0
    L.lib.lamp_destroy(None)
    out = ctypes.c_void_p()
    assert L.lib.lamp_create(ctypes.byref(out), None, None, None) == L.LAMP_E_INVALID
    assert L.lib.lamp_create(None, None, None, None) == L.LAMP_E_INVALID


def test_objective_slots_match_header(L):
    src = (ROOT / "include" / "lamp.h").read_text()
    assert int(re.search(r"#define LAMP_OBJECTIVE_SLOTS (\d+)", src).group(1)) == L.OBJECTIVE_SLOTS
    out = (ctypes.c_double * L.OBJECTIVE_SLOTS)()
    assert L.lib.lamp_objective(None, out) == L.LAMP_E_INVALID


def test_evaluation_entry_points_validate_on_host(L):
    out = (ctypes.c_double * 4)()
    assert L.lib.lamp_round(None, out, None, None, None) == L.LAMP_E_INVALID
    assert L.lib.lamp_dual(None, out) == L.LAMP_E_INVALID
    st = ctypes.c_int(0)
    assert L.lib.lamp_selftest_wait_timeout(0, ctypes.byref(st)) == L.LAMP_E_INVALID
    assert L.lib.lamp_selftest_wait_timeout(1 << 31, ctypes.byref(st)) == L.LAMP_E_INVALID
    assert L.lib.lamp_selftest_wait_timeout(10, None) == L.LAMP_E_INVALID
    assert b"polls" in L.lib.lamp_last_error(None)


def test_struct_layouts_match_header(L, tmp_path):
    """The binding's ctypes structures mirror include/lamp.h: compare every field
    offset and the struct sizes with a C program compiled against the header."""
    import shutil
    import subprocess

    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    structs = {"lamp_problem": L._Problem, "lamp_params": L._Params, "lamp_result": L._Result}
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "lamp.h"', "int main(void){"]
    for cname, cls in structs.items():
        lines.append(f'printf("{cname} size %zu\\n", sizeof({cname}));')
        for f, _ in cls._fields_:
            lines.append(f'printf("{cname} {f} %zu\\n", offsetof({cname}, {f}));')
    lines.append("return 0;}")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run([cc, "-I", str(ROOT / "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    seen = 0
    for line in out:
        if not line.strip():
            continue
        cname, field, val = line.split()
        cls = structs[cname]
        if field == "size":
            assert ctypes.sizeof(cls) == int(val), line
        else:
            assert getattr(cls, field).offset == int(val), line
        seen += 1
    assert seen == sum(len(c._fields_) + 1 for c in structs.values())
