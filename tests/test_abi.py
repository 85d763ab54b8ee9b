"""C-ABI checks that need no GPU: the library builds and loads, exports every symbol the
header declares, the ctypes structs match the C layout, and hydot_setup rejects bad
arguments before touching the device."""
import ctypes as C
import os
import re
import subprocess

import numpy as np
import pytest

import paper_1410_0986_gb300._lib as L
from paper_1410_0986_gb300 import _build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "hydot.h")


@pytest.fixture(scope="module")
def lib():
    _build.build()
    return L.load()


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(hydot_[a-zA-Z0-9_]+)\s*\(", src)))


def test_header_and_exports_agree(lib):
    decl = declared_functions()
    assert decl == sorted(L.EXPORTS)
    out = subprocess.run(["nm", "-D", "--defined-only", L.LIB_PATH], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\sT\s(hydot_\w+)", out))
    assert set(decl) <= exported
    for name in decl:
        assert getattr(lib, name) is not None


def test_version(lib):
    assert lib.hydot_version() == 10000


def test_struct_layout_matches_c(tmp_path):
    prog = tmp_path / "layout.c"
    prog.write_text(r'''
#include <stdio.h>
#include <stddef.h>
#include "hydot.h"
#define O(T, f) printf(#f " %zu\n", offsetof(T, f))
int main(void) {
  printf("sizeof_problem %zu\n", sizeof(hydot_problem));
  printf("sizeof_stats %zu\n", sizeof(hydot_stats));
  O(hydot_problem, h_mm); O(hydot_problem, robin_A); O(hydot_problem, n_lambda); O(hydot_problem, eps);
  O(hydot_problem, omega); O(hydot_problem, c_medium); O(hydot_problem, n_src); O(hydot_problem, src_ijk);
  O(hydot_problem, precision); O(hydot_problem, tol); O(hydot_problem, tol_cw); O(hydot_problem, inner_tol);
  O(hydot_problem, max_iter); O(hydot_problem, deflation_k); O(hydot_problem, max_lambda_per_call);
  O(hydot_problem, cw_floor);
  return 0;
}''')
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c99", "-I", os.path.join(ROOT, "include"), str(prog), "-o", str(exe)], check=True)
    vals = dict(line.split() for line in subprocess.run([str(exe)], capture_output=True, text=True).stdout.splitlines())
    assert int(vals["sizeof_problem"]) == C.sizeof(L.Problem)
    assert int(vals["sizeof_stats"]) == C.sizeof(L.Stats)
    for name, _ in L.Problem._fields_:
        if name in vals:
            assert int(vals[name]) == getattr(L.Problem, name).offset, name


def _problem(**over):
    eps = np.full((3, 2), 0.1)
    cbg = np.array([0.05, 0.05])
    musp = np.ones(3)
    src = np.array([[1, 1, 3]], dtype=np.int32)
    det = np.array([[2, 2, 3]], dtype=np.int32)
    keep = [eps, cbg, musp, src, det]
    p = L.Problem()
    p.nx, p.ny, p.nz, p.h_mm = 4, 4, 4, 2.0
    for f in range(6):
        p.robin_A[f] = 3.0
    p.n_lambda, p.n_chrom = 3, 2
    p.eps = eps.ctypes.data_as(C.POINTER(C.c_double))
    p.c_bg = cbg.ctypes.data_as(C.POINTER(C.c_double))
    p.mus_prime = musp.ctypes.data_as(C.POINTER(C.c_double))
    p.n_src, p.n_det = 1, 1
    p.src_ijk = src.ctypes.data_as(C.POINTER(C.c_int))
    p.det_ijk = det.ctypes.data_as(C.POINTER(C.c_int))
    p.precision, p.tol, p.tol_cw = L.HYDOT_MIXED, 1e-8, 0.0
    for k, v in over.items():
        if k == "det_cell":
            det[0] = v
        else:
            setattr(p, k, v)
    return p, keep


@pytest.mark.parametrize("over,needle", [
    ({"nx": 0}, "grid extents"),
    ({"h_mm": -1.0}, "h_mm"),
    ({"n_chrom": 17}, "n_chrom"),
    ({"det_cell": (9, 0, 0)}, "outside the grid"),
    ({"det_cell": (1, 1, 3)}, "share a cell"),
    ({"tol": 0.0}, "tol must"),
    ({"tol_cw": 2.0}, "tol_cw"),
    ({"precision": 7}, "precision"),
    ({"deflation_k": 33}, "deflation_k"),
    ({"max_lambda_per_call": 4}, "max_lambda_per_call"),
    ({"cw_floor": -1.0}, "cw_floor"),
])
def test_setup_rejects_bad_arguments_without_a_device(lib, over, needle):
    p, keep = _problem(**over)
    out = C.c_void_p(123)
    rc = lib.hydot_setup(C.byref(p), None, C.byref(out))
    assert rc == L.HYDOT_ERR_ARG
    assert out.value is None
    assert needle in lib.hydot_last_error(None).decode()


def test_null_arguments(lib):
    assert lib.hydot_setup(None, None, None) == L.HYDOT_ERR_ARG
    assert lib.hydot_solve_fields(None, 0, 1, None, None, None) == L.HYDOT_ERR_ARG
    assert lib.hydot_born_apply(None, None, None, 0, 1, None, None) == L.HYDOT_ERR_ARG
    # the batch call checks its lists before it asks for a device: an empty batch is a no-op and a
    # missing list or context is an argument error
    i1, v1 = (C.c_int * 1)(0), (C.c_void_p * 1)(None)
    assert lib.hydot_solve_batch(None, 0, None, None, None, None, None, None) == L.HYDOT_OK
    assert lib.hydot_solve_batch(None, -1, None, None, None, None, None, None) == L.HYDOT_ERR_ARG
    assert lib.hydot_solve_batch(None, 1, i1, i1, v1, v1, None, None) == L.HYDOT_ERR_ARG
    st1 = (C.c_int * 1)(7)
    assert lib.hydot_solve_batch(v1, 1, i1, i1, v1, v1, None, st1) == L.HYDOT_ERR_ARG
    assert st1[0] == L.HYDOT_ERR_ARG and "NULL" in lib.hydot_last_error(None).decode()
    lib.hydot_destroy(None)


def test_solve_batch_binding_checks_its_lists_without_a_device(lib):
    """The Python batch call checks the per-context wavelength lists before it touches a context."""
    import paper_1410_0986_gb300 as hd

    assert hd.solve_batch([], 0, 1) == []
    dummies = [object(), object()]
    with pytest.raises(ValueError):
        hd.solve_batch(dummies, [0], 1)
    with pytest.raises(ValueError):
        hd.solve_batch(dummies, 0, [1, 1, 1])


def test_status_codes_match_the_header():
    """The binding's status table is the header's enum, value by value."""
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    body = re.search(r"typedef enum \{(.*?)\} hydot_status;", src, re.S).group(1)
    codes = {name: int(val) for name, val in re.findall(r"(HYDOT_\w+)\s*=\s*(-?\d+)", body)}
    assert codes == {v: k for k, v in L.STATUS_NAMES.items()}


def test_every_status_returning_entry_point_is_exception_guarded():
    """No C++ exception may cross the ABI: every extern "C" function that returns a status runs
    its body inside abi_guard (std::bad_alloc -> HYDOT_ERR_OOM, anything else -> HYDOT_ERR_HOST)."""
    csrc = os.path.join(ROOT, "paper_1410_0986_gb300", "csrc")
    found = 0
    for fn in os.listdir(csrc):
        if not fn.endswith(".cu"):
            continue
        text = open(os.path.join(csrc, fn)).read()
        for m in re.finditer(r"^(?:extern \"C\" )?int (hydot_\w+)\([^)]*\) \{\n(.*?)\n\}", text, re.M | re.S):
            if m.group(1) not in L.EXPORTS:
                continue
            found += 1
            first = m.group(2).lstrip().splitlines()[0]
            if "using namespace" in first:
                first = m.group(2).lstrip().splitlines()[1]
            assert "abi_guard(" in first, (fn, m.group(1))
    assert found == len([n for n in L.EXPORTS if n not in ("hydot_version", "hydot_kernel_launches",
                                                            "hydot_last_error", "hydot_destroy")])
