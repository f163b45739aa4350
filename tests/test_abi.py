"""C-ABI checks that need no GPU: the library builds, loads, exports every
function include/ravanka.h declares, and rejects invalid arguments before any
CUDA call."""
import ctypes
import os
import re

import pytest

from paper_2103_10127_gb300 import _capi

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "ravanka.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?(?:int64_t|int|void|char)\s*\*?\s*([A-Za-z_]\w*)\s*\(", src, flags=re.M)
    return sorted(set(names))


def test_library_exports_every_declared_symbol():
    lib = _capi.load()
    names = declared_functions()
    assert len(names) >= 20
    for n in names:
        assert hasattr(lib, n), n
    assert set(names) <= set(_capi.exported_symbols()) | set()


def test_invalid_arguments_are_rejected_without_a_gpu():
    lib = _capi.load()
    h = ctypes.c_void_p()
    bad = [
        _capi.RavProblem(4, 16, None, 1.0, 0, None, 0),   # dim
        _capi.RavProblem(2, 1, None, 1.0, 0, None, 0),    # N < 2
        _capi.RavProblem(2, 12, None, 1.0, 0, None, 0),   # 12 not divisible by 2^3
        _capi.RavProblem(2, 16, None, 1.0, -1, None, 0),  # negative blob count
        _capi.RavProblem(2, 16, None, 1.0, 0, None, 0, 2, 0.0),  # unknown element
        _capi.RavProblem(2, 16, None, 1.0, 0, None, 0, 1, -0.1),  # negative beta (Q1-Q1)
        _capi.RavProblem(2, 16, None, 1.0, 0, None, 0, 1, float("nan")),  # beta not finite
        _capi.RavProblem(2, 16, None, 1.0, 0, None, 0, 1, float("inf")),
    ]
    for p in bad:
        assert lib.mg_setup(ctypes.byref(p), 4, None, ctypes.byref(h)) == -1
    p = _capi.RavProblem(2, 16, None, 1.0, 0, None, 0)
    assert lib.mg_setup(ctypes.byref(p), 5, None, ctypes.byref(h)) == -1  # coarsest grid 1 cell
    assert lib.mg_setup(ctypes.byref(p), 17, None, ctypes.byref(h)) == -1  # too many levels
    big = _capi.RavProblem(3, 24, None, 1.0, 0, None, 0)  # one 24^3 level: explicit coarse inverse too large
    assert lib.mg_setup(ctypes.byref(big), 1, None, ctypes.byref(h)) == -1
    c = (ctypes.c_double * 34)(*([0.0] * 34))  # non-increasing coordinates
    p = _capi.RavProblem(2, 16, ctypes.cast(c, ctypes.c_void_p), 1.0, 0, None, 0)
    assert lib.mg_setup(ctypes.byref(p), 2, None, ctypes.byref(h)) == -1
    assert lib.mg_setup(None, 2, None, ctypes.byref(h)) == -1
    assert lib.vanka_setup(None, 0, 0, 0.5, None, ctypes.byref(h)) == -1
    assert lib.vcycle(None, None, None, None, 2, 2, None) == -1
    assert lib.solve(None, None, None, None, None, None, None) == -1
    assert lib.rav_set_residual_split(None, 0, 4) == -1
    assert lib.rav_get_residual_split(None, 0) == -1
    rate = ctypes.c_double()
    assert lib.rav_hbm_read_rate(8, ctypes.byref(rate), None) == -1  # fewer than 16 bytes
    assert lib.rav_hbm_read_rate(1 << 20, None, None) == -1
    # the reduced-precision coarse-grid forms and the batched tile choice
    assert lib.rav_set_coarse_residual_f32(None, 1, 0, None) == -1
    assert lib.rav_get_coarse_residual_f32(None) == -1
    assert lib.rav_set_transfers_f32(None, 1, None) == -1
    assert lib.rav_get_transfers_f32(None) == -1
    assert lib.batch_set_coarse_residual_f32(None, 1, None) == -1
    assert lib.batch_coarse_residual_f32(None) == -1
    assert lib.batch_set_transfers_f32(None, 1, None) == -1
    assert lib.batch_transfers_f32(None) == -1
    assert lib.batch_set_apply_tile(None, 2, 2, None) == -1
    tile = (ctypes.c_int * 2)()
    assert lib.batch_get_apply_tile(None, 0, tile) == -1
    assert lib.rav_strerror(-3) == b"singular subdomain system"


def test_struct_layouts_match_the_header(tmp_path):
    """sizeof/offsetof of the ctypes mirrors equal those a C compiler gives the header."""
    import subprocess
    prog = tmp_path / "layout.c"
    prog.write_text(
        '#include <stddef.h>\n#include <stdio.h>\n#include "ravanka.h"\n'
        'int main(void){printf("%zu %zu %zu %zu %zu %zu %zu %zu\\n", sizeof(rav_problem), offsetof(rav_problem, bc),'
        ' offsetof(rav_problem, element), offsetof(rav_problem, beta),'
        ' sizeof(rav_solve_opts), offsetof(rav_solve_opts, fallback_rho), sizeof(rav_solve_info),'
        ' offsetof(rav_solve_info, fell_back)); return 0;}\n')
    exe = tmp_path / "layout"
    subprocess.check_call(["gcc", "-std=c99", "-I", os.path.join(ROOT, "include"), str(prog), "-o", str(exe)])
    got = [int(v) for v in subprocess.check_output([str(exe)]).split()]
    want = [ctypes.sizeof(_capi.RavProblem), _capi.RavProblem.bc.offset, _capi.RavProblem.element.offset,
            _capi.RavProblem.beta.offset, ctypes.sizeof(_capi.RavSolveOpts),
            _capi.RavSolveOpts.fallback_rho.offset, ctypes.sizeof(_capi.RavSolveInfo),
            _capi.RavSolveInfo.fell_back.offset]
    assert got == want
