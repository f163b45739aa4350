"""The C ABI called from C: tests/c/solve_cavity.c is compiled with gcc against
include/ravanka.h, linked to the in-tree libravanka.so and the CUDA runtime,
and run; its iteration counts equal the oracle's (stationary) and its final
ratios meet the tolerance (both solvers), on both elements."""
import os
import subprocess

import pytest

import oracle as O

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_2103_10127_gb300 import _capi  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CUDA = os.environ.get("CUDA_HOME", "/usr/local/cuda")


@pytest.fixture(scope="module")
def exe(tmp_path_factory):
    _capi.load()  # builds the library when stale
    libdir = os.path.join(ROOT, "paper_2103_10127_gb300")
    out = str(tmp_path_factory.mktemp("c_abi") / "solve_cavity")
    subprocess.check_call(["gcc", "-std=c99", "-O1", "-I", os.path.join(ROOT, "include"), "-I",
                           os.path.join(CUDA, "include"), os.path.join(ROOT, "tests", "c", "solve_cavity.c"),
                           "-o", out, "-L", libdir, "-lravanka", "-L", os.path.join(CUDA, "lib64"), "-lcudart",
                           f"-Wl,-rpath,{libdir}", f"-Wl,-rpath,{os.path.join(CUDA, 'lib64')}"])
    return out


@pytest.mark.parametrize("element,omega", [(0, 0.5), (1, 0.66)], ids=["q2q1", "q1q1"])
def test_c_caller_solves_the_cavity(exe, element, omega):
    res = subprocess.run([exe, str(element)], capture_output=True, text=True, timeout=120)
    assert res.returncode == 0, res.stderr
    f = res.stdout.split()
    it_s, ratio_s, it_f, ratio_f = int(f[1]), float(f[2]), int(f[4]), float(f[5])
    assert ratio_s <= 1e-8 and ratio_f <= 1e-8
    orc = O.Oracle(2, 16, 3, bc=O.BC_CAVITY, element=element, beta=0.02)
    orc.setup_smoother(O.RAV, omega)
    _, oit, _ = orc.solve(orc.initial_guess(), orc.rhs(O.F_NONE), tol=1e-8, maxit=100)
    assert it_s == oit
    assert 0 < it_f <= it_s
