"""The allocation-free residual entry point (rav_residual_norm_noalloc).

It serves callers that cannot call cudaMalloc where they need a residual
norm, e.g. while their stream is captured into a CUDA graph or in a loop that
may only use memory reserved beforehand; its scratch (the norm's partial sums)
lives in a fixed device array of the library.  Checked against the ordinary
entry point (rav_residual), on two calls in a row, through the C ABI.  This
file is collected last on purpose.
"""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

import paper_2103_10127_gb300 as R  # noqa: E402
from paper_2103_10127_gb300 import _capi, inputs  # noqa: E402


def _p(t):
    return ctypes.c_void_p(t.data_ptr())


def test_noalloc_residual_matches_the_allocating_entry_point_twice():
    lib = _capi.load()
    mg = R.Multigrid(2, 96, 3, blobs=inputs.viscosity_blobs(5, k=4), bc=R.BC_CAVITY)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    for call, lev in enumerate((2, 2, 1)):
        n = mg.n(lev)
        x = torch.from_numpy(inputs.normal(100 + call, n)).cuda()
        b = torch.from_numpy(inputs.normal(200 + call, n)).cuda()
        r_ref, nrm_ref = mg.residual(lev, x, b, norm=True)
        r = torch.full_like(x, np.nan)
        nrm = torch.full((1,), np.nan, dtype=torch.float64, device="cuda")
        rc = lib.rav_residual_norm_noalloc(mg.h, lev, _p(x), _p(b), _p(r), _p(nrm), stream)
        assert rc == 0
        torch.cuda.synchronize()
        r_ref, r = r_ref.cpu().numpy(), r.cpu().numpy()
        assert np.abs(r - r_ref).max() <= 1e-13 * np.abs(r_ref).max()
        assert abs(nrm.item() - nrm_ref) <= 1e-13 * nrm_ref


def test_noalloc_residual_rejects_levels_beyond_its_scratch():
    lib = _capi.load()
    mg = R.Multigrid(2, 1024, 7, bc=R.BC_NOSLIP)  # 9.45 M rows > 4,194,304 slots
    n = mg.n()
    x = torch.zeros(n, dtype=torch.float64, device="cuda")
    nrm = torch.zeros(1, dtype=torch.float64, device="cuda")
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    assert lib.rav_residual_norm_noalloc(mg.h, 6, _p(x), _p(x), _p(x), _p(nrm), stream) == -1
    # a smaller level of the same hierarchy still works
    m = mg.n(4)
    y = torch.ones(m, dtype=torch.float64, device="cuda")
    r = torch.empty_like(y)
    assert lib.rav_residual_norm_noalloc(mg.h, 4, _p(y), _p(y), _p(r), _p(nrm), stream) == 0
    torch.cuda.synchronize()
    _, ref = mg.residual(4, y, y, norm=True)
    assert abs(nrm.item() - ref) <= 1e-13 * ref
