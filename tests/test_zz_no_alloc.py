"""polyeval_eval_noalloc, the entry point for callers that cannot let the
library allocate device memory (their memory belongs to another allocator or
to a fixed arena): the system, points and outputs live in the caller's own
device buffers, and the only scratch is the library's static device array.

Checked through the C ABI against polyeval_eval (which allocates at create
time) on two calls in a row, within the double-double tolerance the other
tests use.  Kept in a file of its own that pytest collects last.
"""
import numpy as np
import pytest

import synth

from _util import DD_TOL, normwise_vs, scales

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)
    return torch


def _device_system(torch, system):
    """The caller's own device copies of the system arrays, and a pe_system
    whose pointer fields hold their device addresses."""
    import paper_1201_0499_gb300 as pkg

    arrays = [
        torch.from_numpy(np.ascontiguousarray(system.poly_ptr, dtype=np.int64)).cuda(),
        torch.from_numpy(np.ascontiguousarray(system.mono_ptr, dtype=np.int64)).cuda(),
        torch.from_numpy(np.ascontiguousarray(system.pos, dtype=np.int32)).cuda(),
        torch.from_numpy(np.ascontiguousarray(system.exp, dtype=np.int32)).cuda(),
        torch.from_numpy(np.ascontiguousarray(system.coef, dtype=np.float64)).cuda(),
    ]
    ds = pkg.pe_system(system.n_vars, system.n_polys, *[a.data_ptr() for a in arrays])
    return ds, arrays


def test_noalloc_matches_eval_on_two_calls(torch_cuda):
    torch = torch_cuda
    import paper_1201_0499_gb300 as pkg

    system, _ = synth.config(2, n_points=1)
    n, N = system.n_vars, system.n_polys
    P = 200  # 13 tiles of 16 points, the last one ragged
    max_k = int(np.diff(system.mono_ptr).max())
    max_exp = int(system.exp.max())
    ds, keep = _device_system(torch, system)
    ref = pkg.PolyEval(system, pkg.PE_DD, max_points=P)
    for call, seed in enumerate((501, 502)):
        pts = synth.points(seed, n, P)
        x = torch.from_numpy(pts).cuda()
        f = torch.full((N, P, 4), float("nan"), dtype=torch.float64, device="cuda")
        J = torch.full((N, n, P, 4), float("nan"), dtype=torch.float64, device="cuda")
        pkg.polyeval_eval_noalloc(ds, max_k, max_exp, x, P, f, J)
        f_ref, J_ref = ref.eval(x)
        torch.cuda.synchronize()
        Sf, SJ = scales(system, pts)
        assert normwise_vs(f.cpu().numpy(), f_ref.cpu().numpy(), Sf) <= DD_TOL, call
        assert normwise_vs(J.cpu().numpy(), J_ref.cpu().numpy(), SJ) <= DD_TOL, call
    ref.close()
    del keep


def test_noalloc_rejects_sizes_beyond_the_scratch(torch_cuda):
    torch = torch_cuda
    import paper_1201_0499_gb300 as pkg

    system, _ = synth.config(2, n_points=1)
    ds, keep = _device_system(torch, system)
    x = torch.zeros((32, 8, 4), dtype=torch.float64, device="cuda")
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    # (max_exp - 2) * n * P complex double-doubles must fit in 16 MiB (524288 of them)
    with pytest.raises(pkg.PolyEvalError) as e:
        pkg.polyeval_eval_noalloc(ds, 9, 5, x, 6000, out, out)
    assert e.value.code == pkg.PE_ERANGE
    with pytest.raises(pkg.PolyEvalError) as e:
        pkg.polyeval_eval_noalloc(ds, 300, 5, x, 8, out, out)
    assert e.value.code == pkg.PE_ERANGE
    with pytest.raises(pkg.PolyEvalError) as e:
        pkg.polyeval_eval_noalloc(ds, 9, 5, 0, 8, out, out)
    assert e.value.code == pkg.PE_EINVAL
    del keep
