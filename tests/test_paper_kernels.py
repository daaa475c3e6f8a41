"""The paper's own three-kernel design (create flag PE_PAPER_KERNELS,
Sections 3.1-3.3: common factors, Speelpenning products with coefficient
products scattered into the zero-padded Mons array, one thread per output
summing m terms), kept as a comparison for the fused kernel: same parity
bar against the exact oracle, and agreement with the fused kernel."""
import numpy as np
import pytest

import synth
from oracle import exact as E

from _util import DD_TOL, normwise_vs, scales, to_device

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)


def run_both(system, pts):
    import torch

    import paper_1201_0499_gb300 as pkg

    P = pts.shape[1]
    x = to_device(pts)
    paper = pkg.PolyEval(system, pkg.PE_DD, max_points=P, flags=pkg.PE_PAPER_KERNELS)
    fused = pkg.PolyEval(system, pkg.PE_DD, max_points=P)
    fp, Jp = paper.eval(x)
    ff, Jf = fused.eval(x)
    torch.cuda.synchronize()
    assert paper.status() == pkg.PE_OK
    return fp.cpu().numpy(), Jp.cpu().numpy(), ff.cpu().numpy(), Jf.cpu().numpy()


@pytest.mark.parametrize("cfg,P", [(2, 70), (1, 33)])
def test_three_kernels_match_oracle_and_fused(cfg, P):
    s, pts = synth.config(cfg, n_points=P)
    fp, Jp, ff, Jf = run_both(s, pts)
    ef, ej = E.max_errors(s, pts, fp, Jp, [0, P // 2, P - 1], polys=[0, s.n_polys - 1])
    assert ef <= DD_TOL and ej <= DD_TOL, (ef, ej)
    Sf, SJ = scales(s, pts)
    assert normwise_vs(fp, ff, Sf) <= 2 * DD_TOL
    assert normwise_vs(Jp, Jf, SJ) <= 2 * DD_TOL


def test_three_kernels_large_k():
    s, pts = synth.config(5, n_points=2)
    fp, Jp, ff, Jf = run_both(s, pts)
    ef, ej = E.max_errors(s, pts, fp, Jp, [1], polys=[7])
    assert ef <= DD_TOL and ej <= DD_TOL, (ef, ej)


def test_three_kernels_reject_irregular_systems():
    import paper_1201_0499_gb300 as pkg

    rng = np.random.Generator(np.random.PCG64(5))
    ragged = synth.from_monomials(4, [[([0, 1, 2], [1, 1, 1]), ([1, 2, 3], [2, 1, 1])], [([0, 1, 3], [1, 1, 1])]],
                                  synth.random_cdd(rng, 3))
    small_k = synth.from_monomials(4, [[([0, 1], [1, 1])], [([2, 3], [1, 2])]], synth.random_cdd(rng, 2))
    for s, prec in ((ragged, pkg.PE_DD), (small_k, pkg.PE_DD)):
        with pytest.raises(pkg.PolyEvalError) as e:
            pkg.PolyEval(s, prec, max_points=4, flags=pkg.PE_PAPER_KERNELS)
        assert e.value.code == pkg.PE_EINVAL
    s, _ = synth.config(2, n_points=1)
    with pytest.raises(pkg.PolyEvalError) as e:
        pkg.PolyEval(s.as_fp64(), pkg.PE_F64, max_points=4, flags=pkg.PE_PAPER_KERNELS)
    assert e.value.code == pkg.PE_EINVAL
