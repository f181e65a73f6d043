"""Plans with randomized-SVD low-rank blocks (Sec. 2.3, Alg. 1) on the GPU.

At the paper's starting rank (30) the trimmed non-oscillatory blocks of the
default plans are stored dense, so these plans force factorisation with a
small starting rank: every block kind of Sec. 3.3 then takes part (IDBF,
low-rank, trimmed dense), and each precision's kernels must still reproduce
the oracle's transform.
"""
import numpy as np
import pytest

import oracle
import paper_2004_11346_gb300 as sht
from paper_2004_11346_gb300 import _lib, inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def rel_err(a, b):
    a = np.asarray(a).reshape(a.shape[0], -1)
    b = np.asarray(b).reshape(b.shape[0], -1)
    return np.linalg.norm(a - b, axis=1) / np.linalg.norm(b, axis=1)


@pytest.mark.parametrize("prec,eps,tol,F", [(_lib.SHT_FP64, 1e-12, 1e-10, 2), (_lib.SHT_FP32, 1e-9, 1e-6, 9),
                                            (_lib.SHT_MIXED, 1e-9, 1e-6, 33)])
def test_low_rank_blocks(prec, eps, tol, F):
    N = 64
    p = sht.Plan(N, eps, precision=prec, n0=16, n_leaf=8, rsvd_r=4, max_fields=F,
                 flags=_lib.SHT_FLAG_FORCE_FACTOR)
    st = p.stats()
    assert st["n_blocks_lowrank"] > 0 and st["n_blocks_idbf"] > 0 and st["n_blocks_dense"] > 0
    beta = inputs.coefficients(N, F, seed=11)
    g = p.forward(torch.from_numpy(beta).cuda())
    back = p.inverse(g)
    torch.cuda.synchronize()
    p.sync()
    assert np.all(rel_err(g.cpu().numpy(), oracle.alt_forward(N, beta)) <= tol)
    gr = np.random.default_rng(12).standard_normal((F, 4 * N - 1, 2 * N, 2))
    b = p.inverse(torch.from_numpy(gr).cuda())
    torch.cuda.synchronize()
    assert np.all(rel_err(b.cpu().numpy(), oracle.alt_inverse(N, gr)) <= tol)
    assert np.all(rel_err(back.cpu().numpy(), beta) <= 2 * tol)
