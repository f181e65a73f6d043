"""GPU parity of the phi-direction DFT and the full SHT against the oracle.

The oracle's phi sums are direct O(M) sums per output with the angle reduced
exactly in integers; the GPU runs a mixed-radix shared-memory FFT over the
factors of M = 4N-1 (including prime M, e.g. N = 8: M = 31).
"""
import numpy as np
import pytest

import oracle
import paper_2004_11346_gb300 as sht
from paper_2004_11346_gb300 import _lib, inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = {_lib.SHT_FP64: 1e-10, _lib.SHT_FP32: 1e-6}


def rel_err(a, b):
    a = np.asarray(a).reshape(a.shape[0], -1)
    b = np.asarray(b).reshape(b.shape[0], -1)
    return np.linalg.norm(a - b, axis=1) / np.linalg.norm(b, axis=1)


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


@pytest.mark.parametrize("prec", [_lib.SHT_FP64, _lib.SHT_FP32])
# M = 3, 7, 31 (prime: generic pass), 39 = 3*13, 55 = 5*11, 63 = 3*3*7, 195 = 3*5*13,
# 255 = 3*5*17 (17: generic pass): every specialised radix that an odd M can have
@pytest.mark.parametrize("N", [1, 2, 8, 10, 14, 16, 49, 64])
def test_phi_synthesis_and_analysis(N, prec):
    p = sht.Plan(N, 1e-12 if prec == _lib.SHT_FP64 else 1e-7, precision=prec)
    rng = np.random.default_rng(N)
    F = 3
    g = rng.standard_normal((F, 4 * N - 1, 2 * N, 2))
    f = p.phi_synthesis(dev(g))
    torch.cuda.synchronize()
    assert np.all(rel_err(f.cpu().numpy(), oracle.phi_synthesis(N, g)) <= TOL[prec])
    fin = rng.standard_normal((F, 2 * N, 4 * N - 1, 2))
    g2 = p.phi_analysis(dev(fin))
    torch.cuda.synchronize()
    assert np.all(rel_err(g2.cpu().numpy(), oracle.phi_analysis(N, fin)) <= TOL[prec])


@pytest.mark.parametrize("prec", [_lib.SHT_FP64, _lib.SHT_FP32])
def test_sht_forward_inverse(prec):
    N = 32
    eps = 1e-12 if prec == _lib.SHT_FP64 else 1e-7
    # max_fields = 2 < F: the ALT values pass through the workspace in chunks
    p = sht.Plan(N, eps, precision=prec, max_fields=2, n0=16, n_leaf=8, flags=_lib.SHT_FLAG_FORCE_FACTOR)
    F = 5
    beta = inputs.coefficients(N, F, seed=7, real_m0=True)
    f = p.sht_forward(dev(beta))
    torch.cuda.synchronize()
    assert np.all(rel_err(f.cpu().numpy(), oracle.sht_forward(N, beta)) <= TOL[prec])
    fin = f.cpu().numpy()
    b = p.sht_inverse(dev(fin))
    torch.cuda.synchronize()
    assert np.all(rel_err(b.cpu().numpy(), oracle.sht_inverse(N, fin)) <= TOL[prec])
    assert np.all(rel_err(b.cpu().numpy(), beta) <= TOL[prec])


def test_sht_N64_fp64_workload():
    """N=64, eps=1e-12, one field, Re/Im N(0,1), beta_{k,0} real: forward and inverse SHT."""
    N = 64
    p = sht.Plan(N, 1e-12)
    beta = inputs.workload_coefficients("fp64_N64")
    f = p.sht_forward(dev(beta)).cpu().numpy()
    assert np.all(rel_err(f, oracle.sht_forward(N, beta)) <= 1e-10)
    b = p.sht_inverse(dev(f)).cpu().numpy()
    assert np.all(rel_err(b, oracle.sht_inverse(N, f)) <= 1e-10)


@pytest.mark.slow
def _rows_err(got, ref):
    """Relative l2 error of every (field, row) of arrays shaped (F, rows, ..., 2)."""
    d = np.linalg.norm((got - ref).reshape(got.shape[0], got.shape[1], -1), axis=2)
    return d / np.linalg.norm(ref.reshape(ref.shape[0], ref.shape[1], -1), axis=2)


# Rows longer than one CTA's shared memory are spread over a cluster of CTAs:
# M = 15015 = 3 5 7 11 13 (FP64, 240 KB), M = 16383 = 3 43 127 (FP64 with
# the generic pass and its second buffer: the order of the largest config),
# M = 29403 = 3^5 11^2 (FP32, 235 KB).  Phi-only plans: no ALT program.
@pytest.mark.parametrize("N,prec", [(3754, _lib.SHT_FP64), (4096, _lib.SHT_FP64), (7351, _lib.SHT_FP32)])
def test_phi_rows_split_over_a_cluster(N, prec):
    p = sht.Plan(N, 1e-12 if prec == _lib.SHT_FP64 else 1e-7, precision=prec, flags=_lib.SHT_FLAG_DIRECT)
    M, K = 4 * N - 1, 2 * N
    gen = torch.Generator(device="cuda")
    gen.manual_seed(N)
    g = torch.randn((1, M, K, 2), dtype=torch.float64, device="cuda", generator=gen)
    nodes = [0, 1, N, K - 1]
    f = p.phi_synthesis(g)
    ref = oracle.phi_synthesis_nodes(N, g[:, :, nodes].cpu().numpy())
    err = _rows_err(f[:, nodes].cpu().numpy(), ref)
    assert np.all(err <= TOL[prec]), err
    # analysis of the synthesis gives back every order at every node
    g2 = p.phi_analysis(f)
    assert float((g2 - g).norm() / g.norm()) <= TOL[prec]
    del f, g2
    fin = torch.randn((1, K, M, 2), dtype=torch.float64, device="cuda", generator=gen)
    ga = p.phi_analysis(fin)
    refa = oracle.phi_analysis_nodes(N, fin[:, nodes].cpu().numpy())
    erra = _rows_err(np.moveaxis(ga[:, :, nodes].cpu().numpy(), 2, 1), np.moveaxis(refa, 2, 1))
    assert np.all(erra <= TOL[prec]), erra
    del g, fin, ga
    torch.cuda.empty_cache()


def test_direct_plan_nodes_and_refusals():
    N = 8
    p = sht.Plan(N, 1e-12, flags=_lib.SHT_FLAG_DIRECT)
    x, w = p.nodes()
    xo, wo = oracle.gl_rule(2 * N)
    np.testing.assert_allclose(x, xo, atol=1e-14)
    np.testing.assert_allclose(w, wo, atol=1e-14)
    beta_m = dev(np.zeros((1, 2 * N - 3, 2)))
    for call in (lambda: p.forward_m(3, beta_m), lambda: p.save("/dev/null")):
        with pytest.raises(_lib.ShtError) as e:
            call()
        assert e.value.status == _lib.SHT_ERR_UNSUPPORTED
    with pytest.raises(_lib.ShtError):
        sht.Plan(N, 1e-12, flags=_lib.SHT_FLAG_DIRECT | _lib.SHT_FLAG_HOST_ONLY)


def test_phi_row_too_long_is_refused():
    # N = 16384 in FP64: M = 65535 = 3 5 17 257 needs the second buffer, 2 MB
    # per row, more than 8 CTAs hold; the call is refused before any launch
    p = sht.Plan(16384, 1e-12, flags=_lib.SHT_FLAG_DIRECT)
    buf = torch.zeros(16, dtype=torch.float64, device="cuda")
    with pytest.raises(_lib.ShtError) as e:
        _lib.sht_phi_synthesis(p.handle, buf.data_ptr(), buf.data_ptr(), 1, torch.cuda.current_stream().cuda_stream)
    assert e.value.status == _lib.SHT_ERR_UNSUPPORTED


def test_phi_N256():
    N = 256
    p = sht.Plan(N, 1e-12)
    g = np.random.default_rng(0).standard_normal((1, 4 * N - 1, 2 * N, 2))
    f = p.phi_synthesis(dev(g)).cpu().numpy()
    assert np.all(rel_err(f, oracle.phi_synthesis(N, g)) <= 1e-10)
