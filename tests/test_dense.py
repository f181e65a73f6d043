"""The plan builder's dense linear algebra against numpy (CPU).

csrc/dense.hpp holds the small FP64 routines of the precomputation: QR with
column pivoting (the rank-revealing factorisation behind the interpolative
decomposition, Sec. 2.1), the ID built from it, thin QR and the one-sided
Jacobi SVD of the randomized SVD (Sec. 2.3, Alg. 1), and the pseudo-inverse.
tests/native/dense_check.cpp runs them on matrices written here; the results
are checked against numpy's LAPACK routines and against identities that fix
them: R^T R = (A P)^T (A P), rank detection at the tolerance, the ID's
reconstruction error, orthonormal factors and the singular values.
"""
import os
import shutil
import subprocess

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(os.path.dirname(HERE), "paper_2004_11346_gb300", "csrc")


@pytest.fixture(scope="module")
def run(tmp_path_factory):
    if shutil.which("g++") is None:
        pytest.skip("g++ is missing")
    d = tmp_path_factory.mktemp("dense")
    exe = str(d / "dense_check")
    subprocess.run(["g++", "-O2", "-std=c++17", "-I", CSRC, os.path.join(HERE, "native", "dense_check.cpp"),
                    "-o", exe], check=True, capture_output=True, text=True)

    def call(mode, A, tol=0.0):
        A = np.asarray(A, dtype=np.float64)
        fin, fout = str(d / "in.bin"), str(d / "out.bin")
        with open(fin, "wb") as f:
            f.write(np.array(A.shape, dtype=np.int32).tobytes())
            f.write(np.asfortranarray(A).tobytes(order="F"))
        subprocess.run([exe, mode, fin, fout, repr(float(tol))], check=True, timeout=120)
        raw, mats, o = open(fout, "rb").read(), [], 0
        while o < len(raw):
            r, c = np.frombuffer(raw[o: o + 8], dtype=np.int32)
            o += 8
            mats.append(np.frombuffer(raw[o: o + 8 * r * c], dtype=np.float64).reshape((r, c), order="F"))
            o += 8 * r * c
        return mats
    return call


def low_rank(rng, m, n, r, decay=1.0):
    s = decay ** np.arange(r)
    return (rng.standard_normal((m, r)) * s) @ rng.standard_normal((r, n))


@pytest.mark.parametrize("m,n", [(40, 25), (25, 40), (30, 30), (1, 5), (7, 1)])
def test_pivoted_qr_is_a_qr_of_the_permuted_matrix(run, m, n):
    A = np.random.default_rng(m * 100 + n).standard_normal((m, n))
    k, perm, R = run("qr", A)
    k, perm = int(k[0, 0]), perm[0].astype(int)
    assert k == min(m, n) and sorted(perm) == list(range(n))
    AP = A[:, perm]
    # R^T R = (A P)^T (A P) fixes R up to the signs of its rows
    np.testing.assert_allclose(R.T @ R, AP.T @ AP, atol=1e-12 * np.abs(AP.T @ AP).max())
    assert np.allclose(np.tril(R, -1), 0.0)
    # the pivoting orders the diagonal by magnitude (greedy column norms)
    d = np.abs(np.diag(R))
    assert np.all(d[:-1] >= d[1:] * (1 - 1e-12))


@pytest.mark.parametrize("r", [1, 5, 12])
def test_pivoted_qr_detects_the_rank(run, r):
    rng = np.random.default_rng(r)
    A = low_rank(rng, 60, 40, r) + 1e-13 * rng.standard_normal((60, 40))
    k, _, _ = run("qr", A, 1e-9 * np.abs(A).max())
    assert int(k[0, 0]) == r


@pytest.mark.parametrize("tol", [1e-4, 1e-8, 1e-12])
def test_interpolative_decomposition(run, tol):
    # numerically low-rank matrix with geometrically decaying spectrum: the ID
    # keeps the columns whose pivoted residual exceeds tol, and reproduces A to
    # a small multiple of tol (Sec. 2.1)
    rng = np.random.default_rng(7)
    A = low_rank(rng, 80, 60, 40, decay=0.4)
    skel, V = run("id", A, tol)
    skel = skel[0].astype(int)
    k = len(skel)
    assert 0 < k < 40
    np.testing.assert_allclose(V[:, skel], np.eye(k), atol=0)
    # A - A(:, skel) V is the pivoted QR's trailing block R22 (rotated by Q),
    # whose columns the stopping rule left at norm <= tol each
    err = np.linalg.norm(A - A[:, skel] @ V, 2)
    assert err <= np.sqrt(60 - k) * tol * (1 + 1e-6), (err, tol)
    # a smaller tolerance keeps at least as many columns
    if tol > 1e-12:
        assert len(run("id", A, tol * 1e-4)[0][0]) >= k


@pytest.mark.parametrize("m,n", [(30, 10), (12, 12), (50, 3)])
def test_jacobi_svd(run, m, n):
    A = np.random.default_rng(m + n).standard_normal((m, n))
    U, s, V = run("svd", A)
    s = s[0]
    np.testing.assert_allclose(s, np.linalg.svd(A, compute_uv=False), rtol=1e-13)
    np.testing.assert_allclose(U.T @ U, np.eye(n), atol=1e-13)
    np.testing.assert_allclose(V.T @ V, np.eye(n), atol=1e-13)
    np.testing.assert_allclose(U * s @ V.T, A, atol=1e-13 * np.abs(A).max())


def test_jacobi_svd_of_a_rank_deficient_matrix(run):
    A = low_rank(np.random.default_rng(3), 20, 8, 3)
    _, s, _ = run("svd", A)
    s = s[0]
    np.testing.assert_allclose(s[:3], np.linalg.svd(A, compute_uv=False)[:3], rtol=1e-12)
    assert np.all(s[3:] <= 1e-13 * s[0])


@pytest.mark.parametrize("m,n", [(30, 10), (10, 10)])
def test_thin_q(run, m, n):
    A = np.random.default_rng(11).standard_normal((m, n))
    (Q,) = run("thinq", A)
    assert Q.shape == (m, n)
    np.testing.assert_allclose(Q.T @ Q, np.eye(n), atol=1e-14)
    np.testing.assert_allclose(Q @ (Q.T @ A), A, atol=1e-13)  # same column space


@pytest.mark.parametrize("shape", [(20, 6), (6, 20)])
def test_pinv(run, shape):
    A = low_rank(np.random.default_rng(5), *shape, 4)
    (P,) = run("pinv", A)
    np.testing.assert_allclose(P, np.linalg.pinv(A, rcond=1e-14), atol=1e-10 * np.abs(P).max())
