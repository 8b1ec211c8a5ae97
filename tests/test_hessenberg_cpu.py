"""The host routine behind kd_growth_arnoldi's small eigenproblem (kd_hessenberg_eig: the
shifted QR algorithm on a complex upper Hessenberg matrix, eigenvectors from the Schur
form), checked on the CPU against numpy's LAPACK eigensolver and against the definition
H v = lambda v.  No GPU."""
import numpy as np
import pytest


@pytest.fixture(scope="module")
def kd():
    import __graft_entry__
    __graft_entry__.build()
    import paper_1902_00387_gb300 as kd
    kd.load()
    return kd


def hessenberg(m, seed, real=False):
    rng = np.random.default_rng(seed)
    h = rng.standard_normal((m, m)) + (0 if real else 1j * rng.standard_normal((m, m)))
    return np.triu(h, -1).astype(np.complex128)


def same_set(a, b, tol):
    a, b = list(a), list(b)
    for x in a:
        j = int(np.argmin([abs(x - y) for y in b]))
        assert abs(x - b[j]) <= tol * max(1.0, abs(x)), (x, b[j])
        b.pop(j)


@pytest.mark.parametrize("m", [1, 2, 3, 8, 31, 64])
@pytest.mark.parametrize("real", [False, True])
def test_eigenvalues_match_lapack(kd, m, real):
    h = hessenberg(m, 100 + m, real)
    same_set(kd.kd_hessenberg_eig(h), np.linalg.eigvals(h), 1e-10)


@pytest.mark.parametrize("m", [2, 8, 40])
def test_eigenvectors_satisfy_the_definition(kd, m):
    h = hessenberg(m, 200 + m)
    lam, v = kd.kd_hessenberg_eig(h, vectors=True)
    scale = np.linalg.norm(h, 2)
    for p in range(m):
        assert abs(np.linalg.norm(v[:, p]) - 1.0) < 1e-12
        assert np.linalg.norm(h @ v[:, p] - lam[p] * v[:, p]) < 1e-10 * scale, p


def test_special_cases(kd):
    # diagonal; a real rotation block (complex pair +-i); a nilpotent Jordan-like block
    d = np.diag([3.0, -1.0, 0.5 + 2j]).astype(np.complex128)
    same_set(kd.kd_hessenberg_eig(d), [3.0, -1.0, 0.5 + 2j], 1e-14)
    r = np.array([[0.0, -1.0], [1.0, 0.0]], np.complex128)
    same_set(kd.kd_hessenberg_eig(r), [1j, -1j], 1e-14)
    j = np.array([[2.0, 1.0, 0.0], [0.0, 2.0, 1.0], [0.0, 0.0, 2.0]], np.complex128)
    same_set(kd.kd_hessenberg_eig(j), [2.0, 2.0, 2.0], 1e-12)


def test_rejects_a_matrix_that_is_not_hessenberg(kd):
    h = hessenberg(4, 7)
    h[3, 0] = 1.0
    with pytest.raises(kd.KdError):
        kd.kd_hessenberg_eig(h)
