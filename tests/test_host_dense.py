"""Host dense algebra of the solvers (paper_2608_26875_b300/csrc/dense_host.h) against numpy, without a
GPU: the Cholesky factor and triangular inverse of the CholQR steps, the one-sided Jacobi eigen/SVD of the
rank-revealing deflation and of the time-reversal matrix, and the least-squares half of block GMRES (the
block Householder QR of the block Hessenberg matrix, the residual estimates and the truncated block back
substitution; Sec. 4.2 solves the coupled system by GMRES).  The header is compiled with g++ into the
harness tests/host_dense_check.cpp; numpy's factorizations and least-squares solver are the reference."""
import os
import shutil
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2608_26875_b300", "csrc")


@pytest.fixture(scope="module")
def harness(tmp_path_factory):
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("g++ not available")
    exe = str(tmp_path_factory.mktemp("dense") / "host_dense_check")
    subprocess.run([gxx, "-O2", "-std=c++17", "-fopenmp", "-I", CSRC,
                    os.path.join(ROOT, "tests", "host_dense_check.cpp"), "-o", exe], check=True)
    return exe


def run(exe, tmp_path, mode, *parts):
    src, dst = tmp_path / f"{mode}.in", tmp_path / f"{mode}.out"
    with open(src, "wb") as f:
        for p in parts:
            f.write(np.ascontiguousarray(p).tobytes())
    subprocess.run([exe, mode, str(src), str(dst)], check=True)
    return np.fromfile(dst, dtype=np.uint8)


def crandn(rng, *shape):
    return rng.normal(size=shape) + 1j * rng.normal(size=shape)


def block_hessenberg(rng, s, m):
    """(m+1)s x ms block upper-Hessenberg matrix as block Arnoldi builds it: dense blocks on and above the
    diagonal, upper-triangular blocks (CholQR factors) on the first subdiagonal, zero below."""
    H = np.zeros(((m + 1) * s, m * s), complex)
    for j in range(m):
        H[:(j + 1) * s, j * s:(j + 1) * s] = crandn(rng, (j + 1) * s, s)
        H[(j + 1) * s:(j + 2) * s, j * s:(j + 1) * s] = np.triu(crandn(rng, s, s)) + 3 * np.eye(s)
    return H


def lsq(exe, tmp_path, H, S0, floor_rel):
    s = S0.shape[0]
    m = H.shape[1] // s
    out = run(exe, tmp_path, "lsq", np.int32([s, m]), H.astype(complex), S0.astype(complex), np.float64([floor_rel]))
    Y = out[:m * s * s * 16].view(complex).reshape(m * s, s)
    res = out[m * s * s * 16:].view(np.float64)
    return Y, res


@pytest.mark.parametrize("s", [1, 8, 64])
def test_cholesky_factor_reproduces_the_gram_matrix(harness, tmp_path, s):
    rng = np.random.default_rng(s)
    A = crandn(rng, 3 * s, s)
    G = A.conj().T @ A
    out = run(harness, tmp_path, "chol", np.int32([s]), G)
    assert out[:4].view(np.int32)[0] == 1
    R = out[4:].view(complex).reshape(s, s)
    assert np.allclose(np.tril(R, -1), 0) and (np.diag(R).real > 0).all()
    assert np.abs(R.conj().T @ R - G).max() <= 1e-12 * np.abs(G).max()
    assert np.abs(R - np.linalg.cholesky(G).conj().T).max() <= 1e-11 * np.abs(R).max()


def test_cholesky_refuses_an_indefinite_matrix(harness, tmp_path):
    G = np.diag([2.0, 1.0, -1e-3, 4.0]).astype(complex)
    out = run(harness, tmp_path, "chol", np.int32([4]), G)
    assert out[:4].view(np.int32)[0] == 0


@pytest.mark.parametrize("s", [1, 7, 64])
def test_triangular_inverse(harness, tmp_path, s):
    rng = np.random.default_rng(10 + s)
    R = np.triu(crandn(rng, s, s)) + 4 * np.eye(s)
    Ri = run(harness, tmp_path, "triinv", np.int32([s]), R).view(complex).reshape(s, s)
    assert np.allclose(np.tril(Ri, -1), 0)
    assert np.abs(R @ Ri - np.eye(s)).max() <= 1e-12
    assert np.abs(Ri - np.linalg.inv(R)).max() <= 1e-12 * np.abs(Ri).max()


@pytest.mark.parametrize("n,rank", [(12, 12), (40, 40), (12, 5)])
def test_one_sided_jacobi_eigenpairs(harness, tmp_path, n, rank):
    """A V has orthogonal columns whose squared norms are the eigenvalues of A^H A; V is unitary; a
    rank-r matrix leaves n - r eigenvalues at rounding level."""
    rng = np.random.default_rng(n + rank)
    A = crandn(rng, n, rank) @ crandn(rng, rank, n)
    out = run(harness, tmp_path, "jacobi", np.int32([n]), A.T.copy())       # column-major in
    ev = out[:n * 8].view(np.float64)
    V = out[n * 8:n * 8 + n * n * 16].view(complex).reshape(n, n).T          # column-major out
    AV = out[n * 8 + n * n * 16:].view(complex).reshape(n, n).T
    assert np.abs(V.conj().T @ V - np.eye(n)).max() <= 1e-12
    assert np.abs(A @ V - AV).max() <= 1e-11 * np.abs(A).max()
    Gm = AV.conj().T @ AV
    off = Gm - np.diag(np.diag(Gm))
    assert np.abs(off).max() <= 1e-12 * ev.max()
    want = np.sort(np.linalg.eigvalsh(A.conj().T @ A))[::-1]
    got = np.sort(ev)[::-1]
    assert np.abs(got - want).max() <= 1e-11 * want[0]
    if rank < n:
        assert got[rank:].max() <= 1e-24 * got[0] * n


@pytest.mark.parametrize("s,m", [(1, 9), (4, 6), (16, 3)])
def test_block_gmres_least_squares_matches_numpy(harness, tmp_path, s, m):
    """Per column c: Y[:, c] minimises ||H y - [S0; 0][:, c]||; the residual estimate after the last step
    is that minimum."""
    rng = np.random.default_rng(100 * s + m)
    H = block_hessenberg(rng, s, m)
    S0 = np.triu(crandn(rng, s, s)) + 2 * np.eye(s)
    Y, res = lsq(harness, tmp_path, H, S0, 1e-14)
    G = np.zeros(((m + 1) * s, s), complex)
    G[:s] = S0
    want, *_ = np.linalg.lstsq(H, G, rcond=None)
    assert np.abs(Y - want).max() <= 1e-10 * np.abs(want).max()
    r_true = np.linalg.norm(H @ want - G, axis=0)
    assert np.abs(res - r_true).max() <= 1e-10 * np.linalg.norm(S0, axis=0).max()


def test_truncated_back_substitution_drops_an_unresolvable_direction(harness, tmp_path):
    """A last basis direction whose column is zero, or below the floor, gets a zero component; the
    others solve the least-squares problem of the remaining columns (numpy's minimum-norm solution)."""
    s, m = 4, 5
    rng = np.random.default_rng(7)
    for scale in (0.0, 1e-20):
        H = block_hessenberg(rng, s, m)
        H[:, -1] *= scale
        S0 = np.triu(crandn(rng, s, s)) + 2 * np.eye(s)
        Y, res = lsq(harness, tmp_path, H, S0, 1e-14)
        G = np.zeros(((m + 1) * s, s), complex)
        G[:s] = S0
        want = np.zeros_like(Y)
        want[:-1], *_ = np.linalg.lstsq(H[:, :-1], G, rcond=None)
        assert np.isfinite(Y).all()
        assert np.abs(Y[-1]).max() == 0.0
        assert np.abs(Y - want).max() <= 1e-10 * np.abs(want).max()


def test_least_squares_bar_is_sharp(harness, tmp_path):
    """The least-squares pin is sharp: the same comparison against a perturbed H (one entry of one
    subdiagonal block changed by 1e-6) misses by far more than its bar."""
    s, m = 4, 4
    rng = np.random.default_rng(3)
    H = block_hessenberg(rng, s, m)
    S0 = np.triu(crandn(rng, s, s)) + 2 * np.eye(s)
    Hp = H.copy()
    Hp[2 * s, s] += 1e-6
    Y, _ = lsq(harness, tmp_path, Hp, S0, 1e-14)
    G = np.zeros(((m + 1) * s, s), complex)
    G[:s] = S0
    want, *_ = np.linalg.lstsq(H, G, rcond=None)
    assert np.abs(Y - want).max() > 1e-9 * np.abs(want).max()
