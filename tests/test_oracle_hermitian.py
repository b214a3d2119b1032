"""Pins (no GPU) for the complex Hermitian pencils (Peierls phases on the hopping and overlap
blocks) and the oracle pieces that handle them.

Pins come from outside the routines: a pure gauge (theta_ij = phi_i - phi_j) leaves the spectrum of
the real pencil unchanged; the spectrum of the real embedding [[Re M, -Im M], [Im M, Re M]] is the
complex spectrum with every eigenvalue twice (the identity the GPU path's inertia counts rest
on); the inertia count equals the count of the dense eigenvalues below sigma; the complex
derivatives match central finite differences of tied (Hermitian-preserving) real and imaginary
perturbations."""
import numpy as np
import pytest

from gen import make_pair
from oracle import core


def embed(M):
    """Real symmetric embedding of a Hermitian matrix (as a test-side restatement)."""
    return np.block([[M.real, -M.imag], [M.imag, M.real]])


@pytest.fixture(scope="module")
def herm():
    p = make_pair(2, 2, 2, seed=9, phases="peierls")       # n = 256
    A, B = p.A().toarray(), p.B().toarray()
    return p, A, B


def test_generator_hermitian_and_positive_definite(herm):
    p, A, B = herm
    assert A.dtype == np.complex128 and p.meta["phases"] == "peierls"
    assert np.abs(A - A.conj().T).max() == 0.0 and np.abs(B - B.conj().T).max() == 0.0
    assert np.linalg.eigvalsh(B).min() > 0.0
    q = make_pair(2, 2, 2, seed=9)
    assert np.array_equal(q.colind, p.colind) and np.array_equal(q.rowptr, p.rowptr)
    assert np.allclose(np.abs(p.a), np.abs(q.a), rtol=0, atol=1e-15)
    assert np.abs(A.imag).max() > 0.1                          # phases are really there


def test_gauge_phases_keep_the_real_spectrum():
    q = make_pair(2, 2, 2, seed=9)
    phi = np.random.default_rng(4).uniform(-np.pi, np.pi, q.meta["natom"])
    g = make_pair(2, 2, 2, seed=9, phases=phi)
    lam_r = core.gen_eig(q.A().toarray(), q.B().toarray())[0]
    lam_g, X = core.gen_eig(g.A().toarray(), g.B().toarray())
    assert np.abs(lam_r - lam_g).max() <= 1e-12 * np.abs(lam_r).max()
    # B-orthonormal complex eigenvectors
    Bg = g.B().toarray()
    assert np.abs(X.conj().T @ Bg @ X - np.eye(g.n)).max() <= 1e-11
    # a random (non-gauge) phase pattern changes the spectrum
    p = make_pair(2, 2, 2, seed=9, phases="peierls")
    lam_p = core.gen_eig(p.A().toarray(), p.B().toarray())[0]
    assert np.abs(lam_p - lam_r).max() > 1e-3


def test_real_embedding_doubles_the_spectrum(herm):
    p, A, B = herm
    lam = core.gen_eig(A, B)[0]
    lam2 = core.gen_eig(embed(A), embed(B))[0]
    assert np.abs(lam2[0::2] - lam).max() <= 1e-11 * np.abs(lam).max()
    assert np.abs(lam2[1::2] - lam).max() <= 1e-11 * np.abs(lam).max()
    # inertia: nu of the embedding is twice nu of the complex pencil, at any shift off the spectrum
    for sigma in (-3.0, lam[100] + 1e-3, 0.5 * (lam[127] + lam[128]), 4.0):
        nu = core.hermitian_nu(A, B, sigma)
        assert nu == core.count_below(lam, sigma)
        assert core.dense_nu(embed(A), embed(B), sigma) == 2 * nu


def test_complex_eig_grad_matches_finite_differences():
    rng = np.random.default_rng(12)
    n, k, h = 30, 11, 1e-6
    M = rng.normal(size=(n, n)) + 1j * rng.normal(size=(n, n))
    A = 0.5 * (M + M.conj().T)
    R = (rng.normal(size=(n, n)) + 1j * rng.normal(size=(n, n))) * 0.05
    B = np.eye(n) * 2.0 + 0.5 * (R + R.conj().T)
    lam, GA, GB = core.eig_grad(A, B, k)
    assert np.isclose(lam, core.gen_eig(A, B)[0][k - 1])
    scale = np.abs(GA).max()

    def lam_k(AA, BB):
        return core.gen_eig(AA, BB)[0][k - 1]

    for (i, j) in [(0, 0), (3, 7), (12, 25), (29, 29), (5, 21)]:
        Sr = np.zeros((n, n), complex); Sr[i, j] += 1.0
        if i != j:
            Sr[j, i] += 1.0
        fa = (lam_k(A + h * Sr, B) - lam_k(A - h * Sr, B)) / (2 * h)
        fb = (lam_k(A, B + h * Sr) - lam_k(A, B - h * Sr)) / (2 * h)
        ga = (GA[i, j] + GA[j, i]).real if i != j else GA[i, i].real
        gb = (GB[i, j] + GB[j, i]).real if i != j else GB[i, i].real
        assert abs(fa - ga) <= 1e-6 * scale, (i, j, fa, ga)
        assert abs(fb - gb) <= 1e-6 * scale * max(1.0, abs(lam)), (i, j, fb, gb)
        if i != j:                                 # i h at (i, j), -i h at (j, i): 2 Im G_ij
            Si = np.zeros((n, n), complex); Si[i, j] = 1j; Si[j, i] = -1j
            fi = (lam_k(A + h * Si, B) - lam_k(A - h * Si, B)) / (2 * h)
            assert abs(fi - 2 * GA[i, j].imag) <= 1e-6 * scale, (i, j, fi, GA[i, j])
    # the diagonal derivatives are real, |x_i|^2 (up to the rounding of the complex product)
    assert np.abs(np.diag(GA).imag).max() <= 1e-15 * scale
    assert np.allclose(np.diag(GA).real, np.abs(core.gen_eig(A, B)[1][:, k - 1]) ** 2, rtol=1e-12, atol=0)
