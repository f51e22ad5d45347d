"""Oracle eigen solver (balance + Hessenberg + Francis QR) against closed forms."""
import numpy as np
import pytest

from oracle import eig


def _match(a, b):
    """max over a of the distance to the nearest element of b (multiset-greedy)."""
    b = list(b)
    worst = 0.0
    for z in sorted(a, key=lambda v: (v.real, v.imag)):
        k = int(np.argmin([abs(z - w) for w in b]))
        worst = max(worst, abs(z - b[k]))
        b.pop(k)
    return worst


@pytest.mark.parametrize("H,D,K", [(3.0, 1.0, 1.5), (6.0, 0.0, 0.8), (2.0, 50.0, 1.0)])
def test_swing_2x2_closed_form(H, D, K):
    ws = 2 * np.pi * 60
    A = np.array([[0.0, ws], [-K / (2 * H), -D / (2 * H)]])
    lam, ok, _ = eig.eigvals(A)
    a, c = D / (2 * H), ws * K / (2 * H)
    disc = a * a - 4 * c
    root = np.sqrt(complex(disc))
    expect = [(-a + root) / 2, (-a - root) / 2]
    assert ok and _match(lam, expect) < 1e-12 * max(1, abs(c))


def test_companion_matrices_known_roots():
    rng = np.random.default_rng(2)
    for n in (3, 6, 9):
        re = rng.uniform(-3, 1, n // 3)
        im = rng.uniform(0.5, 4, n // 3)
        roots = np.concatenate([re + 1j * im, re - 1j * im, rng.uniform(-2, 2, n - 2 * (n // 3))])
        c = np.real(np.poly(roots))
        C = np.zeros((n, n))
        C[0, :] = -c[1:]
        C[1:, :-1] = np.eye(n - 1)
        lam, ok, _ = eig.eigvals(C)
        assert ok and _match(lam, roots) < 1e-7


def test_planted_spectrum():
    rng = np.random.default_rng(5)
    n = 40
    blocks = []
    lam_true = []
    for k in range(n // 2):
        s, w = rng.uniform(-2, 0.5), rng.uniform(0.1, 20)
        if k % 3 == 0:
            blocks.append(np.diag([s, s - 0.7]))
            lam_true += [s, s - 0.7]
        else:
            blocks.append(np.array([[s, w], [-w, s]]))
            lam_true += [s + 1j * w, s - 1j * w]
    Dm = np.zeros((n, n))
    for k, b in enumerate(blocks):
        Dm[2 * k:2 * k + 2, 2 * k:2 * k + 2] = b
    V = rng.normal(size=(n, n)) + 3 * np.eye(n)
    A = V @ Dm @ np.linalg.inv(V)
    lam, ok, _ = eig.eigvals(A)
    assert ok and _match(lam, np.array(lam_true)) < 1e-9 * np.abs(A).max()


@pytest.mark.parametrize("n", [5, 50, 270])
def test_random_against_numpy_and_trace(n):
    rng = np.random.default_rng(n)
    A = rng.normal(size=(n, n)) * np.exp(rng.uniform(-3, 3, size=(n, 1)))
    lam, ok, sweeps = eig.eigvals(A)
    assert ok
    assert abs(lam.sum().real - np.trace(A)) < 1e-10 * np.abs(A).sum()
    assert abs(lam.sum().imag) < 1e-10 * np.abs(A).sum()
    assert _match(lam, np.linalg.eigvals(A)) < 1e-10 * np.abs(A).max() * n


def test_hessenberg_form_is_orthogonal_similarity():
    rng = np.random.default_rng(9)
    A = rng.normal(size=(30, 30))
    Hs = eig.hessenberg(A, balance=False)
    assert np.abs(np.tril(Hs, -2)).max() == 0.0
    assert abs(np.linalg.norm(Hs) - np.linalg.norm(A)) < 1e-12 * np.linalg.norm(A)
    assert abs(np.trace(Hs) - np.trace(A)) < 1e-12 * np.abs(A).sum()


def test_balancing_is_exact_similarity():
    rng = np.random.default_rng(11)
    n = 12
    Dg = np.diag(2.0 ** rng.integers(-20, 20, n))
    A0 = rng.normal(size=(n, n))
    A = Dg @ A0 @ np.linalg.inv(Dg)
    lam, ok, _ = eig.eigvals(A, balance=True)
    assert ok and _match(lam, np.linalg.eigvals(A0)) < 1e-10


def test_stability_stats():
    lam = np.array([-1 + 10j, -1 - 10j, -0.2, -3 + 1j, -3 - 1j])
    mr, mz = eig.stability_stats(lam)
    assert mr == -0.2
    assert abs(mz - 1 / np.sqrt(101)) < 1e-15
    mr, mz = eig.stability_stats(np.array([0.3, -1.0]))
    assert mr == 0.3 and mz == -1.0
