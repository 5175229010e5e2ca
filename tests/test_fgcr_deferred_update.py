"""The deferred solution update of the GPU FGCR, in numpy.  Each step the
GPU orthogonalises only w_k = A z_k (w_k -= sum_{j<k} beta_jk w_j, classical
Gram-Schmidt), stores beta and alpha_k = <w_k, r> / |w_k|^2, and updates r;
x is updated once per cycle by x += sum_j gamma_j z_j with gamma from the back
substitution gamma_k = a_k, a_j -= gamma_k beta_jk (k descending, a = alpha),
the same steps as its backsolve kernel.  This equals the textbook FGCR that
orthogonalises z alongside w and updates x every step, with a flexible
(step-dependent) preconditioner and a non-Hermitian A."""
import numpy as np
import pytest


def problem(seed, n=48):
    rng = np.random.default_rng(seed)
    A = 3 * np.eye(n) + 0.3 * (rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n)))
    P = np.linalg.inv(A) + 0.05 * (rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n)))
    b = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    return A, (lambda r, k: P @ r + 0.02 * k * r), b


def fgcr_explicit(A, M, b, K):
    x, r, W, Z = np.zeros_like(b), b.copy(), [], []
    for k in range(K):
        z = M(r, k)
        w = A @ z
        for wj, zj in zip(W, Z):
            beta = np.vdot(wj, w) / np.vdot(wj, wj)
            w, z = w - beta * wj, z - beta * zj
        alpha = np.vdot(w, r) / np.vdot(w, w)
        x, r = x + alpha * z, r - alpha * w
        W.append(w)
        Z.append(z)
    return x, r


def fgcr_deferred(A, M, b, K):
    r, W, Z = b.copy(), [], []
    beta = np.zeros((K, K), complex)
    alpha = np.zeros(K, complex)
    for k in range(K):
        z = M(r, k)
        w = A @ z
        for j, wj in enumerate(W):          # all dots first (classical Gram-Schmidt) ...
            beta[j, k] = np.vdot(wj, w) / np.vdot(wj, wj)
        for j, wj in enumerate(W):          # ... then one update pass
            w = w - beta[j, k] * wj
        alpha[k] = np.vdot(w, r) / np.vdot(w, w)
        r = r - alpha[k] * w
        W.append(w)
        Z.append(z)                          # stored as produced
    a, gamma = alpha.copy(), np.zeros(K, complex)
    for k in range(K - 1, -1, -1):
        gamma[k] = a[k]
        a[:k] -= gamma[k] * beta[:k, k]
    return sum(g * z for g, z in zip(gamma, Z)), r


@pytest.mark.parametrize("seed,K", [(0, 1), (1, 2), (2, 7), (3, 16), (4, 32)])
def test_deferred_update_equals_the_explicit_one(seed, K):
    A, M, b = problem(seed)
    x1, r1 = fgcr_explicit(A, M, b, K)
    x2, r2 = fgcr_deferred(A, M, b, K)
    assert np.linalg.norm(x2 - x1) <= 1e-12 * np.linalg.norm(x1)
    assert np.linalg.norm(r2 - r1) <= 1e-12 * np.linalg.norm(b)
    # and the recursive residual is the true one
    assert np.linalg.norm(r2 - (b - A @ x2)) <= 1e-12 * np.linalg.norm(b)


def test_a_transposed_coefficient_is_caught():
    """Planted mistake: beta_kj in place of beta_jk in the back substitution."""
    A, M, b = problem(5)
    K = 8
    x1, _ = fgcr_explicit(A, M, b, K)
    r, W, Z = b.copy(), [], []
    beta = np.zeros((K, K), complex)
    alpha = np.zeros(K, complex)
    for k in range(K):
        z = M(r, k)
        w = A @ z
        for j, wj in enumerate(W):
            beta[j, k] = np.vdot(wj, w) / np.vdot(wj, wj)
        for j, wj in enumerate(W):
            w = w - beta[j, k] * wj
        alpha[k] = np.vdot(w, r) / np.vdot(w, w)
        r = r - alpha[k] * w
        W.append(w)
        Z.append(z)
    a, gamma = alpha.copy(), np.zeros(K, complex)
    for k in range(K - 1, -1, -1):
        gamma[k] = a[k]
        a[:k] -= gamma[k] * beta[k, :k]
    x_bad = sum(g * z for g, z in zip(gamma, Z))
    assert np.linalg.norm(x_bad - x1) > 1e-6 * np.linalg.norm(x1)
