"""Plain numpy oracle of the learned preconditioner's building blocks (TEST
INFRASTRUCTURE ONLY): a parallel-transport convolution layer and flexible GCR.

Parallel-transport convolution (a gauge-equivariant linear layer).  A field
phi has C channels, each a spinor phi_i(x)[spin][colour].  With the
transports
    T_0 phi(x)       = phi(x)
    T_{+mu} phi(x)   = U_mu(x) phi(x+mu)
    T_{-mu} phi(x)   = U_mu(x-mu)^+ phi(x-mu)          (k = 1 + 2 mu + {0, 1})
the layer is
    out_o(x)[s'][c] = sum_{k, i, s} (T_k phi_i)(x)[s][c] W[k, i, s][o, s']
with complex weights W of shape (9, C_in, 4, C_out, 4) acting on channel and
spin only, never on colour, so that out transforms like phi under a gauge
transformation.  The boundary phases are applied with the links as in the
Dirac operator: a hop across the boundary of mu multiplies by exp(+-i phi_mu).

Flexible GCR (Notay 2000; generalised conjugate residual with a varying
preconditioner): z_k = M(r), w_k = D z_k, w_k and z_k orthogonalised against
the previous w_j (modified Gram-Schmidt), alpha = <w_k, r>/<w_k, w_k>,
x += alpha z_k, r -= alpha w_k, restart after m directions.
"""
import numpy as np


def _shift(dims, field, mu, step):
    """field(x + step*mu) on canonical (V, ...) arrays."""
    f = field.reshape(tuple(dims) + field.shape[1:])
    return np.roll(f, -step, axis=mu).reshape(field.shape)


def _edge(dims, mu, last):
    T, X, Y, Z = dims
    c = np.meshgrid(np.arange(T), np.arange(X), np.arange(Y), np.arange(Z), indexing="ij")[mu].reshape(-1)
    return c == (dims[mu] - 1 if last else 0)


def transports(lat, R, phi):
    """The 9 transported copies of phi (V, C, 4, d) -> (9, V, C, 4, d)."""
    out = [phi]
    for mu in range(4):
        fwd_ph = np.where(_edge(lat.dims, mu, True), np.exp(1j * lat.phase[mu]), 1.0)
        bwd_ph = np.where(_edge(lat.dims, mu, False), np.exp(-1j * lat.phase[mu]), 1.0)
        nxt = _shift(lat.dims, phi, mu, +1)
        out.append(fwd_ph[:, None, None, None] * np.einsum("vab,vcsb->vcsa", R[:, mu], nxt))
        Rb = _shift(lat.dims, R[:, mu], mu, -1)           # U_mu(x - mu)
        prv = _shift(lat.dims, phi, mu, -1)
        out.append(bwd_ph[:, None, None, None] * np.einsum("vba,vcsb->vcsa", np.conj(Rb), prv))
    return np.stack(out)


def ptc_layer(lat, R, phi, W):
    """out (V, C_out, 4, d) = sum over k, i, s of (T_k phi_i)[s] W[k, i, s, o, s']."""
    X = transports(lat, R, phi)
    return np.einsum("kvisc,kisot->votc", X, W)


def fgcr(apply_D, apply_M, b, tol=1e-10, max_iter=1000, restart=16):
    """Flexible GCR on D x = b with preconditioner M; returns (x, iterations,
    final |b - D x| / |b|)."""
    x = np.zeros_like(b)
    r = b.copy()
    bn = np.linalg.norm(b)
    it = 0
    Z, Wd = [], []
    while it < max_iter:
        if np.linalg.norm(r) <= tol * bn:
            break
        z = apply_M(r)
        w = apply_D(z)
        for zj, wj in zip(Z, Wd):
            beta = np.vdot(wj, w) / np.vdot(wj, wj)
            w = w - beta * wj
            z = z - beta * zj
        alpha = np.vdot(w, r) / np.vdot(w, w)
        x = x + alpha * z
        r = r - alpha * w
        Z.append(z)
        Wd.append(w)
        if len(Z) == restart:
            Z, Wd = [], []
        it += 1
    return x, it, np.linalg.norm(b - apply_D(x)) / bn
