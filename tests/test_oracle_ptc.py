"""Pins for the oracle of the learned preconditioner (oracle/ptc.py):
- with spin weights W_0 = A, W_{+mu} = -(1 - g_mu)/2, W_{-mu} = -(1 + g_mu)/2
  a one-channel parallel-transport layer IS the Wilson operator, so it must
  equal the (physics-pinned) oracle D: this fixes transport directions, link
  daggers, boundary phases and the spin contraction;
- with random weights the layer is gauge equivariant;
- flexible GCR with the identity preconditioner solves D x = b as a dense
  solve does, and with the exact inverse converges in one step."""
import numpy as np
import pytest

import oracle as orc
from oracle import ptc
from paper_1401_3733_gb300 import fields


def wilson_weights(m0):
    A = 4.0 + m0
    W = np.zeros((9, 1, 4, 1, 4), np.complex128)
    W[0, 0, :, 0, :] = A * np.eye(4)
    for mu in range(4):
        g = orc.gamma(mu)
        # out[s'] = sum_s X[s] W[s][s']  =>  W = M^T for out = M X
        W[1 + 2 * mu, 0, :, 0, :] = (-0.5 * (np.eye(4) - g)).T
        W[2 + 2 * mu, 0, :, 0, :] = (-0.5 * (np.eye(4) + g)).T
    return W


@pytest.mark.parametrize("dims,N,phase", [((4, 4, 2, 6), 3, (np.pi, 0.4, 0, -1.0)), ((2, 2, 2, 2), 2, (0, 0, 0, 0))])
def test_ptc_layer_with_wilson_weights_is_the_dirac_operator(dims, N, phase):
    lat = orc.Lattice(dims, N, orc.FUND, 0.1, phase)
    R = orc.links_to_rep(lat, fields.gauge_field(dims, N, "haar", seed=3))
    psi = fields.gaussian_spinor(dims, N, 4)
    out = ptc.ptc_layer(lat, R, psi[:, None], wilson_weights(lat.m0))[:, 0]
    want = orc.dirac(lat, R, psi)
    assert np.linalg.norm(out - want) / np.linalg.norm(want) < 1e-14


def test_ptc_layer_is_gauge_equivariant():
    dims, N, C_in, C_out = (4, 2, 4, 2), 3, 2, 3
    lat = orc.Lattice(dims, N, orc.FUND, 0.1, (np.pi, 0, 0, 0))
    U = fields.gauge_field(dims, N, "haar", seed=5)
    g = fields.gauge_transform(dims, N, 6)
    xs = fields.site_coords(dims)
    T, X, Y, Z = dims
    Ug = np.empty_like(U)
    for mu in range(4):
        c = xs.copy()
        c[:, mu] = (c[:, mu] + 1) % dims[mu]
        fwd = ((c[:, 0] * X + c[:, 1]) * Y + c[:, 2]) * Z + c[:, 3]
        Ug[:, mu] = g @ U[:, mu] @ np.conj(np.transpose(g[fwd], (0, 2, 1)))
    rng = np.random.default_rng(7)
    W = rng.standard_normal((9, C_in, 4, C_out, 4)) + 1j * rng.standard_normal((9, C_in, 4, C_out, 4))
    phi = rng.standard_normal((lat.V, C_in, 4, N)) + 1j * rng.standard_normal((lat.V, C_in, 4, N))
    rot = lambda f: np.einsum("vab,vcsb->vcsa", g, f)
    lhs = ptc.ptc_layer(lat, orc.links_to_rep(lat, Ug), rot(phi), W)
    rhs = rot(ptc.ptc_layer(lat, orc.links_to_rep(lat, U), phi, W))
    assert np.linalg.norm(lhs - rhs) / np.linalg.norm(rhs) < 1e-13


def test_fgcr_identity_and_exact_preconditioners():
    dims, N = (2, 2, 2, 2), 2
    lat = orc.Lattice(dims, N, orc.FUND, 0.1, (np.pi, 0, 0, 0))
    R = orc.links_to_rep(lat, fields.gauge_field(dims, N, "haar", seed=8))
    b = fields.gaussian_spinor(dims, N, 9)
    M = orc.dense_dirac(lat, R)
    x_ref = np.linalg.solve(M, b.reshape(-1)).reshape(b.shape)
    D = lambda v: orc.dirac(lat, R, v)
    x, it, res = ptc.fgcr(D, lambda r: r, b, tol=1e-12, restart=200)
    assert res <= 1e-12 and np.linalg.norm(x - x_ref) / np.linalg.norm(x_ref) < 1e-9
    Minv = np.linalg.inv(M)
    x1, it1, res1 = ptc.fgcr(D, lambda r: (Minv @ r.reshape(-1)).reshape(r.shape), b, tol=1e-12)
    assert it1 == 1 and res1 < 1e-12


def test_two_layers_compose_the_degree_two_neumann_polynomial():
    """Two layers (1 -> 2 -> 1 channels) with hand-set weights give
    M = (1 + K + K^2)/A, K = H/(2A) = (A - D)/A: the truncated series of
    D^{-1}.  Checked with the oracle's D only, on a lattice with phases."""
    dims, N = (4, 2, 4, 2), 3
    lat = orc.Lattice(dims, N, orc.FUND, -0.3, (np.pi, 0.2, 0, 0))
    R = orc.links_to_rep(lat, fields.gauge_field(dims, N, "haar", seed=31))
    A = 4.0 + lat.m0
    W1 = np.zeros((9, 1, 4, 2, 4), np.complex128)
    W2 = np.zeros((9, 2, 4, 1, 4), np.complex128)
    W1[0, 0, :, 0, :] = np.eye(4)
    W2[0, 0, :, 0, :] = W2[0, 1, :, 0, :] = np.eye(4) / A
    for mu in range(4):
        g = orc.gamma(mu)
        for k, P in ((1 + 2 * mu, np.eye(4) - g), (2 + 2 * mu, np.eye(4) + g)):
            W1[k, 0, :, 1, :] = (P / (2 * A)).T
            W2[k, 1, :, 0, :] = (P / (2 * A * A)).T
    psi = fields.gaussian_spinor(dims, N, 32)
    out = ptc.ptc_layer(lat, R, ptc.ptc_layer(lat, R, psi[:, None], W1), W2)[:, 0]
    K = lambda v: (A * v - orc.dirac(lat, R, v)) / A
    Kp = K(psi)
    want = (psi + Kp + K(Kp)) / A
    assert np.linalg.norm(out - want) / np.linalg.norm(want) < 1e-14
    # and D M = 1 - K^3 (the residual operator of the truncation)
    res = orc.dirac(lat, R, out) - psi
    assert np.linalg.norm(res + K(K(Kp))) / np.linalg.norm(psi) < 1e-13
