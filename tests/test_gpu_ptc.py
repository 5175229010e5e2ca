"""GPU learned preconditioner and flexible GCR through the C ABI:
- the two-layer parallel-transport network against the oracle's layers
  (FP32 and BF16 inference), and against the degree-2 Neumann polynomial of
  the Wilson operator that it represents exactly with hand-set weights
  (checked with the oracle's D alone);
- the training gradient against central differences of the oracle's loss
  (exact for a loss quadratic along the direction), one Adam step against
  its formula, and a short training run that lowers the loss;
- FGCR without preconditioner against the oracle's FGCR, FGCR with the
  network converging to the same solution in fewer iterations, and the
  error statuses."""
import numpy as np
import pytest
import torch

import oracle as orc
from oracle import ptc
from paper_1401_3733_gb300 import bsm, fields
from tests.gpu_helpers import gpu_links, gpu_spinor, rel, to_canon, zeros_field

pytestmark = pytest.mark.gpu

CASES = [((4, 4, 4, 6), 3, bsm.FUND, (np.pi, 0.4, 0, -1.0)), ((4, 4, 4, 4), 2, bsm.FUND, (np.pi, 0, 0, 0)),
         ((2, 4, 4, 2), 2, bsm.SYM, (0.3, 0, 0, 0)), ((4, 4, 4, 2), 3, bsm.ASYM, (np.pi, 0, 0.7, 0))]
CASE_IDS = ["SU3-F", "SU2-F", "SU2-S", "SU3-AS"]


def lats(dims, N, rep, phase, m0=0.1):
    return orc.Lattice(dims, N, rep, m0, phase), bsm.lattice(dims, N, rep, m0, phase)


def rand_c(rng, shape, scale=1.0):
    return scale * (rng.standard_normal(shape) + 1j * rng.standard_normal(shape))


def dev_c64(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.complex64)).to("cuda")


def ptc_field(blat, psis):
    """canonical spinors (nb, V, 4, d) -> nb-sample one-channel PTC field"""
    nb = len(psis)
    V = int(np.prod(list(blat.dims)))
    d = bsm.bsm_rep_dim(blat.N, blat.rep)
    F = torch.empty(nb * V * d * 4, dtype=torch.complex64, device="cuda")
    for b, psi in enumerate(psis):
        bsm.bsm_ptc_pack(blat, gpu_spinor(blat, psi, bsm.F64), F[b * V * d * 4:(b + 1) * V * d * 4])
    return F


def from_ptc_field(blat, F, nb):
    V = int(np.prod(list(blat.dims)))
    d = bsm.bsm_rep_dim(blat.N, blat.rep)
    out = []
    for b in range(nb):
        psi = zeros_field(blat, bsm.FIELD_SPINOR, bsm.F64)
        bsm.bsm_ptc_unpack(blat, F[b * V * d * 4:(b + 1) * V * d * 4], psi)
        out.append(to_canon(blat, psi, bsm.F64))
    return np.stack(out)


def gpu_net(blat, U32, W1, W2, C, psis, prec):
    nb = len(psis)
    F = ptc_field(blat, psis)
    out = torch.empty_like(F)
    ws = torch.empty(bsm.bsm_ptc_workspace_bytes(blat, C, nb, 0), dtype=torch.uint8, device="cuda")
    bsm.bsm_ptc_apply(blat, U32, dev_c64(W1), dev_c64(W2), C, F, out, nb, prec, ws)
    return from_ptc_field(blat, out, nb)


def oracle_net(olat, R, psi, W1, W2, C):
    y1 = ptc.ptc_layer(olat, R, psi[:, None], W1.reshape(9, 1, 4, C, 4))
    return ptc.ptc_layer(olat, R, y1, W2.reshape(9, C, 4, 1, 4))[:, 0]


def neumann_weights(m0):
    """C = 2 weights with M = (1 + K + K^2)/A, K = H/(2A): the degree-2
    truncation of D^{-1} = (A - H/2)^{-1} = (1/A) sum_n K^n."""
    A = 4.0 + m0
    W1 = np.zeros((9, 1, 4, 2, 4), np.complex128)
    W2 = np.zeros((9, 2, 4, 1, 4), np.complex128)
    W1[0, 0, :, 0, :] = np.eye(4)                       # channel 0 = phi
    W2[0, 0, :, 0, :] = np.eye(4) / A                   # out = phi/A + ...
    W2[0, 1, :, 0, :] = np.eye(4) / A                   # ... + K phi / A + ...
    for mu in range(4):
        g = orc.gamma(mu)
        for k, P in ((1 + 2 * mu, np.eye(4) - g), (2 + 2 * mu, np.eye(4) + g)):
            W1[k, 0, :, 1, :] = (P / (2 * A)).T          # channel 1 = K phi
            W2[k, 1, :, 0, :] = (P / (2 * A * A)).T      # ... + K^2 phi / A
    return W1.reshape(36, 8), W2.reshape(72, 4)


@pytest.mark.parametrize("C", [5, 12], ids=["C5", "C12"])
@pytest.mark.parametrize("prec,tol", [(bsm.F32, 1e-5), (bsm.BF16, 2e-2)], ids=["f32", "bf16"])
@pytest.mark.parametrize("case", CASES, ids=CASE_IDS)
def test_ptc_net_matches_oracle_layers(case, prec, tol, C):
    """C = 12 in BF16 runs the fused transport + two-GEMM kernel, C = 5 the
    transport kernels and library GEMMs; the lattices give parity blocks of
    192, 128, 32 and 64 sites against the fused kernel's 128-site tiles
    (ragged, exact and partial), and two samples per call."""
    dims, N, rep, phase = case
    olat, blat = lats(dims, N, rep, phase)
    U = fields.gauge_field(dims, N, "haar", seed=11)
    R = orc.links_to_rep(olat, U)
    U32 = gpu_links(blat, U, bsm.F32)
    rng = np.random.default_rng(12)
    W1, W2 = rand_c(rng, (36, 4 * C), 0.3), rand_c(rng, (36 * C, 4), 0.1)
    psis = [fields.gaussian_spinor(dims, olat.d, 13 + b) for b in range(2)]
    got = gpu_net(blat, U32, W1, W2, C, psis, prec)
    for b in range(2):
        want = oracle_net(olat, R, psis[b], W1, W2, C)
        assert rel(got[b], want) < tol


@pytest.mark.parametrize("C", [2, 4, 8], ids=["C2", "C4", "C8"])
def test_ptc_net_fused_kernel_other_channel_counts(C):
    """The fused BF16 kernel at its other channel counts (GEMM widths 8C =
    16, 32, 64 and GEMM2 depths 8C), against the oracle's two layers."""
    dims, N, rep, phase = CASES[0]
    olat, blat = lats(dims, N, rep, phase)
    U = fields.gauge_field(dims, N, "haar", seed=11)
    R = orc.links_to_rep(olat, U)
    U32 = gpu_links(blat, U, bsm.F32)
    rng = np.random.default_rng(50 + C)
    W1, W2 = rand_c(rng, (36, 4 * C), 0.3), rand_c(rng, (36 * C, 4), 0.1)
    psis = [fields.gaussian_spinor(dims, olat.d, 60 + b) for b in range(2)]
    got = gpu_net(blat, U32, W1, W2, C, psis, bsm.BF16)
    for b in range(2):
        assert rel(got[b], oracle_net(olat, R, psis[b], W1, W2, C)) < 2e-2


def test_ptc_net_fused_kernel_walks_several_tiles_per_block():
    """12 x 10^3 SU(3), 4 samples: parity blocks of 6000 sites give 47 tiles
    of 128 sites (the last one ragged, 112 sites), 376 tiles in all, so each
    block of the persistent fused kernel takes two or three tiles and both
    of its shared-memory buffers are refilled."""
    dims, N, rep, phase = (12, 10, 10, 10), 3, bsm.FUND, (np.pi, 0, 0.3, 0)
    olat, blat = lats(dims, N, rep, phase)
    U = fields.gauge_field(dims, N, "smooth", seed=40, eps=0.5)
    R = orc.links_to_rep(olat, U)
    U32 = gpu_links(blat, U, bsm.F32)
    rng = np.random.default_rng(41)
    C = 12
    W1, W2 = rand_c(rng, (36, 4 * C), 0.3), rand_c(rng, (36 * C, 4), 0.1)
    psis = [fields.gaussian_spinor(dims, olat.d, 42 + b) for b in range(4)]
    got = gpu_net(blat, U32, W1, W2, C, psis, bsm.BF16)
    for b in range(4):
        assert rel(got[b], oracle_net(olat, R, psis[b], W1, W2, C)) < 2e-2


@pytest.mark.parametrize("prec,tol", [(bsm.F32, 1e-5), (bsm.BF16, 1e-2)], ids=["f32", "bf16-fused"])
def test_ptc_net_with_neumann_weights_is_the_polynomial_of_d(prec, tol):
    dims, N, rep, phase = CASES[0]
    olat, blat = lats(dims, N, rep, phase, m0=-0.3)
    U = fields.gauge_field(dims, N, "haar", seed=14)
    R = orc.links_to_rep(olat, U)
    A = 4.0 + olat.m0
    psi = fields.gaussian_spinor(dims, olat.d, 15)
    K = lambda v: (A * v - orc.dirac(olat, R, v)) / A      # K = H / (2A) = (A - D)/A
    Kpsi = K(psi)
    want = (psi + Kpsi + K(Kpsi)) / A
    W1, W2 = neumann_weights(olat.m0)
    got = gpu_net(blat, gpu_links(blat, U, bsm.F32), W1, W2, 2, [psi], prec)[0]
    assert rel(got, want) < tol


def _loss_oracle(olat, R, rs, es, W1, W2, C):
    return sum(np.linalg.norm(oracle_net(olat, R, r, W1, W2, C) - e) ** 2 / np.linalg.norm(e) ** 2
               for r, e in zip(rs, es))


def test_ptc_gradient_against_central_differences():
    dims, N, rep, phase = (4, 4, 4, 4), 3, bsm.FUND, (np.pi, 0, 0, 0)
    olat, blat = lats(dims, N, rep, phase)
    U = fields.gauge_field(dims, N, "smooth", seed=16, eps=0.5)
    R = orc.links_to_rep(olat, U)
    U32 = gpu_links(blat, U, bsm.F32)
    rng = np.random.default_rng(17)
    C, nb = 3, 2
    W1, W2 = rand_c(rng, (36, 4 * C), 0.2), rand_c(rng, (36 * C, 4), 0.1)
    rs = [fields.gaussian_spinor(dims, 3, 18 + b) for b in range(nb)]
    es = [fields.gaussian_spinor(dims, 3, 28 + b) for b in range(nb)]
    G1 = torch.empty((36, 4 * C), dtype=torch.complex64, device="cuda")
    G2 = torch.empty((36 * C, 4), dtype=torch.complex64, device="cuda")
    ws = torch.empty(bsm.bsm_ptc_workspace_bytes(blat, C, nb, 1), dtype=torch.uint8, device="cuda")
    loss = bsm.bsm_ptc_loss_grad(blat, U32, dev_c64(W1), dev_c64(W2), C, ptc_field(blat, rs), ptc_field(blat, es),
                                 nb, G1, G2, ws)
    L0 = _loss_oracle(olat, R, rs, es, W1, W2, C)
    assert abs(loss - L0) / L0 < 1e-5
    g1, g2 = G1.cpu().numpy().astype(np.complex128), G2.cpu().numpy().astype(np.complex128)
    h = 1e-3
    # directional derivatives along random directions (loss quadratic in t)
    for which in (1, 2):
        D = rand_c(rng, W1.shape if which == 1 else W2.shape)
        if which == 1:
            f = lambda t: _loss_oracle(olat, R, rs, es, W1 + t * D, W2, C)
            g = g1
        else:
            f = lambda t: _loss_oracle(olat, R, rs, es, W1, W2 + t * D, C)
            g = g2
        fd = (f(h) - f(-h)) / (2 * h)
        an = float(np.real(np.vdot(g, D)))
        assert abs(fd - an) <= 1e-4 * (abs(fd) + np.linalg.norm(g) * np.linalg.norm(D) * 1e-2), (which, fd, an)
    # single entries, real and imaginary parts
    for which, W, g in ((1, W1, g1), (2, W2, g2)):
        for j in rng.choice(W.size, 3, replace=False):
            for unit, part in ((1.0, np.real), (1j, np.imag)):
                D = np.zeros_like(W)
                D.reshape(-1)[j] = unit
                if which == 1:
                    fd = (_loss_oracle(olat, R, rs, es, W1 + h * D, W2, C) -
                          _loss_oracle(olat, R, rs, es, W1 - h * D, W2, C)) / (2 * h)
                else:
                    fd = (_loss_oracle(olat, R, rs, es, W1, W2 + h * D, C) -
                          _loss_oracle(olat, R, rs, es, W1, W2 - h * D, C)) / (2 * h)
                an = part(g.reshape(-1)[j])
                assert abs(fd - an) <= 1e-4 * np.abs(g).max(), (which, j, fd, an)


def test_adam_step_formula():
    rng = np.random.default_rng(19)
    n = 1000
    W, G = rng.standard_normal(n).astype(np.float32), rng.standard_normal(n).astype(np.float32)
    m, v = (0.1 * rng.standard_normal(n)).astype(np.float32), rng.random(n).astype(np.float32)
    tW, tG, tm, tv = (torch.from_numpy(a.copy()).cuda() for a in (W, G, m, v))
    bsm.bsm_ptc_adam_step(tW, tG, tm, tv, 1e-2, 3)
    m1 = 0.9 * m + 0.1 * G
    v1 = 0.999 * v + 0.001 * G * G
    W1 = W - 1e-2 * (m1 / (1 - 0.9 ** 3)) / (np.sqrt(v1 / (1 - 0.999 ** 3)) + 1e-8)
    assert np.allclose(tm.cpu().numpy(), m1, rtol=1e-6, atol=1e-7)
    assert np.allclose(tv.cpu().numpy(), v1, rtol=1e-6, atol=1e-7)
    assert np.allclose(tW.cpu().numpy(), W1, rtol=1e-5, atol=1e-6)


def train(blat, U64, U32, C, steps, nb, seed, lr=3e-3):
    """Adam on loss = sum |M(D e) - e|^2 / |e|^2 over Gaussian e (drawn on the
    host with the seeded generator; D e by the library's FP64 operator)."""
    V = int(np.prod(list(blat.dims)))
    d = bsm.bsm_rep_dim(blat.N, blat.rep)
    es = [fields.gaussian_spinor(tuple(blat.dims), d, seed + b) for b in range(nb)]
    rs = []
    for e in es:
        out = zeros_field(blat, bsm.FIELD_SPINOR, bsm.F64)
        bsm.bsm_dslash(blat, U64, gpu_spinor(blat, e, bsm.F64), out, bsm.FULL, 0, bsm.F64)
        rs.append(to_canon(blat, out, bsm.F64))
    R, E = ptc_field(blat, rs), ptc_field(blat, es)
    rng = np.random.default_rng(seed)
    A = 4.0 + blat.m0
    W1 = rand_c(rng, (9, 1, 4, C, 4), 0.05)
    W1[0, 0, :, 0, :] += np.eye(4)
    W2 = rand_c(rng, (9, C, 4, 1, 4), 0.01)
    W2[0, 0, :, 0, :] += np.eye(4) / A
    tW = [dev_c64(W1.reshape(36, 4 * C)), dev_c64(W2.reshape(36 * C, 4))]
    tG = [torch.empty_like(t) for t in tW]
    tm = [torch.zeros_like(t) for t in tW]
    tv = [torch.zeros_like(t) for t in tW]
    ws = torch.empty(bsm.bsm_ptc_workspace_bytes(blat, C, nb, 1), dtype=torch.uint8, device="cuda")
    losses = []
    for step in range(1, steps + 1):
        losses.append(bsm.bsm_ptc_loss_grad(blat, U32, tW[0], tW[1], C, R, E, nb, tG[0], tG[1], ws) / nb)
        for k in range(2):
            bsm.bsm_ptc_adam_step(tW[k], tG[k], tm[k], tv[k], lr, step)
    return tW, losses


def test_training_lowers_the_loss():
    dims = (4, 4, 4, 4)
    blat = bsm.lattice(dims, 3, bsm.FUND, -0.2, (np.pi, 0, 0, 0))
    U = fields.gauge_field(dims, 3, "smooth", seed=20, eps=0.4)
    U64, U32 = gpu_links(blat, U, bsm.F64), gpu_links(blat, U, bsm.F32)
    _, losses = train(blat, U64, U32, C=4, steps=150, nb=4, seed=21)
    assert np.all(np.isfinite(losses))
    assert losses[-1] < 0.5 * losses[0], (losses[0], losses[-1])


def fgcr(blat, U64, U32, b_dev, opts, W=(None, None)):
    x = zeros_field(blat, bsm.FIELD_SPINOR, bsm.F64)
    ws = torch.empty(bsm.bsm_fgcr_workspace_bytes(blat, opts), dtype=torch.uint8, device="cuda")
    st, stats = bsm.bsm_fgcr_solve(blat, U64, U32, W[0], W[1], b_dev, x, opts, ws, raise_on_error=False)
    return st, stats, x


@pytest.mark.parametrize("restart", [8, 7], ids=["restart8", "restart7"])
def test_fgcr_without_preconditioner_matches_oracle(restart):
    """An odd restart puts an odd number of FP64 norms in the scalar block:
    its 16-byte arrays must stay aligned."""
    dims, N = (4, 4, 4, 4), 2
    olat, blat = lats(dims, N, bsm.FUND, (np.pi, 0, 0, 0))
    U = fields.gauge_field(dims, N, "haar", seed=22)
    R = orc.links_to_rep(olat, U)
    b = fields.gaussian_spinor(dims, N, 23)
    x_ref, it_ref, res_ref = ptc.fgcr(lambda v: orc.dirac(olat, R, v), lambda r: r, b, tol=1e-10, restart=restart)
    st, stats, x = fgcr(blat, gpu_links(blat, U, bsm.F64), None, gpu_spinor(blat, b, bsm.F64),
                        bsm.fgcr_opts(tol=1e-10, restart=restart))
    assert st == bsm.OK
    assert abs(stats.iters - it_ref) <= 2, (stats.iters, it_ref)
    assert stats.true_res <= 2e-10
    xg = to_canon(blat, x, bsm.F64)
    assert rel(xg, x_ref) < 1e-8
    assert rel(orc.dirac(olat, R, xg), b) < 2e-10


@pytest.mark.parametrize("prec", [bsm.F32, bsm.BF16], ids=["f32", "bf16"])
def test_fgcr_with_ptc_preconditioner_converges_faster(prec):
    dims, N = (4, 4, 4, 8), 3
    olat, blat = lats(dims, N, bsm.FUND, (np.pi, 0, 0, 0), m0=0.05)
    U = fields.gauge_field(dims, N, "smooth", seed=24, eps=0.4)
    R = orc.links_to_rep(olat, U)
    U64, U32 = gpu_links(blat, U, bsm.F64), gpu_links(blat, U, bsm.F32)
    b = fields.gaussian_spinor(dims, N, 25)
    bd = gpu_spinor(blat, b, bsm.F64)
    st0, s0, x0 = fgcr(blat, U64, None, bd, bsm.fgcr_opts(tol=1e-10, restart=16))
    W1, W2 = neumann_weights(olat.m0)
    st1, s1, x1 = fgcr(blat, U64, U32, bd,
                       bsm.fgcr_opts(tol=1e-10, restart=16, precond=bsm.FGCR_PTC, ptc_prec=prec, channels=2),
                       (dev_c64(W1), dev_c64(W2)))
    assert st0 == bsm.OK and st1 == bsm.OK
    assert s1.true_res <= 2e-10
    assert s1.iters < s0.iters, (s1.iters, s0.iters)
    x = to_canon(blat, x1, bsm.F64)
    assert rel(orc.dirac(olat, R, x), b) < 2e-10
    assert rel(x, to_canon(blat, x0, bsm.F64)) < 1e-8


def test_fgcr_statuses():
    dims, N = (4, 4, 4, 4), 2
    _, blat = lats(dims, N, bsm.FUND, (0, 0, 0, 0))
    U64 = gpu_links(blat, fields.gauge_field(dims, N, "haar", seed=26), bsm.F64)
    b = fields.gaussian_spinor(dims, N, 27)
    st, stats, _ = fgcr(blat, U64, None, gpu_spinor(blat, b, bsm.F64), bsm.fgcr_opts(tol=1e-12, max_iter=2))
    assert st == bsm.ENOCONV and stats.iters == 2
    st, stats, x = fgcr(blat, U64, None, zeros_field(blat, bsm.FIELD_SPINOR, bsm.F64), bsm.fgcr_opts())
    assert st == bsm.OK and stats.iters == 0 and float(x.abs().max()) == 0.0
    bn = b.copy()
    bn[3, 1, 0] = np.nan
    st, _, _ = fgcr(blat, U64, None, gpu_spinor(blat, bn, bsm.F64), bsm.fgcr_opts())
    assert st == bsm.ENAN


@pytest.mark.parametrize("cause", ["max_iter", "nan_weights"])
@pytest.mark.parametrize("eo", [True, False], ids=["eo", "full"])
def test_fgcr_falls_back_to_cg(cause, eo):
    """With opts.fallback, an FGCR solve that ends in BSM_ENOCONV (max_iter = 1)
    or BSM_ENAN (a NaN in the network's weights, planted on the host) is
    finished by the plain CG solver on the normal equations: the call returns
    OK, reports FGCR's own status and the CG iterations, and x solves D x = b
    (checked with the oracle's D).  Without fallback the same call fails."""
    dims, N = (4, 4, 4, 8), 3
    olat, blat = lats(dims, N, bsm.FUND, (np.pi, 0, 0, 0), m0=0.05)
    U = fields.gauge_field(dims, N, "smooth", seed=24, eps=0.4)
    R = orc.links_to_rep(olat, U)
    U64, U32 = gpu_links(blat, U, bsm.F64), gpu_links(blat, U, bsm.F32)
    b = fields.gaussian_spinor(dims, N, 25)
    bd = gpu_spinor(blat, b, bsm.F64)
    W1, W2 = neumann_weights(olat.m0)
    if cause == "nan_weights":
        W1 = W1.copy()
        W1[3, 1] = np.nan
    W = (dev_c64(W1), dev_c64(W2))
    kw = dict(tol=1e-11, restart=16, precond=bsm.FGCR_PTC, ptc_prec=bsm.BF16, channels=2, eo=eo,
              prec_inner=bsm.F32, inner_tol=1e-3, max_iter=1 if cause == "max_iter" else 1000)
    want = bsm.ENOCONV if cause == "max_iter" else bsm.ENAN
    st, _, _ = fgcr(blat, U64, U32, bd, bsm.fgcr_opts(**kw), W)
    assert st == want
    st, stats, x = fgcr(blat, U64, U32, bd, bsm.fgcr_opts(fallback=True, **kw), W)
    assert st == bsm.OK, bsm.bsm_strerror(st)
    assert stats.fgcr_status == want and stats.fallback_iters > 0
    assert stats.true_res <= 1e-9
    assert rel(orc.dirac(olat, R, to_canon(blat, x, bsm.F64)), b) <= 1e-9


def test_fused_kernel_wait_that_gives_up_is_reported(monkeypatch):
    """BSM_PTC_WAIT_POLLS=0 makes the first MMA-completion wait of every
    block of the fused BF16 kernel give up at once: the block waits (bounded)
    for its MMAs in flight, issues no more, stores NaN and sets the
    workspace's error word, which bsm_ptc_status reports as BSM_ETIMEOUT.
    The next call, with the default bound, clears the word and matches the
    oracle: the GPU context stays usable."""
    dims, N, rep, phase = CASES[0]
    olat, blat = lats(dims, N, rep, phase)
    U = fields.gauge_field(dims, N, "haar", seed=71)
    R = orc.links_to_rep(olat, U)
    U32 = gpu_links(blat, U, bsm.F32)
    rng = np.random.default_rng(72)
    C, nb = 12, 2
    W1, W2 = rand_c(rng, (36, 4 * C), 0.3), rand_c(rng, (36 * C, 4), 0.1)
    psis = [fields.gaussian_spinor(dims, olat.d, 73 + b) for b in range(nb)]
    F = ptc_field(blat, psis)
    out = torch.zeros_like(F)
    ws = torch.empty(bsm.bsm_ptc_workspace_bytes(blat, C, nb, 0), dtype=torch.uint8, device="cuda")
    W1d, W2d = dev_c64(W1), dev_c64(W2)
    monkeypatch.setenv("BSM_PTC_WAIT_POLLS", "0")
    bsm.bsm_ptc_apply(blat, U32, W1d, W2d, C, F, out, nb, bsm.BF16, ws)
    assert bsm.bsm_ptc_status(ws) == bsm.ETIMEOUT
    assert not bool(torch.isfinite(out).all())
    monkeypatch.delenv("BSM_PTC_WAIT_POLLS")
    bsm.bsm_ptc_apply(blat, U32, W1d, W2d, C, F, out, nb, bsm.BF16, ws)
    assert bsm.bsm_ptc_status(ws) == bsm.OK
    got = from_ptc_field(blat, out, nb)
    for b in range(nb):
        assert rel(got[b], oracle_net(olat, R, psis[b], W1, W2, C)) < 2e-2


@pytest.mark.parametrize("eo", [True, False], ids=["eo", "full"])
def test_fgcr_falls_back_when_the_network_wait_gives_up(monkeypatch, eo):
    """An FGCR solve whose BF16 network had a tensor-core wait give up
    (BSM_PTC_WAIT_POLLS=0) ends with BSM_ETIMEOUT; with opts.fallback the
    plain CG solver finishes it and x solves D x = b (the oracle's D)."""
    dims, N = (4, 4, 4, 8), 3
    olat, blat = lats(dims, N, bsm.FUND, (np.pi, 0, 0, 0), m0=0.05)
    U = fields.gauge_field(dims, N, "smooth", seed=74, eps=0.4)
    R = orc.links_to_rep(olat, U)
    U64, U32 = gpu_links(blat, U, bsm.F64), gpu_links(blat, U, bsm.F32)
    b = fields.gaussian_spinor(dims, N, 75)
    bd = gpu_spinor(blat, b, bsm.F64)
    W1, W2 = neumann_weights(olat.m0)
    W = (dev_c64(W1), dev_c64(W2))
    kw = dict(tol=1e-11, restart=16, precond=bsm.FGCR_PTC, ptc_prec=bsm.BF16, channels=2, eo=eo,
              prec_inner=bsm.F32, inner_tol=1e-3, max_iter=1000)
    monkeypatch.setenv("BSM_PTC_WAIT_POLLS", "0")
    st, _, _ = fgcr(blat, U64, U32, bd, bsm.fgcr_opts(**kw), W)
    assert st == bsm.ETIMEOUT
    st, stats, x = fgcr(blat, U64, U32, bd, bsm.fgcr_opts(fallback=True, **kw), W)
    monkeypatch.delenv("BSM_PTC_WAIT_POLLS")
    assert st == bsm.OK, bsm.bsm_strerror(st)
    assert stats.fgcr_status == bsm.ETIMEOUT and stats.fallback_iters > 0
    assert stats.true_res <= 1e-9
    assert rel(orc.dirac(olat, R, to_canon(blat, x, bsm.F64)), b) <= 1e-9
    st, stats, _ = fgcr(blat, U64, U32, bd, bsm.fgcr_opts(**kw), W)
    assert st == bsm.OK and stats.fgcr_status == bsm.OK


@pytest.mark.parametrize("precond", ["none", "ptc-bf16"])
def test_mixed_precision_fgcr_reaches_fp64_accuracy(precond):
    """FP32 restart cycles with the residual recomputed in FP64: the same
    1e-10 true residual and solution as all-FP64 FGCR."""
    dims, N = (4, 4, 4, 8), 3
    olat, blat = lats(dims, N, bsm.FUND, (np.pi, 0, 0, 0), m0=0.05)
    U = fields.gauge_field(dims, N, "smooth", seed=24, eps=0.4)
    R = orc.links_to_rep(olat, U)
    U64, U32 = gpu_links(blat, U, bsm.F64), gpu_links(blat, U, bsm.F32)
    b = fields.gaussian_spinor(dims, N, 25)
    bd = gpu_spinor(blat, b, bsm.F64)
    kw = {} if precond == "none" else dict(precond=bsm.FGCR_PTC, ptc_prec=bsm.BF16, channels=2)
    W = (None, None) if precond == "none" else tuple(dev_c64(w) for w in neumann_weights(olat.m0))
    st0, s0, x0 = fgcr(blat, U64, U32, bd, bsm.fgcr_opts(tol=1e-10, restart=16, **kw), W)
    st1, s1, x1 = fgcr(blat, U64, U32, bd, bsm.fgcr_opts(tol=1e-10, restart=16, prec_inner=bsm.F32, inner_tol=1e-3,
                                                        **kw), W)
    assert st0 == bsm.OK and st1 == bsm.OK, (st0, st1)
    assert s1.true_res <= 1e-10 and s1.cycles >= 2
    x = to_canon(blat, x1, bsm.F64)
    assert rel(orc.dirac(olat, R, x), b) <= 1e-10
    assert rel(x, to_canon(blat, x0, bsm.F64)) < 1e-8
    assert s1.iters <= 2 * s0.iters + 16


@pytest.mark.parametrize("eo", [True, False], ids=["eo", "full"])
@pytest.mark.parametrize("precond", ["none", "ptc-bf16"])
def test_double_float_outer_operator(precond, eo):
    """FP32 cycles with the FP64-accurate operator (right-hand side, residual
    after each cycle, odd sites, true residual) in double-float on DF64
    links: the same steps and solution as with the FP64 operator, and a full
    residual <= 1e-10 checked with the oracle's D."""
    dims, N = (4, 4, 4, 8), 3
    olat, blat = lats(dims, N, bsm.FUND, (np.pi, 0, 0, 0), m0=0.05)
    U = fields.gauge_field(dims, N, "smooth", seed=24, eps=0.4)
    U64, U32, Udf = gpu_links(blat, U, bsm.F64), gpu_links(blat, U, bsm.F32), gpu_links(blat, U, bsm.DF64)
    b = fields.gaussian_spinor(dims, N, 25)
    bd = gpu_spinor(blat, b, bsm.F64)
    kw = dict(tol=1e-10, restart=16, prec_inner=bsm.F32, inner_tol=1e-3, eo=eo, check_every=2)
    W = (None, None)
    if precond != "none":
        kw.update(precond=bsm.FGCR_PTC, ptc_prec=bsm.BF16, channels=2)
        W = tuple(dev_c64(w) for w in neumann_weights(olat.m0))
    st0, s0, x0 = fgcr(blat, U64, U32, bd, bsm.fgcr_opts(**kw), W)
    st1, s1, x1 = fgcr(blat, Udf, U32, bd, bsm.fgcr_opts(prec_outer=bsm.DF64, **kw), W)
    assert st0 == bsm.OK and st1 == bsm.OK, (st0, st1)
    assert abs(s1.iters - s0.iters) <= 2 and s1.true_res <= 1e-10
    x = to_canon(blat, x1, bsm.F64)
    assert rel(orc.dirac(olat, orc.links_to_rep(olat, U), x), b) <= 1e-10
    assert rel(x, to_canon(blat, x0, bsm.F64)) < 1e-8


@pytest.mark.parametrize("prec_inner", [bsm.F64, bsm.F32], ids=["fp64", "fp32cycles"])
@pytest.mark.parametrize("precond", ["none", "ptc-f32", "ptc-bf16"])
def test_even_odd_fgcr_solves_the_full_system(precond, prec_inner):
    """FGCR on the Schur system Dhat x_e = bhat_e (preconditioned by the
    even-even block of the network) with x_o reconstructed: the full system's
    solution to 1e-10, checked with the oracle's D and against its dense solve."""
    dims, N = (4, 4, 4, 4), 2
    olat, blat = lats(dims, N, bsm.FUND, (np.pi, 0, 0, 0), m0=0.05)
    U = fields.gauge_field(dims, N, "smooth", seed=30, eps=0.4)
    R = orc.links_to_rep(olat, U)
    U64, U32 = gpu_links(blat, U, bsm.F64), gpu_links(blat, U, bsm.F32)
    b = fields.gaussian_spinor(dims, N, 31)
    kw = {}
    W = (None, None)
    if precond != "none":
        kw = dict(precond=bsm.FGCR_PTC, ptc_prec=bsm.F32 if precond == "ptc-f32" else bsm.BF16, channels=2)
        W = tuple(dev_c64(w) for w in neumann_weights(olat.m0))
    st, s_eo, x = fgcr(blat, U64, U32, gpu_spinor(blat, b, bsm.F64),
                       bsm.fgcr_opts(tol=1e-10, restart=12, eo=True, prec_inner=prec_inner, inner_tol=1e-3, **kw), W)
    assert st == bsm.OK
    assert s_eo.true_res <= 1.5e-10
    xg = to_canon(blat, x, bsm.F64)
    assert rel(orc.dirac(olat, R, xg), b) <= 1.5e-10
    x_ref = np.linalg.solve(orc.dense_dirac(olat, R), b.reshape(-1)).reshape(b.shape)
    assert rel(xg, x_ref) < 1e-8
    # fewer iterations than the same solver on the full operator
    st, s_full, _ = fgcr(blat, U64, U32, gpu_spinor(blat, b, bsm.F64),
                         bsm.fgcr_opts(tol=1e-10, restart=12, prec_inner=prec_inner, inner_tol=1e-3, **kw), W)
    assert st == bsm.OK and s_eo.iters < s_full.iters, (s_eo.iters, s_full.iters)


def test_fgcr_check_every_bounds_the_overshoot():
    dims, N = (4, 4, 4, 4), 2
    olat, blat = lats(dims, N, bsm.FUND, (np.pi, 0, 0, 0), m0=0.05)
    U = fields.gauge_field(dims, N, "smooth", seed=32, eps=0.4)
    R = orc.links_to_rep(olat, U)
    U64, U32 = gpu_links(blat, U, bsm.F64), gpu_links(blat, U, bsm.F32)
    b = fields.gaussian_spinor(dims, N, 33)
    bd = gpu_spinor(blat, b, bsm.F64)
    st1, s1, _ = fgcr(blat, U64, U32, bd, bsm.fgcr_opts(tol=1e-10, restart=12, eo=True))
    st4, s4, x4 = fgcr(blat, U64, U32, bd, bsm.fgcr_opts(tol=1e-10, restart=12, eo=True, check_every=4))
    assert st1 == bsm.OK and st4 == bsm.OK
    assert s1.iters <= s4.iters <= s1.iters + 3 + s4.cycles
    assert rel(orc.dirac(olat, R, to_canon(blat, x4, bsm.F64)), b) <= 1e-10


@pytest.mark.parametrize("dims", [(8, 4, 4, 6), (18, 14, 14, 14)], ids=["6-tiles", "386-tiles"])
def test_even_only_network_application_matches_the_full_one(dims):
    """In even-odd FGCR the BF16 fused path applies only the even-even block
    of the network (even sites skip their neighbours' transports, the
    stencil skips odd outputs); the FP32 path applies the whole network and
    keeps the even part.  The same preconditioner up to BF16 rounding: the
    two solves take the same number of steps within 2.  The larger lattice
    (parity blocks of 24696 sites: 193 tiles, the last ragged) gives each
    block of the persistent fused kernel several tiles."""
    N = 3
    olat, blat = lats(dims, N, bsm.FUND, (np.pi, 0, 0, 0), m0=0.05)
    U = fields.gauge_field(dims, N, "smooth", seed=34, eps=0.4)
    U64, U32 = gpu_links(blat, U, bsm.F64), gpu_links(blat, U, bsm.F32)
    b = gpu_spinor(blat, fields.gaussian_spinor(dims, N, 35), bsm.F64)
    W = tuple(dev_c64(w) for w in neumann_weights(olat.m0))
    its = {}
    for prec in (bsm.F32, bsm.BF16):
        st, s, _ = fgcr(blat, U64, U32, b, bsm.fgcr_opts(tol=1e-10, restart=16, eo=True, precond=bsm.FGCR_PTC,
                                                          channels=2, ptc_prec=prec), W)
        assert st == bsm.OK and s.true_res <= 1.5e-10
        its[prec] = s.iters
    assert abs(its[bsm.F32] - its[bsm.BF16]) <= 2, its


def test_full_size_16c32_fgcr_with_the_network():
    """The learned-preconditioner workload at full size (16^3 x 32 SU(3),
    smooth links eps 0.5, m0 = -0.62, antiperiodic time), solved as the
    benchmark's best configuration runs (even-odd FGCR(32), BF16 network on
    the tensor cores, FP32 cycles, double-float outer operator) with the
    degree-2 Neumann weights standing in for trained ones: the oracle's D
    applied to the GPU solution gives back b."""
    dims, N, m0 = (32, 16, 16, 16), 3, -0.62
    olat, blat = lats(dims, N, bsm.FUND, (np.pi, 0, 0, 0), m0=m0)
    U = fields.gauge_field(dims, N, "smooth", seed=3, eps=0.5)
    R = orc.links_to_rep(olat, U)
    Udf, U32 = gpu_links(blat, U, bsm.DF64), gpu_links(blat, U, bsm.F32)
    b = fields.gaussian_spinor(dims, N, 4)
    bd = gpu_spinor(blat, b, bsm.F64)
    W1, W2 = neumann_weights(m0)
    opts = bsm.fgcr_opts(tol=1e-10, restart=32, precond=bsm.FGCR_PTC, ptc_prec=bsm.BF16, channels=2, eo=True,
                         prec_inner=bsm.F32, prec_outer=bsm.DF64, inner_tol=1e-3, max_iter=20000)
    st, stats, x = fgcr(blat, Udf, U32, bd, opts, (dev_c64(W1), dev_c64(W2)))
    assert st == bsm.OK, bsm.bsm_strerror(st)
    assert stats.true_res <= 1e-10
    assert rel(orc.dirac(olat, R, to_canon(blat, x, bsm.F64)), b) <= 2e-10
