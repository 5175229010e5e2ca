"""GPU parity of the representation links, the hopping block, the full Wilson
operator and the even-odd Schur operator against the FP64 oracle, element by
element on the same seeded inputs, through the C ABI.  Bars: relative L2
<= 1e-13 in FP64 and <= 2e-6 in FP32.  Also physics invariants evaluated on
the GPU output itself (closed-form free field, gamma5-hermiticity, gauge
covariance), so that a convention shared by both sides cannot hide."""
import numpy as np
import pytest
import torch

import oracle as orc
from paper_1401_3733_gb300 import bsm, fields
from tests.gpu_helpers import (REP_CASES, REP_IDS, TOL, gpu_links, gpu_spinor, half, rel, to_canon,
                               zeros_field)

pytestmark = pytest.mark.gpu

PRECS = [bsm.F64, bsm.F32, bsm.DF64, bsm.BF16]
PREC_IDS = ["f64", "f32", "df64", "bf16"]


def setup(dims, N, rep, m0, phase, seed, kind="haar", eps=0.3):
    olat = orc.Lattice(dims, N, rep, m0, phase)
    blat = bsm.lattice(dims, N, rep, m0, phase)
    U = fields.gauge_field(dims, N, kind, seed=seed, eps=eps)
    R = orc.links_to_rep(olat, U)
    psi = fields.gaussian_spinor(dims, olat.d, seed + 1000)
    return olat, blat, U, R, psi


def gpu_hop_parity(blat, U, psi, p, dagger, prec):
    Ud = gpu_links(blat, U, prec)
    inp = gpu_spinor(blat, psi, prec)
    out = zeros_field(blat, bsm.FIELD_SPINOR, prec)
    bsm.bsm_dslash(blat, Ud, half(blat, inp, 1 - p, prec), half(blat, out, p, prec), p, dagger, prec)
    return to_canon(blat, out, prec)


@pytest.mark.parametrize("prec", PRECS, ids=PREC_IDS)
def test_pack_unpack_roundtrip(prec):
    dims = (4, 2, 6, 4)
    lat = bsm.lattice(dims, 3)
    psi = fields.gaussian_spinor(dims, 3, 5)
    back = to_canon(lat, gpu_spinor(lat, psi, prec), prec)
    if prec in (bsm.DF64, bsm.BF16):
        # DF64: hi + lo carries 48 significand bits, |error| <= 2^-48 |x|;
        # BF16: 8 significand bits, |error| <= 2^-8 |x| (round to nearest)
        err = np.maximum(np.abs(back.real - psi.real) / np.abs(psi.real),
                         np.abs(back.imag - psi.imag) / np.abs(psi.imag))
        assert err.max() <= (2.0 ** -48 if prec == bsm.DF64 else 2.0 ** -8)
        return
    want = psi if prec == bsm.F64 else psi.astype(np.complex64).astype(np.complex128)
    assert np.array_equal(back, want)


@pytest.mark.parametrize("prec", PRECS, ids=PREC_IDS)
@pytest.mark.parametrize("N,rep", REP_CASES, ids=REP_IDS)
def test_hop_parity_blocks_all_reps(N, rep, prec):
    dims = (4, 4, 4, 4)
    phase = (np.pi, 0, 0, 0) if rep == bsm.ADJ else (np.pi, 0.4, -1.3, 0.0)
    olat, blat, U, R, psi = setup(dims, N, rep, 0.1, phase, seed=100 + 7 * N + rep)
    for p in (0, 1):
        for dagger in (False, True):
            got = gpu_hop_parity(blat, U, psi, p, dagger, prec)
            want = orc.hop(olat, R, psi, out_parity=p, dagger=dagger)
            assert rel(got, want) <= TOL[prec], (p, dagger, rel(got, want))


@pytest.mark.parametrize("prec", PRECS, ids=PREC_IDS)
@pytest.mark.parametrize("dims", [(2, 2, 2, 2), (2, 2, 2, 6), (6, 4, 2, 10), (4, 6, 8, 2), (8, 4, 4, 6)],
                         ids=["2^4", "ragged24", "ragged240", "nonc-z2", "8x4x4x6"])
def test_full_dirac_shapes(dims, prec):
    """Full D and D^+ on small, non-cubic and ragged lattices (V_h not a
    multiple of the block size; Z = 2 and L = 2, where both neighbours of a
    site coincide)."""
    olat, blat, U, R, psi = setup(dims, 3, bsm.FUND, 0.05, (np.pi, 0.3, 0, 1.1), seed=200)
    Ud = gpu_links(blat, U, prec)
    inp = gpu_spinor(blat, psi, prec)
    out = zeros_field(blat, bsm.FIELD_SPINOR, prec)
    for dagger in (False, True):
        bsm.bsm_dslash(blat, Ud, inp, out, bsm.FULL, dagger, prec)
        got = to_canon(blat, out, prec)
        want = orc.dirac(olat, R, psi, dagger=dagger)
        assert rel(got, want) <= TOL[prec], (dagger, rel(got, want))


@pytest.mark.parametrize("prec", PRECS, ids=PREC_IDS)
@pytest.mark.parametrize("N,rep", [(2, bsm.FUND), (3, bsm.FUND), (2, bsm.ADJ), (4, bsm.ASYM), (3, bsm.SYM)],
                         ids=["SU2-F", "SU3-F", "SU2-ADJ", "SU4-AS", "SU3-S"])
def test_dirac_eo_ops(N, rep, prec):
    dims = (4, 4, 2, 6)
    olat, blat, U, R, psi = setup(dims, N, rep, 0.1, (np.pi, 0, 0, 0), seed=300 + N)
    odd = orc.parity_mask(dims)
    psi[odd] = 0
    Ud = gpu_links(blat, U, prec)
    inp = gpu_spinor(blat, psi, prec)
    ws = torch.empty(bsm.bsm_workspace_bytes(blat, bsm.CALL_DIRAC_EO, prec), dtype=torch.uint8, device="cuda")
    for op in (bsm.OP_DHAT, bsm.OP_DHAT_DAG, bsm.OP_DHAT_DAG_DHAT):
        out = zeros_field(blat, bsm.FIELD_SPINOR, prec)
        bsm.bsm_dirac_eo(blat, Ud, half(blat, inp, 0, prec), half(blat, out, 0, prec), op, prec, ws)
        got = to_canon(blat, out, prec)
        want = orc.dhat(olat, R, psi, op)
        assert rel(got, want) <= TOL[prec], (op, rel(got, want))


# ----------------------------------------------------------------------------
# SU(3) links stored as two rows (BSM_F32R12)
# ----------------------------------------------------------------------------

@pytest.mark.parametrize("phase", [(np.pi, 0.4, -1.3, 0.0), (0.0, 0.0, 0.0, 0.0), (2.1, 0.0, 0.7, -0.2)],
                         ids=["antiperiodic+twists", "periodic", "generic"])
@pytest.mark.parametrize("dims", [(4, 4, 4, 4), (6, 4, 2, 10), (2, 2, 2, 6)], ids=["4^4", "ragged240", "L2"])
def test_two_row_links_hop_matches_oracle(dims, phase):
    """Hop (both parities, dagger), full D and D^+ from two-row links: the
    third row and the boundary factor c^3 rebuilt in the kernel.  Haar links
    (far from the identity), boundary phases that cross every direction."""
    olat, blat, U, R, psi = setup(dims, 3, bsm.FUND, 0.1, phase, seed=500)
    prec = bsm.F32R12
    for p in (0, 1):
        for dagger in (False, True):
            got = gpu_hop_parity(blat, U, psi, p, dagger, prec)
            want = orc.hop(olat, R, psi, out_parity=p, dagger=dagger)
            assert rel(got, want) <= TOL[prec], (p, dagger, rel(got, want))
    Ud = gpu_links(blat, U, prec)
    inp = gpu_spinor(blat, psi, prec)
    out = zeros_field(blat, bsm.FIELD_SPINOR, prec)
    for dagger in (False, True):
        bsm.bsm_dslash(blat, Ud, inp, out, bsm.FULL, dagger, prec)
        assert rel(to_canon(blat, out, prec), orc.dirac(olat, R, psi, dagger=dagger)) <= TOL[prec]


def test_two_row_links_dirac_eo_and_sizes():
    dims = (4, 4, 2, 6)
    olat, blat, U, R, psi = setup(dims, 3, bsm.FUND, 0.1, (np.pi, 0, 0, 0), seed=510)
    prec = bsm.F32R12
    psi[orc.parity_mask(dims)] = 0
    Ud = gpu_links(blat, U, prec)
    # 2 parities x padded V_h x 8 links x 12 floats
    assert Ud.numel() == 2 * 96 * 8 * 12 * 4
    assert bsm.bsm_field_bytes(blat, bsm.FIELD_SPINOR, prec) == bsm.bsm_field_bytes(blat, bsm.FIELD_SPINOR, bsm.F32)
    inp = gpu_spinor(blat, psi, prec)
    ws = torch.empty(bsm.bsm_workspace_bytes(blat, bsm.CALL_DIRAC_EO, prec), dtype=torch.uint8, device="cuda")
    for op in (bsm.OP_DHAT, bsm.OP_DHAT_DAG, bsm.OP_DHAT_DAG_DHAT):
        out = zeros_field(blat, bsm.FIELD_SPINOR, prec)
        bsm.bsm_dirac_eo(blat, Ud, half(blat, inp, 0, prec), half(blat, out, 0, prec), op, prec, ws)
        got = to_canon(blat, out, prec)
        want = orc.dhat(olat, R, psi, op)
        assert rel(got, want) <= TOL[prec], (op, rel(got, want))


# ----------------------------------------------------------------------------
# invariants on the GPU output itself
# ----------------------------------------------------------------------------

def free_symbol(m0, p):
    D = (m0 + np.sum(1 - np.cos(p))) * np.eye(4, dtype=np.complex128)
    for mu in range(4):
        D = D + 1j * np.sin(p[mu]) * orc.gamma(mu)
    return D


@pytest.mark.parametrize("prec", PRECS, ids=PREC_IDS)
def test_gpu_free_field_plane_wave(prec):
    dims, phase, m0 = (8, 4, 6, 4), (np.pi, 0.5, 0, -0.8), 0.07
    blat = bsm.lattice(dims, 3, bsm.FUND, m0, phase)
    Ud = gpu_links(blat, fields.gauge_field(dims, 3, "unit"), prec)
    xs = fields.site_coords(dims)
    rng = np.random.default_rng(11)
    for _ in range(3):
        n = np.array([rng.integers(0, L) for L in dims])
        p = (2 * np.pi * n + np.array(phase)) / np.array(dims)
        chi = rng.standard_normal((4, 3)) + 1j * rng.standard_normal((4, 3))
        wave = np.exp(1j * xs @ p)
        out = zeros_field(blat, bsm.FIELD_SPINOR, prec)
        bsm.bsm_dslash(blat, Ud, gpu_spinor(blat, wave[:, None, None] * chi[None], prec), out, bsm.FULL, 0, prec)
        want = wave[:, None, None] * (free_symbol(m0, p) @ chi)[None]
        assert rel(to_canon(blat, out, prec), want) <= TOL[prec]


@pytest.mark.parametrize("N,rep", [(3, bsm.FUND), (2, bsm.ADJ), (4, bsm.ASYM)], ids=["SU3-F", "SU2-ADJ", "SU4-AS"])
def test_gpu_gamma5_hermiticity_and_gauge_covariance(N, rep):
    prec = bsm.F64
    dims = (4, 4, 2, 4)
    olat, blat, U, R, psi = setup(dims, N, rep, 0.1, (np.pi, 0, 0, 0), seed=400)
    phi = fields.gaussian_spinor(dims, olat.d, 401)
    Ud = gpu_links(blat, U, prec)

    def D(links, f, dagger=False):
        out = zeros_field(blat, bsm.FIELD_SPINOR, prec)
        bsm.bsm_dslash(blat, links, gpu_spinor(blat, f, prec), out, bsm.FULL, dagger, prec)
        return to_canon(blat, out, prec)

    G5 = lambda f: np.einsum("ab,sbc->sac", np.diag([-1.0, -1.0, 1.0, 1.0]), f)
    lhs = np.vdot(phi.reshape(-1), G5(D(Ud, G5(psi))).reshape(-1))
    rhs = np.vdot(D(Ud, phi).reshape(-1), psi.reshape(-1))
    assert abs(lhs - rhs) / abs(rhs) < 1e-13
    assert rel(D(Ud, psi, dagger=True), G5(D(Ud, G5(psi)))) < 1e-13

    g = fields.gauge_transform(dims, N, 402)
    xs = fields.site_coords(dims)
    T, X, Y, Z = dims
    Ug = np.empty_like(U)
    for mu in range(4):
        c = xs.copy()
        c[:, mu] = (c[:, mu] + 1) % dims[mu]
        fwd = ((c[:, 0] * X + c[:, 1]) * Y + c[:, 2]) * Z + c[:, 3]
        Ug[:, mu] = g @ U[:, mu] @ np.conj(np.transpose(g[fwd], (0, 2, 1)))
    Rg = orc.links_to_rep(olat, np.repeat(g[:, None], 4, axis=1))[:, 0]
    rot = lambda f: np.einsum("sab,sib->sia", Rg, f)
    assert rel(D(gpu_links(blat, Ug, prec), rot(psi)), rot(D(Ud, psi))) < 1e-13


# ----------------------------------------------------------------------------
# the 32^3 x 64 SU(3) workload at full size, in the benchmark's launch shape
# ----------------------------------------------------------------------------

@pytest.fixture(scope="module")
def big_case():
    dims = (64, 32, 32, 32)
    olat, blat, U, R, psi = setup(dims, 3, bsm.FUND, 0.05, (np.pi, 0, 0, 0), seed=3, kind="smooth", eps=0.3)
    return olat, blat, U, R, psi


@pytest.mark.parametrize("prec", PRECS + [bsm.F32R12], ids=PREC_IDS + ["f32r12"])
def test_full_size_32c64_hop(big_case, prec):
    """Both parity blocks of the hop on the whole 32^3 x 64 lattice, every
    output element compared with the oracle."""
    olat, blat, U, R, psi = big_case
    Ud = gpu_links(blat, U, prec)
    inp = gpu_spinor(blat, psi, prec)
    out = zeros_field(blat, bsm.FIELD_SPINOR, prec)
    bsm.bsm_dslash(blat, Ud, half(blat, inp, 1, prec), half(blat, out, 0, prec), bsm.EVEN, 0, prec)
    bsm.bsm_dslash(blat, Ud, half(blat, inp, 0, prec), half(blat, out, 1, prec), bsm.ODD, 0, prec)
    got = to_canon(blat, out, prec)
    want = orc.hop(olat, R, psi, out_parity=orc.FULL)
    assert rel(got, want) <= TOL[prec]


def test_full_size_48c96_hop_f32_and_two_row():
    """The 48^3 x 96 workload of the benchmark's `large` lines (links drawn on
    the device with the same generator), both parity blocks, every output
    element against the oracle, full-link and two-row FP32 links."""
    dims, N = (96, 48, 48, 48), 3
    phase = (np.pi, 0, 0, 0)
    olat = orc.Lattice(dims, N, orc.FUND, 0.05, phase)
    blat = bsm.lattice(dims, N, bsm.FUND, 0.05, phase)
    Ud = fields.device_smooth_gauge_field(dims, N, 5, 0.3)
    psid = fields.device_gaussian_spinors(dims, N, 1, 6)[0]
    want = orc.hop(olat, orc.links_to_rep(olat, Ud.cpu().numpy()), psid.cpu().numpy(), out_parity=orc.FULL)
    for prec in (bsm.F32, bsm.F32R12):
        links = bsm.empty_field(blat, bsm.FIELD_LINKS, prec)
        bsm.bsm_links_to_rep(blat, Ud, links, prec)
        inp = bsm.empty_field(blat, bsm.FIELD_SPINOR, prec)
        bsm.bsm_pack_spinor(blat, psid, inp, prec)
        out = zeros_field(blat, bsm.FIELD_SPINOR, prec)
        bsm.bsm_dslash(blat, links, half(blat, inp, 1, prec), half(blat, out, 0, prec), bsm.EVEN, 0, prec)
        bsm.bsm_dslash(blat, links, half(blat, inp, 0, prec), half(blat, out, 1, prec), bsm.ODD, 0, prec)
        assert rel(to_canon(blat, out, prec), want) <= TOL[prec], prec
        del links, inp, out
