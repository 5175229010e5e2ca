"""Multi-RHS hopping block (bsm_dslash_mrhs): every right-hand side of a
batch equals the oracle's operator applied to that RHS alone, for every
representation, both parity blocks and the full operator, the adjoint, FP32
and BF16 storage, and batch sizes that exercise every compiled RHS block
(including an odd count and a ragged lattice)."""
import numpy as np
import pytest
import torch

import oracle as orc
from paper_1401_3733_gb300 import bsm, fields
from tests.gpu_helpers import REP_CASES, REP_IDS, TOL, dev_c128, gpu_links, rel

pytestmark = pytest.mark.gpu


def mrhs_field(lat, nrhs, prec):
    n = bsm.bsm_field_bytes(lat, bsm.FIELD_SPINOR, prec) * nrhs
    return torch.zeros(n, dtype=torch.uint8, device="cuda")


def pack(lat, psis, prec):
    out = mrhs_field(lat, len(psis), prec)
    bsm.bsm_pack_spinor_mrhs(lat, dev_c128(np.stack(psis)), out, len(psis), prec)
    return out


def unpack(lat, dev, nrhs, prec):
    V = int(np.prod(list(lat.dims)))
    d = bsm.bsm_rep_dim(lat.N, lat.rep)
    c = torch.empty((nrhs, V, 4, d), dtype=torch.complex128, device="cuda")
    bsm.bsm_unpack_spinor_mrhs(lat, dev, c, nrhs, prec)
    torch.cuda.synchronize()
    return c.cpu().numpy()


def setup(dims, N, rep, nrhs, seed):
    phase = (np.pi, 0, 0, 0) if rep == bsm.ADJ else (np.pi, 0.3, 0, -0.7)
    olat = orc.Lattice(dims, N, rep, 0.1, phase)
    blat = bsm.lattice(dims, N, rep, 0.1, phase)
    U = fields.gauge_field(dims, N, "haar", seed=seed)
    R = orc.links_to_rep(olat, U)
    psis = [fields.gaussian_spinor(dims, olat.d, seed + 10 + r) for r in range(nrhs)]
    return olat, blat, U, R, psis


@pytest.mark.parametrize("prec", [bsm.F32, bsm.BF16], ids=["f32", "bf16"])
def test_mrhs_pack_roundtrip(prec):
    dims = (4, 2, 2, 6)
    lat = bsm.lattice(dims, 3)
    psis = [fields.gaussian_spinor(dims, 3, 40 + r) for r in range(5)]
    back = unpack(lat, pack(lat, psis, prec), 5, prec)
    want = np.stack(psis)
    bound = 2.0 ** -24 if prec == bsm.F32 else 2.0 ** -8
    for part in (np.real, np.imag):
        assert (np.abs(part(back) - part(want)) <= bound * np.abs(part(want))).all()


def test_mrhs_layout_is_site_major():
    """The documented multi-RHS layout, read back byte for byte: FP32 element
    (plane q = s d + c, eo site i, RHS r) of parity p sits at
    (p V_h + i) 2d n_rhs + q n_rhs + r as the float4 (psi[s][c], psi[s+2][c])
    of RHS r, with eo site i = canonical index >> 1 (z fastest)."""
    dims = (4, 2, 2, 6)
    d, nrhs = 3, 5
    lat = bsm.lattice(dims, 3)
    psis = np.stack([fields.gaussian_spinor(dims, d, 70 + r) for r in range(nrhs)])  # [r][V][4][d]
    dev = pack(lat, list(psis), bsm.F32)
    torch.cuda.synchronize()
    V = int(np.prod(dims))
    got = dev.cpu().numpy().view(np.float32).reshape(2, V // 2, 2 * d, nrhs, 4)
    t, x, y, z = np.unravel_index(np.arange(V), dims)
    par, i = (t + x + y + z) & 1, np.arange(V) >> 1
    want = np.full_like(got, np.nan)
    for r in range(nrhs):
        for s in range(2):
            for c in range(d):
                up, lo = psis[r, :, s, c], psis[r, :, s + 2, c]
                for k, v in enumerate((up.real, up.imag, lo.real, lo.imag)):
                    want[par, i, s * d + c, r, k] = v.astype(np.float32)
    assert np.array_equal(got, want)


@pytest.mark.parametrize("prec", [bsm.F32, bsm.BF16], ids=["f32", "bf16"])
@pytest.mark.parametrize("N,rep", REP_CASES, ids=REP_IDS)
def test_mrhs_all_reps(N, rep, prec):
    dims, nrhs = (4, 4, 4, 4), 4
    olat, blat, U, R, psis = setup(dims, N, rep, nrhs, 500 + 3 * N + rep)
    Ud = gpu_links(blat, U, prec)
    inp = pack(blat, psis, prec)
    for out_parity in (bsm.EVEN, bsm.ODD, bsm.FULL):
        for dagger in (False, True):
            out = mrhs_field(blat, nrhs, prec)
            half = bsm.bsm_field_bytes(blat, bsm.FIELD_HALF_SPINOR, prec) * nrhs
            if out_parity == bsm.FULL:
                bsm.bsm_dslash_mrhs(blat, Ud, inp, out, nrhs, bsm.FULL, dagger, prec)
            else:
                p = out_parity
                bsm.bsm_dslash_mrhs(blat, Ud, inp[(1 - p) * half:(2 - p) * half], out[p * half:(p + 1) * half],
                                    nrhs, p, dagger, prec)
            got = unpack(blat, out, nrhs, prec)
            for r in range(nrhs):
                if out_parity == bsm.FULL:
                    want = orc.dirac(olat, R, psis[r], dagger=dagger)
                else:
                    want = orc.hop(olat, R, psis[r], out_parity=out_parity, dagger=dagger)
                assert rel(got[r], want) <= TOL[prec], (out_parity, dagger, r, rel(got[r], want))


@pytest.mark.parametrize("nrhs", [1, 3, 5, 12])
@pytest.mark.parametrize("N,rep", [(3, bsm.FUND), (4, bsm.ASYM), (2, bsm.ADJ)], ids=["SU3-F", "SU4-AS", "SU2-ADJ"])
def test_mrhs_batch_sizes_ragged(N, rep, nrhs):
    """RHS counts that select every compiled RHS block (1..4 for d <= 3, 1..2
    for d = 6) on a lattice whose V_h (120) fills no whole thread block."""
    dims = (2, 6, 4, 10)
    olat, blat, U, R, psis = setup(dims, N, rep, nrhs, 600 + nrhs)
    Ud = gpu_links(blat, U, bsm.F32)
    out = mrhs_field(blat, nrhs, bsm.F32)
    bsm.bsm_dslash_mrhs(blat, Ud, pack(blat, psis, bsm.F32), out, nrhs, bsm.FULL, 0, bsm.F32)
    got = unpack(blat, out, nrhs, bsm.F32)
    for r in range(nrhs):
        assert rel(got[r], orc.dirac(olat, R, psis[r])) <= TOL[bsm.F32]


def test_mrhs_matches_single_rhs_calls():
    """The batch result equals bsm_dslash applied to each RHS (same
    arithmetic per RHS, so equal to rounding-order differences only)."""
    dims, nrhs, prec = (8, 4, 4, 8), 6, bsm.F32
    olat, blat, U, R, psis = setup(dims, 3, bsm.FUND, nrhs, 700)
    Ud = gpu_links(blat, U, prec)
    out = mrhs_field(blat, nrhs, prec)
    bsm.bsm_dslash_mrhs(blat, Ud, pack(blat, psis, prec), out, nrhs, bsm.FULL, 0, prec)
    got = unpack(blat, out, nrhs, prec)
    for r in range(nrhs):
        one = bsm.empty_field(blat, bsm.FIELD_SPINOR, prec)
        res = bsm.empty_field(blat, bsm.FIELD_SPINOR, prec)
        bsm.bsm_pack_spinor(blat, dev_c128(psis[r]), one, prec)
        bsm.bsm_dslash(blat, Ud, one, res, bsm.FULL, 0, prec)
        c = torch.empty_like(dev_c128(psis[r]))
        bsm.bsm_unpack_spinor(blat, res, c, prec)
        assert rel(got[r], c.cpu().numpy()) < 1e-6


@pytest.mark.parametrize("nrhs", [4, 8, 12, 16])
@pytest.mark.parametrize("N,rep", [(4, bsm.FUND), (6, bsm.FUND), (4, bsm.ASYM), (3, bsm.SYM), (8, bsm.FUND)],
                         ids=["SU4-F", "SU6-F", "SU4-AS", "SU3-S", "SU8-F"])
def test_mrhs_tensor_core_path(N, rep, nrhs):
    """The tensor-core kernel (BF16 mma.sync block products, FP32
    accumulation), pinned, against the oracle per RHS and against the SIMT
    kernel on the same BF16 inputs, for the full operator and the adjoint
    parity blocks."""
    dims, prec = (4, 4, 2, 6), bsm.BF16
    olat, blat, U, R, psis = setup(dims, N, rep, nrhs, 800 + N + nrhs)
    Ud = gpu_links(blat, U, prec)
    inp = pack(blat, psis, prec)
    half = bsm.bsm_field_bytes(blat, bsm.FIELD_HALF_SPINOR, prec) * nrhs
    results = {}
    for block in (bsm.MRHS_TENSOR_CORE_BLOCK, 1):
        bsm.bsm_dslash_mrhs_set_block(blat, nrhs, prec, block)
        assert bsm.bsm_dslash_mrhs_block(blat, nrhs, prec) == block
        full = mrhs_field(blat, nrhs, prec)
        bsm.bsm_dslash_mrhs(blat, Ud, inp, full, nrhs, bsm.FULL, 0, prec)
        odd = mrhs_field(blat, nrhs, prec)
        bsm.bsm_dslash_mrhs(blat, Ud, inp[:half], odd[half:], nrhs, bsm.ODD, 1, prec)
        results[block] = (unpack(blat, full, nrhs, prec), unpack(blat, odd, nrhs, prec))
    bsm.bsm_dslash_mrhs_set_block(blat, nrhs, prec, 0)
    tc, simt = results[bsm.MRHS_TENSOR_CORE_BLOCK], results[1]
    for r in range(nrhs):
        assert rel(tc[0][r], orc.dirac(olat, R, psis[r])) <= TOL[prec]
        assert rel(tc[1][r], orc.hop(olat, R, psis[r], out_parity=orc.ODD, dagger=True)) <= TOL[prec]
        assert rel(tc[0][r], simt[0][r]) <= TOL[prec]


@pytest.mark.parametrize("nrhs", [12, 16])
@pytest.mark.parametrize("dims", [(12, 8, 8, 8), (6, 6, 2, 10)], ids=["8^3x12", "ragged"])
def test_mrhs_tensor_core_many_sites_per_block(dims, nrhs):
    """8^3 x 12 (V_h = 3072) has more 4-site groups than the persistent
    grid has blocks, so warps carry their copy pipeline from one site into
    the next; 6 x 6 x 2 x 10 (V_h = 360) ends in a partly filled 32-site link
    tile.  Every RHS against the oracle and against the SIMT kernel."""
    N, prec = 6, bsm.BF16
    olat, blat, U, R, psis = setup(dims, N, bsm.FUND, nrhs, 900 + nrhs)
    Ud = gpu_links(blat, U, prec)
    inp = pack(blat, psis, prec)
    results = {}
    for block in (bsm.MRHS_TENSOR_CORE_BLOCK, 1):
        bsm.bsm_dslash_mrhs_set_block(blat, nrhs, prec, block)
        full = mrhs_field(blat, nrhs, prec)
        bsm.bsm_dslash_mrhs(blat, Ud, inp, full, nrhs, bsm.FULL, 0, prec)
        results[block] = unpack(blat, full, nrhs, prec)
    bsm.bsm_dslash_mrhs_set_block(blat, nrhs, prec, 0)
    for r in range(nrhs):
        assert rel(results[bsm.MRHS_TENSOR_CORE_BLOCK][r], orc.dirac(olat, R, psis[r])) <= TOL[prec]
        assert rel(results[bsm.MRHS_TENSOR_CORE_BLOCK][r], results[1][r]) <= TOL[prec]


def test_mrhs_set_block_rejects_unavailable_blocks():
    lat = bsm.lattice((4, 4, 4, 4), 3)
    with pytest.raises(bsm.BsmError):
        bsm.bsm_dslash_mrhs_set_block(lat, 12, bsm.F32, bsm.MRHS_TENSOR_CORE_BLOCK)   # FP32, d = 3
    with pytest.raises(bsm.BsmError):
        bsm.bsm_dslash_mrhs_set_block(lat, 12, bsm.F32, 5)
    with pytest.raises(bsm.BsmError):
        bsm.bsm_dslash_mrhs_set_block(lat, 6, bsm.F32, 104)                          # 4 paired RHS, 6 RHS
    six = bsm.lattice((4, 4, 4, 4), 6)
    with pytest.raises(bsm.BsmError):
        bsm.bsm_dslash_mrhs_set_block(six, 12, bsm.F32, 104)                         # 4 paired RHS, d = 6


@pytest.mark.parametrize("prec", [bsm.F32, bsm.BF16], ids=["f32", "bf16"])
@pytest.mark.parametrize("N,rep,block", [(2, bsm.FUND, 104), (3, bsm.FUND, 102), (3, bsm.FUND, 104),
                                         (2, bsm.ADJ, 104), (6, bsm.FUND, 102), (4, bsm.ASYM, 102)],
                         ids=["SU2-F-4pair", "SU3-F-2pair", "SU3-F-4pair", "SU2-ADJ-4pair", "SU6-F-2pair",
                              "SU4-AS-2pair"])
def test_mrhs_paired_kernel_is_bit_identical(N, rep, block, prec):
    """The f32x2-paired kernel (two RHS per packed register) performs the
    scalar kernel's operations lane by lane: pinned, it gives the same bits as
    the one-RHS-per-thread kernel for both parity blocks, the adjoint and the
    full operator, and the oracle's operator per RHS."""
    dims, nrhs = (4, 4, 2, 6), 12
    olat, blat, U, R, psis = setup(dims, N, rep, nrhs, 900 + N + block)
    Ud = gpu_links(blat, U, prec)
    inp = pack(blat, psis, prec)
    half = bsm.bsm_field_bytes(blat, bsm.FIELD_HALF_SPINOR, prec) * nrhs
    results = {}
    for b in (block, 1):
        bsm.bsm_dslash_mrhs_set_block(blat, nrhs, prec, b)
        assert bsm.bsm_dslash_mrhs_block(blat, nrhs, prec) == b
        full = mrhs_field(blat, nrhs, prec)
        bsm.bsm_dslash_mrhs(blat, Ud, inp, full, nrhs, bsm.FULL, 0, prec)
        odd = mrhs_field(blat, nrhs, prec)
        bsm.bsm_dslash_mrhs(blat, Ud, inp[:half], odd[half:], nrhs, bsm.ODD, 1, prec)
        results[b] = (full, odd)
    bsm.bsm_dslash_mrhs_set_block(blat, nrhs, prec, 0)
    assert torch.equal(results[block][0], results[1][0])
    assert torch.equal(results[block][1], results[1][1])
    got = unpack(blat, results[block][0], nrhs, prec)
    for r in range(nrhs):
        assert rel(got[r], orc.dirac(olat, R, psis[r])) <= TOL[prec]


# ----------------------------------------------------------------------------
# the benchmark's multi-RHS workload at full size: 24^4, SU(6) fundamental,
# 12 RHS, in the launch shapes the benchmark times
# ----------------------------------------------------------------------------

@pytest.fixture(scope="module")
def mrhs_full_case():
    dims, N, nrhs = (24, 24, 24, 24), 6, 12
    phase = (np.pi, 0, 0, 0)
    olat = orc.Lattice(dims, N, orc.FUND, 0.1, phase)
    blat = bsm.lattice(dims, N, bsm.FUND, 0.1, phase)
    U = fields.gauge_field(dims, N, "smooth", seed=7, eps=0.4)
    R = orc.links_to_rep(olat, U)
    src = fields.device_gaussian_spinors(dims, N, nrhs, seed=9)
    return olat, blat, U, R, src, nrhs


@pytest.mark.parametrize("prec,block", [(bsm.BF16, 0), (bsm.BF16, bsm.MRHS_TENSOR_CORE_BLOCK), (bsm.BF16, 1),
                                        (bsm.F32, 0)], ids=["bf16-tuned", "bf16-tc", "bf16-simt", "f32-tuned"])
def test_full_size_24c4_mrhs(mrhs_full_case, prec, block):
    """The full operator D on all 12 RHS of the 24^4 SU(6) workload, with the
    RHS block the tuner picks (as the benchmark runs it) or pinned; RHS 0, 7
    and 11 compared with the oracle element by element."""
    olat, blat, U, R, src, nrhs = mrhs_full_case
    Ud = gpu_links(blat, U, prec)
    n = bsm.bsm_field_bytes(blat, bsm.FIELD_SPINOR, prec) * nrhs
    inp = torch.empty(n, dtype=torch.uint8, device="cuda")
    out = torch.zeros_like(inp)
    bsm.bsm_pack_spinor_mrhs(blat, src, inp, nrhs, prec)
    if block:
        bsm.bsm_dslash_mrhs_set_block(blat, nrhs, prec, block)
    bsm.bsm_dslash_mrhs(blat, Ud, inp, out, nrhs, bsm.FULL, 0, prec)
    if block:
        bsm.bsm_dslash_mrhs_set_block(blat, nrhs, prec, 0)
    got = torch.empty_like(src)
    bsm.bsm_unpack_spinor_mrhs(blat, out, got, nrhs, prec)
    for r in (0, 7, 11):
        want = orc.dirac(olat, R, src[r].cpu().numpy())
        assert rel(got[r].cpu().numpy(), want) <= TOL[prec], r
