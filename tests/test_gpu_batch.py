"""bsm_dslash_batch: uneven SU(2)/SU(3) lattices, each with its own number
of right-hand sides, in one persistent cooperative launch fed by a device
work queue.  Every RHS of every lattice equals the oracle's operator; the
two-phase even-odd operator crosses a grid barrier whose bounded wait is
also driven to time out (an arrival that never comes) to check that the call
returns BSM_ETIMEOUT and leaves the GPU usable."""
import numpy as np
import pytest
import torch

import oracle as orc
from paper_1401_3733_gb300 import bsm, fields
from tests.gpu_helpers import TOL, dev_c128, gpu_links, rel

pytestmark = pytest.mark.gpu

SHAPES = [((4, 4, 4, 4), 3, 2), ((2, 4, 6, 8), 2, 3), ((6, 6, 4, 4), 3, 1), ((8, 4, 2, 4), 2, 2),
          ((4, 2, 2, 2), 3, 3)]   # (dims, N, nrhs)


def make_batch(op, seed=900, shapes=SHAPES):
    items, refs = [], []
    for k, (dims, N, nrhs) in enumerate(shapes):
        phase = (np.pi, 0, 0, 0)
        olat = orc.Lattice(dims, N, orc.FUND, 0.1 + 0.05 * k, phase)
        blat = bsm.lattice(dims, N, bsm.FUND, 0.1 + 0.05 * k, phase)
        U = fields.gauge_field(dims, N, "haar", seed=seed + k)
        R = orc.links_to_rep(olat, U)
        psis = [fields.gaussian_spinor(dims, N, seed + 100 * k + r) for r in range(nrhs)]
        if op == bsm.BATCH_DHAT:
            odd = orc.parity_mask(dims)
            for p in psis:
                p[odd] = 0
        full = bsm.bsm_field_bytes(blat, bsm.FIELD_SPINOR, bsm.F32) * nrhs
        inp = torch.zeros(full, dtype=torch.uint8, device="cuda")
        out = torch.zeros(full, dtype=torch.uint8, device="cuda")
        bsm.bsm_pack_spinor_mrhs(blat, dev_c128(np.stack(psis)), inp, nrhs, bsm.F32)
        Ud = gpu_links(blat, U, bsm.F32)
        if op == bsm.BATCH_DHAT:   # even halves
            half = full // 2
            items.append((blat, Ud, inp[:half], out[:half], nrhs))
        else:
            items.append((blat, Ud, inp, out, nrhs))
        refs.append((olat, R, psis, blat, out, nrhs))
    return items, refs


def unpack(blat, dev, nrhs):
    V = int(np.prod(list(blat.dims)))
    c = torch.empty((nrhs, V, 4, blat.N), dtype=torch.complex128, device="cuda")
    bsm.bsm_unpack_spinor_mrhs(blat, dev, c, nrhs, bsm.F32)
    torch.cuda.synchronize()
    return c.cpu().numpy()


@pytest.mark.parametrize("op", [bsm.BATCH_D, bsm.BATCH_DHAT], ids=["D", "Dhat"])
def test_batch_matches_oracle(op):
    items, refs = make_batch(op)
    arr = bsm.batch_items(items)
    opts = bsm.BatchOpts(op, bsm.F32, 0.0, 0)
    ws = torch.empty(bsm.bsm_batch_workspace_bytes(arr, opts), dtype=torch.uint8, device="cuda")
    assert bsm.bsm_dslash_batch(arr, opts, ws) == bsm.OK
    for olat, R, psis, blat, out, nrhs in refs:
        got = unpack(blat, out, nrhs)
        for r in range(nrhs):
            want = orc.dirac(olat, R, psis[r]) if op == bsm.BATCH_D else orc.dhat(olat, R, psis[r], orc.DHAT)
            assert rel(got[r], want) <= TOL[bsm.F32], (blat.dims[:], r, rel(got[r], want))


def test_barrier_timeout_returns_etimeout_and_gpu_stays_usable():
    items, refs = make_batch(bsm.BATCH_DHAT, seed=950)
    arr = bsm.batch_items(items)
    ws_opts = bsm.BatchOpts(bsm.BATCH_DHAT, bsm.F32, 0.05, 0)
    ws = torch.empty(bsm.bsm_batch_workspace_bytes(arr, ws_opts), dtype=torch.uint8, device="cuda")
    # one phantom arrival that never comes: every block's bounded wait expires
    st = bsm.bsm_dslash_batch(arr, bsm.BatchOpts(bsm.BATCH_DHAT, bsm.F32, 0.05, 1), ws, raise_on_error=False)
    assert st == bsm.ETIMEOUT
    # the context is intact: the same batch now completes and is correct
    assert bsm.bsm_dslash_batch(arr, ws_opts, ws) == bsm.OK
    olat, R, psis, blat, out, nrhs = refs[0]
    got = unpack(blat, out, nrhs)
    assert rel(got[0], orc.dhat(olat, R, psis[0], orc.DHAT)) <= TOL[bsm.F32]


@pytest.mark.parametrize("op", [bsm.BATCH_D, bsm.BATCH_DHAT], ids=["D", "Dhat"])
def test_batch_captured_in_a_cuda_graph(op):
    """bsm_dslash_batch_async captured into a CUDA graph on a side stream:
    each replay reruns the whole persistent batch (work queue reset by the
    captured memset) and gives the oracle's result; the status query reads
    the error flag after the replays."""
    items, refs = make_batch(op, seed=970)
    arr = bsm.batch_items(items)
    opts = bsm.BatchOpts(op, bsm.F32, 0.0, 0)
    ws = torch.empty(bsm.bsm_batch_workspace_bytes(arr, opts), dtype=torch.uint8, device="cuda")
    s = torch.cuda.Stream()
    bsm.bsm_dslash_batch_async(arr, opts, ws, stream=s)   # eager run first (occupancy query, module load)
    assert bsm.bsm_dslash_batch_status(ws, stream=s) == bsm.OK
    for _, _, _, _, out, _ in refs:
        out.zero_()
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s, capture_error_mode="relaxed"):
        bsm.bsm_dslash_batch_async(arr, opts, ws, stream=s)
    for _ in range(3):
        g.replay()
    torch.cuda.synchronize()
    assert bsm.bsm_dslash_batch_status(ws, stream=s) == bsm.OK
    for olat, R, psis, blat, out, nrhs in refs:
        got = unpack(blat, out, nrhs)
        for r in range(nrhs):
            want = orc.dirac(olat, R, psis[r]) if op == bsm.BATCH_D else orc.dhat(olat, R, psis[r], orc.DHAT)
            assert rel(got[r], want) <= TOL[bsm.F32], (blat.dims[:], r, rel(got[r], want))


def test_async_batch_timeout_is_reported_by_the_status_query():
    items, refs = make_batch(bsm.BATCH_DHAT, seed=990)
    arr = bsm.batch_items(items)
    opts = bsm.BatchOpts(bsm.BATCH_DHAT, bsm.F32, 0.05, 0)
    ws = torch.empty(bsm.bsm_batch_workspace_bytes(arr, opts), dtype=torch.uint8, device="cuda")
    assert bsm.bsm_dslash_batch_async(arr, bsm.BatchOpts(bsm.BATCH_DHAT, bsm.F32, 0.05, 1), ws) == bsm.OK
    assert bsm.bsm_dslash_batch_status(ws) == bsm.ETIMEOUT
    assert bsm.bsm_dslash_batch_async(arr, opts, ws) == bsm.OK
    assert bsm.bsm_dslash_batch_status(ws) == bsm.OK


EVEN_SHAPES = [((4, 4, 4, 4), 3, 2), ((6, 4, 2, 4), 2, 4), ((8, 4, 4, 2), 3, 2)]


@pytest.mark.parametrize("op", [bsm.BATCH_D, bsm.BATCH_DHAT], ids=["D", "Dhat"])
def test_tuned_launch_configuration_changes_nothing(op, monkeypatch):
    """The first call on a batch shape times every (RHS per thread, chunks
    per grab) candidate, packed-pair blocks included, and keeps the fastest;
    with BSM_BATCH_TUNE=0 an untuned shape runs (1, 4).  Both give the same
    bits, and the oracle's."""
    items, refs = make_batch(op, seed=970, shapes=EVEN_SHAPES)
    arr = bsm.batch_items(items)
    opts = bsm.BatchOpts(op, bsm.F32, 0.0, 0)
    ws = torch.empty(bsm.bsm_batch_workspace_bytes(arr, opts), dtype=torch.uint8, device="cuda")
    monkeypatch.setenv("BSM_BATCH_TUNE", "0")
    assert bsm.bsm_dslash_batch(arr, opts, ws) == bsm.OK
    assert bsm.bsm_batch_last_config() == (1, 4)
    first = [ref[4].clone() for ref in refs]
    monkeypatch.delenv("BSM_BATCH_TUNE")
    assert bsm.bsm_dslash_batch(arr, opts, ws) == bsm.OK
    rb, grab = bsm.bsm_batch_last_config()
    assert rb in (1, 2, 102, 104) and grab in (1, 2, 4, 8)
    for (olat, R, psis, blat, out, nrhs), f in zip(refs, first):
        assert torch.equal(out, f)
        got = unpack(blat, out, nrhs)
        for r in range(nrhs):
            want = orc.dirac(olat, R, psis[r]) if op == bsm.BATCH_D else orc.dhat(olat, R, psis[r], orc.DHAT)
            assert rel(got[r], want) <= TOL[bsm.F32]


@pytest.mark.parametrize("op", [bsm.BATCH_D, bsm.BATCH_DHAT], ids=["D", "Dhat"])
def test_every_launch_configuration_gives_the_same_bits(op, monkeypatch):
    """Each RHS block (1 and 2 RHS per thread, 2 and 4 as packed pairs),
    pinned with BSM_BATCH_CONFIG, against the default (1, 4): the same bits,
    on lattices whose nrhs (4) admit every block."""
    shapes = [((4, 4, 4, 4), 3, 4), ((6, 4, 2, 4), 2, 4), ((8, 4, 4, 2), 3, 4)]
    items, refs = make_batch(op, seed=980, shapes=shapes)
    arr = bsm.batch_items(items)
    opts = bsm.BatchOpts(op, bsm.F32, 0.0, 0)
    ws = torch.empty(bsm.bsm_batch_workspace_bytes(arr, opts), dtype=torch.uint8, device="cuda")
    monkeypatch.setenv("BSM_BATCH_CONFIG", "1:4")
    assert bsm.bsm_dslash_batch(arr, opts, ws) == bsm.OK
    base = [ref[4].clone() for ref in refs]
    for olat, R, psis, blat, out, nrhs in refs:
        got = unpack(blat, out, nrhs)
        for r in range(nrhs):
            want = orc.dirac(olat, R, psis[r]) if op == bsm.BATCH_D else orc.dhat(olat, R, psis[r], orc.DHAT)
            assert rel(got[r], want) <= TOL[bsm.F32]
    for cfg in ("2:1", "102:2", "104:8", "104:1"):
        monkeypatch.setenv("BSM_BATCH_CONFIG", cfg)
        for ref in refs:
            ref[4].zero_()
        assert bsm.bsm_dslash_batch(arr, opts, ws) == bsm.OK
        assert bsm.bsm_batch_last_config() == tuple(int(v) for v in cfg.split(":"))
        for ref, b in zip(refs, base):
            assert torch.equal(ref[4], b), cfg


# the benchmark's uneven batch: 16 lattices 8^4 .. 48 x 24^3, SU(2) and SU(3)
FULL_SHAPES = [((8, 8, 8, 8), 2), ((16, 8, 8, 8), 3), ((12, 12, 12, 12), 2), ((24, 12, 12, 12), 3),
               ((16, 16, 16, 16), 2), ((32, 16, 16, 16), 3), ((20, 20, 20, 20), 2), ((24, 16, 16, 16), 3),
               ((12, 8, 8, 8), 3), ((8, 12, 12, 12), 2), ((16, 12, 12, 12), 3), ((24, 24, 24, 24), 2),
               ((32, 24, 24, 24), 3), ((48, 24, 24, 24), 2), ((40, 24, 24, 24), 3), ((48, 24, 24, 24), 3)]


def test_full_size_uneven_batch_of_the_benchmark():
    """The 16-lattice batch at full size, 8 RHS each, the full operator in
    one persistent launch in the tuned configuration (as the benchmark runs
    it): on the two largest and two small lattices RHS 0 and 7 against the
    oracle, and on every lattice all RHS against one multi-RHS launch per
    lattice (the same site arithmetic, so to rounding order)."""
    nrhs, phase = 8, (np.pi, 0, 0, 0)
    entries, refs = [], []
    for k, (dims, N) in enumerate(FULL_SHAPES):
        blat = bsm.lattice(dims, N, bsm.FUND, 0.1, phase)
        U = fields.gauge_field(dims, N, "smooth", seed=20 + k, eps=0.3)
        Ud = gpu_links(blat, U, bsm.F32)
        src = fields.device_gaussian_spinors(dims, N, nrhs, seed=40 + k)
        n = bsm.bsm_field_bytes(blat, bsm.FIELD_SPINOR, bsm.F32) * nrhs
        inp = torch.empty(n, dtype=torch.uint8, device="cuda")
        out = torch.zeros_like(inp)
        bsm.bsm_pack_spinor_mrhs(blat, src, inp, nrhs, bsm.F32)
        entries.append((blat, Ud, inp, out, nrhs))
        refs.append((dims, N, U, src))
    arr = bsm.batch_items(entries)
    opts = bsm.BatchOpts(bsm.BATCH_D, bsm.F32, 0.0, 0)
    ws = torch.empty(bsm.bsm_batch_workspace_bytes(arr, opts), dtype=torch.uint8, device="cuda")
    assert bsm.bsm_dslash_batch(arr, opts, ws) == bsm.OK
    for k, ((blat, Ud, inp, out, _), (dims, N, U, src)) in enumerate(zip(entries, refs)):
        got = torch.empty_like(src)
        bsm.bsm_unpack_spinor_mrhs(blat, out, got, nrhs, bsm.F32)
        one = torch.zeros_like(out)
        bsm.bsm_dslash_mrhs(blat, Ud, inp, one, nrhs, bsm.FULL, 0, bsm.F32)
        ref = torch.empty_like(src)
        bsm.bsm_unpack_spinor_mrhs(blat, one, ref, nrhs, bsm.F32)
        assert float((got - ref).norm() / ref.norm()) <= 1e-6, dims
        if k in (0, 1, 13, 15):
            olat = orc.Lattice(dims, N, orc.FUND, 0.1, phase)
            R = orc.links_to_rep(olat, U)
            for r in (0, 7):
                assert rel(got[r].cpu().numpy(), orc.dirac(olat, R, src[r].cpu().numpy())) <= TOL[bsm.F32], (dims, r)
