"""Batched mixed-precision CG (bsm_cg_solve_batch): several lattices of
uneven size, SU(2) and SU(3), each with several right-hand sides, solved
together.  Every system's solution must solve D x = b (checked with the
oracle's D on the GPU solution), its FP64-recomputed normal-equation
residual must be <= tol, and it must agree with the single-system solver's
solution; with and without the captured CUDA graph, with FP64 and
double-float reliable updates."""
import numpy as np
import pytest
import torch

import oracle as orc
from paper_1401_3733_gb300 import bsm, fields
from tests.gpu_helpers import dev_c128, gpu_links, rel

pytestmark = pytest.mark.gpu

BATCH = [((4, 4, 4, 4), 2, 2), ((8, 4, 4, 4), 3, 4), ((6, 4, 2, 4), 3, 1), ((4, 4, 4, 8), 2, 8), ((8, 6, 6, 4), 3, 2)]
PHASE = (np.pi, 0.0, 0.0, 0.0)


def build(batch, prec_outer, m0=0.05, seed=60):
    entries, ref = [], []
    for k, (dims, N, nrhs) in enumerate(batch):
        olat = orc.Lattice(dims, N, orc.FUND, m0, PHASE)
        blat = bsm.lattice(dims, N, bsm.FUND, m0, PHASE)
        U = fields.gauge_field(dims, N, "smooth", seed=seed + k, eps=0.4)
        U64, U32 = gpu_links(blat, U, prec_outer), gpu_links(blat, U, bsm.F32)
        fb = bsm.bsm_field_bytes(blat, bsm.FIELD_SPINOR, bsm.F64)
        b = torch.empty(nrhs * fb, dtype=torch.uint8, device="cuda")
        x = torch.zeros_like(b)
        psis = []
        for r in range(nrhs):
            psi = fields.gaussian_spinor(dims, N, 100 * (seed + k) + r)
            bsm.bsm_pack_spinor(blat, dev_c128(psi), b[r * fb:(r + 1) * fb], bsm.F64)
            psis.append(psi)
        entries.append((blat, U64, U32, b, x, nrhs))
        ref.append((olat, orc.links_to_rep(olat, U), psis, fb))
    return entries, ref


def solution(blat, x, fb, r):
    V = int(np.prod(list(blat.dims)))
    c = torch.empty((V, 4, blat.N), dtype=torch.complex128, device="cuda")
    bsm.bsm_unpack_spinor(blat, x[r * fb:(r + 1) * fb], c, bsm.F64)
    torch.cuda.synchronize()
    return c.cpu().numpy()


@pytest.mark.parametrize("graph", [True, False], ids=["graph", "direct"])
@pytest.mark.parametrize("prec_outer", [bsm.F64, bsm.DF64], ids=["fp64-updates", "df64-updates"])
def test_batch_solves_every_system(prec_outer, graph):
    entries, ref = build(BATCH, prec_outer)
    items = bsm.cg_batch_items(entries)
    ws = torch.empty(bsm.bsm_cg_batch_workspace_bytes(items), dtype=torch.uint8, device="cuda")
    opts = bsm.cg_opts(tol=1e-10, max_iter=4000, prec_inner=bsm.F32, prec_outer=prec_outer, delta=0.01,
                       check_every=8, use_graph=graph)
    stream = torch.cuda.Stream()
    st, stats = bsm.bsm_cg_solve_batch(items, opts, ws, stream=stream)
    assert st == bsm.OK
    assert len(stats) == sum(n for _, _, n in BATCH)
    sys = 0
    for (blat, U64, U32, b, x, nrhs), (olat, R, psis, fb) in zip(entries, ref):
        for r in range(nrhs):
            s = stats[sys]
            assert s.true_res_normal <= 1e-10 and s.true_res_full <= 1e-9 and s.iters > 0, s.as_dict()
            xs = solution(blat, x, fb, r)
            assert rel(orc.dirac(olat, R, xs), psis[r]) <= 1e-9
            sys += 1
    # the single-system solver on one system of each lattice gives the same solution
    for (blat, U64, U32, b, x, nrhs), (olat, R, psis, fb) in zip(entries, ref):
        r = nrhs - 1
        x1 = torch.zeros(fb, dtype=torch.uint8, device="cuda")
        ws1 = torch.empty(bsm.bsm_workspace_bytes(blat, bsm.CALL_CG, bsm.F32), dtype=torch.uint8, device="cuda")
        bsm.bsm_cg_solve(blat, U64, U32, b[r * fb:(r + 1) * fb], x1,
                         bsm.cg_opts(tol=1e-10, prec_inner=bsm.F32, prec_outer=prec_outer), ws1)
        V = int(np.prod(list(blat.dims)))
        c = torch.empty((V, 4, blat.N), dtype=torch.complex128, device="cuda")
        bsm.bsm_unpack_spinor(blat, x1, c, bsm.F64)
        torch.cuda.synchronize()
        assert rel(solution(blat, x, fb, r), c.cpu().numpy()) < 1e-8


def test_batch_statuses():
    entries, _ = build(BATCH[:2], bsm.F64)
    items = bsm.cg_batch_items(entries)
    ws = torch.empty(bsm.bsm_cg_batch_workspace_bytes(items), dtype=torch.uint8, device="cuda")
    st, _ = bsm.bsm_cg_solve_batch(items, bsm.cg_opts(tol=1e-12, max_iter=8, prec_inner=bsm.F32, check_every=8), ws,
                                   raise_on_error=False)
    assert st == bsm.ENOCONV
    st, _ = bsm.bsm_cg_solve_batch(items, bsm.cg_opts(prec_inner=bsm.F64), ws, raise_on_error=False)
    assert st == bsm.EUNSUPPORTED
    st, _ = bsm.bsm_cg_solve_batch(items, bsm.cg_opts(prec_inner=bsm.F32), ws[:1024], raise_on_error=False)
    assert st == bsm.EWORKSPACE


# the benchmark's uneven batch: 16 lattices 8^4 .. 48 x 24^3, SU(2) and SU(3)
FULL_SHAPES = [((8, 8, 8, 8), 2), ((16, 8, 8, 8), 3), ((12, 12, 12, 12), 2), ((24, 12, 12, 12), 3),
               ((16, 16, 16, 16), 2), ((32, 16, 16, 16), 3), ((20, 20, 20, 20), 2), ((24, 16, 16, 16), 3),
               ((12, 8, 8, 8), 3), ((8, 12, 12, 12), 2), ((16, 12, 12, 12), 3), ((24, 24, 24, 24), 2),
               ((32, 24, 24, 24), 3), ((48, 24, 24, 24), 2), ((40, 24, 24, 24), 3), ((48, 24, 24, 24), 3)]


def test_full_size_batch_of_the_benchmark():
    """All 128 systems of the benchmark's batch (16 lattices, 8 Gaussian RHS
    each, m0 = 0.1, antiperiodic time) in one batched solve as the benchmark
    runs it (captured graph, double-float reliable updates, tol 1e-10):
    every system's recomputed normal-equation residual <= 1e-10, and on the
    two largest and two small lattices the oracle's D applied to the GPU
    solution gives back b (RHS 0 and 7)."""
    nrhs, phase, m0 = 8, (np.pi, 0.0, 0.0, 0.0), 0.1
    entries, refs = [], []
    for k, (dims, N) in enumerate(FULL_SHAPES):
        blat = bsm.lattice(dims, N, bsm.FUND, m0, phase)
        U = fields.gauge_field(dims, N, "smooth", seed=20 + k, eps=0.3)
        U64, U32 = gpu_links(blat, U, bsm.DF64), gpu_links(blat, U, bsm.F32)
        fb = bsm.bsm_field_bytes(blat, bsm.FIELD_SPINOR, bsm.F64)
        src = fields.device_gaussian_spinors(dims, N, nrhs, seed=40 + k)
        b = torch.empty(nrhs * fb, dtype=torch.uint8, device="cuda")
        for r in range(nrhs):
            bsm.bsm_pack_spinor(blat, src[r], b[r * fb:(r + 1) * fb], bsm.F64)
        entries.append((blat, U64, U32, b, torch.zeros_like(b), nrhs))
        refs.append((dims, N, U, src, fb))
    items = bsm.cg_batch_items(entries)
    ws = torch.empty(bsm.bsm_cg_batch_workspace_bytes(items), dtype=torch.uint8, device="cuda")
    opts = bsm.cg_opts(tol=1e-10, max_iter=20000, prec_inner=bsm.F32, prec_outer=bsm.DF64, delta=0.01,
                       check_every=16, use_graph=True)
    st, stats = bsm.bsm_cg_solve_batch(items, opts, ws, stream=torch.cuda.Stream())
    assert st == bsm.OK
    assert len(stats) == 16 * nrhs
    assert max(s.true_res_normal for s in stats) <= 1e-10
    for k in (0, 1, 13, 15):
        dims, N, U, src, fb = refs[k]
        blat, _, _, _, x, _ = entries[k]
        olat = orc.Lattice(dims, N, orc.FUND, m0, phase)
        R = orc.links_to_rep(olat, U)
        for r in (0, 7):
            b = src[r].cpu().numpy()
            assert rel(orc.dirac(olat, R, solution(blat, x, fb, r)), b) <= 1e-9, (dims, r)
