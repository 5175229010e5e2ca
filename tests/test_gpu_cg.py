"""GPU CG through the C ABI: the FP64 solver against the oracle's CG (same
iteration, so the iterates and the iteration count agree), the mixed-precision
solver with FP64 reliable updates against the FP64 one, and the error
statuses that a caller can trigger from the host (NaN in the source,
max_iter exhaustion, a short workspace)."""
import numpy as np
import pytest
import torch

import oracle as orc
from paper_1401_3733_gb300 import bsm, fields
from tests.gpu_helpers import gpu_links, gpu_spinor, rel, to_canon, zeros_field

pytestmark = pytest.mark.gpu


def solve(blat, U64, U32, b_dev, opts, x0=None):
    x = zeros_field(blat, bsm.FIELD_SPINOR, bsm.F64)
    if x0 is not None:
        x.copy_(x0)
    ws = torch.empty(bsm.bsm_workspace_bytes(blat, bsm.CALL_CG, opts.prec_inner), dtype=torch.uint8, device="cuda")
    st, stats = bsm.bsm_cg_solve(blat, U64, U32, b_dev, x, opts, ws, raise_on_error=False)
    return st, stats, x


def cfg1():
    dims, N = (4, 4, 4, 4), 2
    olat = orc.Lattice(dims, N, orc.FUND, 0.1, (np.pi, 0, 0, 0))
    blat = bsm.lattice(dims, N, bsm.FUND, 0.1, (np.pi, 0, 0, 0))
    U = fields.gauge_field(dims, N, "haar", seed=1)
    b = fields.gaussian_spinor(dims, 2, 2)
    return olat, blat, U, b


@pytest.mark.parametrize("outer", [bsm.F64, bsm.DF64], ids=["f64", "df64"])
@pytest.mark.parametrize("eo", [True, False], ids=["eo", "full"])
def test_plain_cg_matches_oracle_cg(eo, outer):
    """Plain CG in FP64, and in FP64-accurate double-float (DF64)."""
    olat, blat, U, b = cfg1()
    R = orc.links_to_rep(olat, U)
    x_ref, it_ref, _ = orc.cg(olat, R, b, eo=eo, tol=1e-10, max_iter=5000)
    assert it_ref > 0
    U64 = gpu_links(blat, U, outer)
    st, stats, x = solve(blat, U64, None, gpu_spinor(blat, b, bsm.F64),
                         bsm.cg_opts(tol=1e-10, eo=eo, check_every=4, prec_inner=outer, prec_outer=outer))
    assert st == bsm.OK
    assert stats.true_res_normal <= 1e-10
    assert abs(stats.iters - it_ref) <= 3, (stats.iters, it_ref)
    xg = to_canon(blat, x, bsm.F64)
    assert rel(xg, x_ref) < 1e-8
    # the solution solves the full system: D x = b, checked with the oracle's D
    assert rel(orc.dirac(olat, R, xg), b) < 1e-8
    assert stats.true_res_full < 1e-8


def test_fp64_cg_initial_guess_restart():
    olat, blat, U, b = cfg1()
    U64 = gpu_links(blat, U, bsm.F64)
    bd = gpu_spinor(blat, b, bsm.F64)
    st, s1, x1 = solve(blat, U64, None, bd, bsm.cg_opts(tol=1e-5))
    assert st == bsm.OK
    st, s2, x2 = solve(blat, U64, None, bd, bsm.cg_opts(tol=1e-10, use_x0=True), x0=x1)
    st3, s3, x3 = solve(blat, U64, None, bd, bsm.cg_opts(tol=1e-10))
    assert st == bsm.OK and st3 == bsm.OK and s2.iters < s3.iters
    assert s2.true_res_normal <= 1e-10
    assert rel(to_canon(blat, x2, bsm.F64), to_canon(blat, x3, bsm.F64)) < 1e-8


@pytest.mark.parametrize("outer", [bsm.F64, bsm.DF64], ids=["f64", "df64"])
@pytest.mark.parametrize("dims,N,rep,eps", [((8, 8, 8, 8), 3, bsm.FUND, 0.3), ((8, 4, 4, 8), 2, bsm.ADJ, 0.4),
                                            ((6, 6, 4, 4), 4, bsm.ASYM, 0.4)], ids=["SU3-F", "SU2-ADJ", "SU4-AS"])
def test_mixed_precision_cg_reaches_fp64_residual(dims, N, rep, eps, outer):
    """FP32 inner iteration with reliable updates in FP64 or DF64, against
    plain FP64 CG."""
    m0 = 0.05
    blat = bsm.lattice(dims, N, rep, m0, (np.pi, 0, 0, 0))
    U = fields.gauge_field(dims, N, "smooth", seed=3, eps=eps)
    d = bsm.bsm_rep_dim(N, rep)
    b = fields.gaussian_spinor(dims, d, 4)
    U64, U32, Uo = gpu_links(blat, U, bsm.F64), gpu_links(blat, U, bsm.F32), gpu_links(blat, U, outer)
    bd = gpu_spinor(blat, b, bsm.F64)
    st64, s64, x64 = solve(blat, U64, None, bd, bsm.cg_opts(tol=1e-10))
    stm, sm, xm = solve(blat, Uo, U32, bd, bsm.cg_opts(tol=1e-10, prec_inner=bsm.F32, prec_outer=outer))
    assert st64 == bsm.OK and stm == bsm.OK
    assert s64.true_res_normal <= 1e-10 and sm.true_res_normal <= 1e-10
    assert sm.reliable_updates >= 1
    assert rel(to_canon(blat, xm, bsm.F64), to_canon(blat, x64, bsm.F64)) < 1e-7
    # the odd-site reconstruction makes x solve D x = b
    assert sm.true_res_full < 1e-7


@pytest.mark.parametrize("outer", [bsm.F64, bsm.DF64], ids=["f64", "df64"])
@pytest.mark.parametrize("eo", [True, False], ids=["eo", "full"])
def test_mixed_cg_with_two_row_links(outer, eo):
    """The FP32 inner iteration on two-row SU(3) links (BSM_F32R12), with
    antiperiodic time (the rebuilt third row carries the boundary factor),
    reaches the FP64 solution."""
    dims, N = (8, 8, 8, 8), 3
    olat = orc.Lattice(dims, N, orc.FUND, 0.05, (np.pi, 0, 0, 0))
    blat = bsm.lattice(dims, N, bsm.FUND, 0.05, (np.pi, 0, 0, 0))
    U = fields.gauge_field(dims, N, "smooth", seed=3, eps=0.3)
    b = fields.gaussian_spinor(dims, N, 4)
    U64, U12, Uo = gpu_links(blat, U, bsm.F64), gpu_links(blat, U, bsm.F32R12), gpu_links(blat, U, outer)
    bd = gpu_spinor(blat, b, bsm.F64)
    st64, s64, x64 = solve(blat, U64, None, bd, bsm.cg_opts(tol=1e-10, eo=eo))
    stm, sm, xm = solve(blat, Uo, U12, bd, bsm.cg_opts(tol=1e-10, eo=eo, prec_inner=bsm.F32R12, prec_outer=outer))
    assert st64 == bsm.OK and stm == bsm.OK
    assert sm.true_res_normal <= 1e-10 and sm.reliable_updates >= 1
    assert abs(sm.iters - s64.iters) <= max(5, s64.iters // 10), (sm.iters, s64.iters)
    x = to_canon(blat, xm, bsm.F64)
    assert rel(x, to_canon(blat, x64, bsm.F64)) < 1e-7
    R = orc.links_to_rep(olat, U)
    assert rel(orc.dirac(olat, R, x), b) < 1e-7


def test_cg_statuses_from_host_side_faults():
    olat, blat, U, b = cfg1()
    U64 = gpu_links(blat, U, bsm.F64)
    # NaN injected into the source on the host
    bn = b.copy()
    bn[5, 1, 0] = np.nan
    st, _, _ = solve(blat, U64, None, gpu_spinor(blat, bn, bsm.F64), bsm.cg_opts())
    assert st == bsm.ENAN
    # max_iter exhausted
    st, stats, _ = solve(blat, U64, None, gpu_spinor(blat, b, bsm.F64), bsm.cg_opts(max_iter=3))
    assert st == bsm.ENOCONV and stats.iters >= 3
    # workspace too small
    x = zeros_field(blat, bsm.FIELD_SPINOR, bsm.F64)
    ws = torch.empty(1024, dtype=torch.uint8, device="cuda")
    st, _ = bsm.bsm_cg_solve(blat, U64, None, gpu_spinor(blat, b, bsm.F64), x, bsm.cg_opts(), ws,
                             raise_on_error=False)
    assert st == bsm.EWORKSPACE


def test_zero_source_gives_zero_solution():
    olat, blat, U, b = cfg1()
    U64 = gpu_links(blat, U, bsm.F64)
    st, stats, x = solve(blat, U64, None, gpu_spinor(blat, np.zeros_like(b), bsm.F64), bsm.cg_opts())
    assert st == bsm.OK and stats.iters == 0
    assert np.abs(to_canon(blat, x, bsm.F64)).max() == 0


@pytest.mark.parametrize("inner,outer", [(bsm.F64, bsm.F64), (bsm.F32, bsm.DF64)], ids=["plain-f64", "mixed-df64"])
def test_graph_replay_is_bit_identical(inner, outer):
    """Capturing the iterations between host checks as a CUDA graph replays
    the same kernels in the same order: the solution is bit-identical."""
    dims, N = (8, 8, 4, 8), 3
    blat = bsm.lattice(dims, N, bsm.FUND, 0.05, (np.pi, 0, 0, 0))
    U = fields.gauge_field(dims, N, "smooth", seed=5, eps=0.3)
    b = fields.gaussian_spinor(dims, 3, 6)
    Uo, U32 = gpu_links(blat, U, outer), gpu_links(blat, U, bsm.F32)
    bd = gpu_spinor(blat, b, bsm.F64)
    stream = torch.cuda.Stream()
    xs = []
    for graph in (False, True):
        x = zeros_field(blat, bsm.FIELD_SPINOR, bsm.F64)
        ws = torch.empty(bsm.bsm_workspace_bytes(blat, bsm.CALL_CG, inner), dtype=torch.uint8, device="cuda")
        torch.cuda.synchronize()
        st, stats = bsm.bsm_cg_solve(blat, Uo, U32, bd, x,
                                     bsm.cg_opts(tol=1e-10, prec_inner=inner, prec_outer=outer, use_graph=graph),
                                     ws, stream=stream, raise_on_error=False)
        assert st == bsm.OK and stats.true_res_normal <= 1e-10
        xs.append((x.clone(), stats.iters))
    assert xs[0][1] == xs[1][1]
    assert torch.equal(xs[0][0], xs[1][0])


def test_full_size_32c64_mixed_cg_in_the_benchmark_configuration():
    """The benchmark's CG workload at full size (32^3 x 64 SU(3), smooth
    eps = 0.3 links, m0 = 0.05, antiperiodic time) in its fastest
    configuration: FP32 inner iteration on two-row links, reliable updates in
    DF64, delta = 0.01, convergence test every 16 steps.  The solution is
    checked with the oracle's Dirac operator on the CPU (the normal-equation
    tolerance 1e-10 leaves a full-system residual near 2e-10 here) and
    against plain FP64 CG."""
    dims, N, m0, phase = (64, 32, 32, 32), 3, 0.05, (np.pi, 0, 0, 0)
    olat = orc.Lattice(dims, N, orc.FUND, m0, phase)
    blat = bsm.lattice(dims, N, bsm.FUND, m0, phase)
    U = fields.gauge_field(dims, N, "smooth", seed=3, eps=0.3)
    b = fields.gaussian_spinor(dims, N, 4)
    bd = gpu_spinor(blat, b, bsm.F64)
    U12, Udf = gpu_links(blat, U, bsm.F32R12), gpu_links(blat, U, bsm.DF64)
    stm, sm, xm = solve(blat, Udf, U12, bd, bsm.cg_opts(tol=1e-10, prec_inner=bsm.F32R12, prec_outer=bsm.DF64,
                                                         delta=0.01, check_every=16))
    assert stm == bsm.OK and sm.true_res_normal <= 1e-10 and sm.reliable_updates >= 1
    x = to_canon(blat, xm, bsm.F64)
    del U12, Udf, xm
    U64 = gpu_links(blat, U, bsm.F64)
    st64, s64, x64 = solve(blat, U64, None, bd, bsm.cg_opts(tol=1e-10))
    assert st64 == bsm.OK and abs(sm.iters - s64.iters) <= max(5, s64.iters // 10), (sm.iters, s64.iters)
    assert rel(x, to_canon(blat, x64, bsm.F64)) < 1e-7
    assert rel(orc.dirac(olat, orc.links_to_rep(olat, U), x), b) < 1e-9
