"""The C-ABI library without a GPU: it builds, loads, exports every symbol
that include/bsm.h declares, answers size queries, and rejects bad arguments
on the host before any launch (fake device addresses are passed where the
call must return before touching them)."""
import ctypes
import math
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def bsm():
    from paper_1401_3733_gb300 import build
    build.build()
    from paper_1401_3733_gb300 import bsm as mod
    return mod


def declared_functions():
    text = open(os.path.join(ROOT, "include", "bsm.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(bsm_[a-z0-9_]+)\s*\(", text)))


def test_every_declared_symbol_is_exported(bsm):
    names = declared_functions()
    assert len(names) >= 11
    lib = ctypes.CDLL(bsm.library_path())
    for n in names:
        assert hasattr(lib, n), n


def test_rep_dims(bsm):
    want = {(2, bsm.FUND): 2, (3, bsm.FUND): 3, (4, bsm.FUND): 4, (6, bsm.FUND): 6, (8, bsm.FUND): 8,
            (2, bsm.ADJ): 3, (3, bsm.ADJ): 8, (2, bsm.SYM): 3, (3, bsm.SYM): 6, (3, bsm.ASYM): 3, (4, bsm.ASYM): 6}
    for (N, r), d in want.items():
        assert bsm.bsm_rep_dim(N, r) == d
    for N, r in [(5, bsm.FUND), (2, bsm.ASYM), (4, bsm.ADJ), (1, bsm.FUND), (3, 9)]:
        assert bsm.bsm_rep_dim(N, r) == bsm.EUNSUPPORTED


def test_field_and_workspace_sizes(bsm):
    lat = bsm.lattice((64, 32, 32, 32), 3)
    V, Vh, d = 64 * 32 ** 3, 64 * 32 ** 3 // 2, 3
    assert bsm.bsm_field_bytes(lat, bsm.FIELD_SPINOR, bsm.F64) == V * 4 * d * 16
    assert bsm.bsm_field_bytes(lat, bsm.FIELD_SPINOR, bsm.F32) == V * 4 * d * 8
    assert bsm.bsm_field_bytes(lat, bsm.FIELD_HALF_SPINOR, bsm.F32) == Vh * 4 * d * 8
    # every link stored twice (forward of its site, backward of its neighbour)
    assert bsm.bsm_field_bytes(lat, bsm.FIELD_LINKS, bsm.F64) == 2 * 4 * V * d * d * 16
    assert bsm.bsm_field_bytes(lat, bsm.FIELD_LINKS, bsm.F32) == 2 * 4 * V * d * d * 8
    # links are tiled by 32 sites: a 2^4 lattice (V_h = 8) pads to one tile
    tiny = bsm.lattice((2, 2, 2, 2), 3)
    assert bsm.bsm_field_bytes(tiny, bsm.FIELD_LINKS, bsm.F32) == 2 * 32 * 8 * 9 * 4 * 2
    adj = bsm.lattice((4, 4, 4, 4), 2, bsm.ADJ)
    assert bsm.bsm_field_bytes(adj, bsm.FIELD_LINKS, bsm.F32) == 2 * 4 * 256 * 9 * 4
    assert bsm.bsm_field_bytes(lat, bsm.FIELD_FUND_CANON) == V * 4 * 9 * 16
    assert bsm.bsm_field_bytes(lat, bsm.FIELD_SPINOR_CANON) == V * 4 * d * 16
    assert bsm.bsm_workspace_bytes(lat, bsm.CALL_DIRAC_EO, bsm.F32) == 2 * Vh * 4 * d * 8
    ws64 = bsm.bsm_workspace_bytes(lat, bsm.CALL_CG, bsm.F64)
    ws32 = bsm.bsm_workspace_bytes(lat, bsm.CALL_CG, bsm.F32)
    assert ws64 >= 6 * Vh * 4 * d * 16 and ws32 > ws64


@pytest.mark.parametrize("dims", [(4, 4, 4, 3), (0, 4, 4, 4), (4, 4, 1, 4), (-2, 4, 4, 4)])
def test_bad_extents_rejected(bsm, dims):
    lat = bsm.lattice(dims, 3)
    assert bsm.bsm_field_bytes(lat, bsm.FIELD_SPINOR, bsm.F64) == 0
    assert bsm._lib.bsm_dslash(ctypes.byref(lat), 256, 512, 1024, bsm.EVEN, 0, bsm.F64, 0) == bsm.EINVAL


def test_host_validation_paths(bsm):
    L = ctypes.byref
    good = bsm.lattice((4, 4, 4, 4), 3, bsm.FUND, 0.1, (math.pi, 0, 0, 0))
    A = 1 << 20  # fake, 16-byte aligned device addresses: never dereferenced
    # unsupported (N, rep), real representation with a generic phase, A == 0
    assert bsm._lib.bsm_dslash(L(bsm.lattice((4, 4, 4, 4), 5)), A, 2 * A, 3 * A, 0, 0, 0, 0) == bsm.EUNSUPPORTED
    adj = bsm.lattice((4, 4, 4, 4), 2, bsm.ADJ, 0.1, (0.3, 0, 0, 0))
    assert bsm._lib.bsm_links_to_rep(L(adj), A, 2 * A, bsm.F64, 0) == bsm.EUNSUPPORTED
    assert bsm._lib.bsm_dslash(L(bsm.lattice((4, 4, 4, 4), 3, bsm.FUND, -4.0)), A, 2 * A, 3 * A, 0, 0, 0, 0) \
        == bsm.EINVAL
    # null and misaligned pointers, bad enums, aliasing input and output
    assert bsm._lib.bsm_dslash(L(good), None, 2 * A, 3 * A, 0, 0, 0, 0) == bsm.EINVAL
    assert bsm._lib.bsm_dslash(L(good), A, 2 * A + 8, 3 * A, 0, 0, 0, 0) == bsm.EINVAL
    assert bsm._lib.bsm_dslash(L(good), A, 2 * A, 3 * A, 7, 0, 0, 0) == bsm.EINVAL
    assert bsm._lib.bsm_dslash(L(good), A, 2 * A, 3 * A, 0, 0, 5, 0) == bsm.EUNSUPPORTED
    assert bsm._lib.bsm_dslash(L(good), A, 2 * A, 2 * A + 256, 0, 0, 0, 0) == bsm.EINVAL
    assert bsm._lib.bsm_pack_spinor(L(good), None, A, 0, 0) == bsm.EINVAL
    # dirac_eo: bad op, short workspace
    assert bsm._lib.bsm_dirac_eo(L(good), A, 2 * A, 3 * A, 9, 0, 4 * A, 1 << 30, 0) == bsm.EINVAL
    assert bsm._lib.bsm_dirac_eo(L(good), A, 2 * A, 3 * A, 0, 0, 4 * A, 16, 0) == bsm.EWORKSPACE


def test_cg_option_validation(bsm):
    L = ctypes.byref
    good = bsm.lattice((4, 4, 4, 4), 2, bsm.FUND, 0.1, (math.pi, 0, 0, 0))
    A = 1 << 24
    big = 1 << 40

    def call(opts, ws_bytes=big, U32=None):
        st = bsm.CgStats()
        return bsm._lib.bsm_cg_solve(L(good), A, U32, 2 * A, 3 * A, L(opts), L(st), 4 * A, ws_bytes, 0)

    assert call(bsm.cg_opts(tol=0.0)) == bsm.EINVAL
    assert call(bsm.cg_opts(tol=-1.0)) == bsm.EINVAL
    assert call(bsm.cg_opts(max_iter=0)) == bsm.EINVAL
    assert call(bsm.cg_opts(delta=1.5)) == bsm.EINVAL
    assert call(bsm.cg_opts(prec_inner=9)) == bsm.EUNSUPPORTED
    assert call(bsm.cg_opts(prec_inner=bsm.F32)) == bsm.EINVAL        # mixed precision needs FP32 links
    assert call(bsm.cg_opts(), ws_bytes=4096) == bsm.EWORKSPACE


def test_mrhs_validation(bsm):
    L = ctypes.byref
    good = bsm.lattice((4, 4, 4, 4), 3)
    A = 1 << 20
    assert bsm._lib.bsm_dslash_mrhs(L(good), A, 2 * A, 3 * A, 0, bsm.FULL, 0, bsm.F32, 0) == bsm.EINVAL
    assert bsm._lib.bsm_dslash_mrhs(L(good), A, 2 * A, 3 * A, 4, bsm.FULL, 0, bsm.F64, 0) == bsm.EUNSUPPORTED
    assert bsm._lib.bsm_dslash_mrhs(L(good), A, 2 * A, 3 * A, 4, 9, 0, bsm.F32, 0) == bsm.EINVAL
    assert bsm._lib.bsm_dslash_mrhs(L(good), A, 2 * A, 2 * A + 64, 4, bsm.EVEN, 0, bsm.F32, 0) == bsm.EINVAL
    big = bsm.lattice((64, 64, 64, 64), 3)   # V * nrhs beyond 2^30
    assert bsm._lib.bsm_dslash_mrhs(L(big), A, 2 * A, 3 * A, 128, bsm.FULL, 0, bsm.F32, 0) == bsm.EUNSUPPORTED
    assert bsm._lib.bsm_pack_spinor_mrhs(L(good), None, A, 4, bsm.F32, 0) == bsm.EINVAL
    assert bsm.bsm_dslash_mrhs_block(good, 12, bsm.F32) == 0        # nothing tuned yet
    assert bsm.bsm_dslash_mrhs_block(good, 12, bsm.F64) == bsm.EUNSUPPORTED


def test_batch_validation(bsm):
    A = 1 << 20
    good = bsm.lattice((4, 4, 4, 4), 3)
    items = bsm.batch_items([(good, A, 2 * A, 3 * A, 2), (bsm.lattice((2, 4, 6, 8), 2), 4 * A, 5 * A, 6 * A, 1)])
    ok = bsm.BatchOpts(bsm.BATCH_D, bsm.F32, 0.0, 0)
    assert bsm.bsm_batch_workspace_bytes(items, ok) > 0
    assert bsm._lib.bsm_dslash_batch(items, 0, ctypes.byref(ok), 7 * A, 1 << 30, 0) == bsm.EINVAL
    assert bsm._lib.bsm_dslash_batch(items, 2, ctypes.byref(bsm.BatchOpts(9, bsm.F32, 0, 0)), 7 * A, 1 << 30, 0) \
        == bsm.EINVAL
    assert bsm._lib.bsm_dslash_batch(items, 2, ctypes.byref(bsm.BatchOpts(0, bsm.F64, 0, 0)), 7 * A, 1 << 30, 0) \
        == bsm.EUNSUPPORTED
    assert bsm._lib.bsm_dslash_batch(items, 2, ctypes.byref(ok), 7 * A, 16, 0) == bsm.EWORKSPACE
    su4 = bsm.batch_items([(bsm.lattice((4, 4, 4, 4), 4), A, 2 * A, 3 * A, 1)])
    assert bsm._lib.bsm_dslash_batch(su4, 1, ctypes.byref(ok), 7 * A, 1 << 30, 0) == bsm.EUNSUPPORTED


def test_two_row_links_are_su3_fundamental_only(bsm):
    L = ctypes.byref
    A = 1 << 20
    su3 = bsm.lattice((4, 4, 4, 4), 3, bsm.FUND, 0.1, (math.pi, 0, 0, 0))
    Vh = 128
    assert bsm.bsm_field_bytes(su3, bsm.FIELD_LINKS, bsm.F32R12) == 2 * Vh * 8 * 12 * 4
    assert bsm.bsm_field_bytes(su3, bsm.FIELD_SPINOR, bsm.F32R12) == bsm.bsm_field_bytes(su3, bsm.FIELD_SPINOR,
                                                                                         bsm.F32)
    assert bsm.bsm_workspace_bytes(su3, bsm.CALL_CG, bsm.F32R12) == bsm.bsm_workspace_bytes(su3, bsm.CALL_CG, bsm.F32)
    for lat in (bsm.lattice((4, 4, 4, 4), 2), bsm.lattice((4, 4, 4, 4), 3, bsm.SYM), bsm.lattice((4, 4, 4, 4), 4)):
        assert bsm.bsm_field_bytes(lat, bsm.FIELD_LINKS, bsm.F32R12) == 0
        assert bsm._lib.bsm_dslash(L(lat), A, 2 * A, 3 * A, 0, 0, bsm.F32R12, 0) == bsm.EUNSUPPORTED
        assert bsm._lib.bsm_links_to_rep(L(lat), A, 2 * A, bsm.F32R12, 0) == bsm.EUNSUPPORTED
        st = bsm.CgStats()
        assert bsm._lib.bsm_cg_solve(L(lat), A, 2 * A, 3 * A, 4 * A, L(bsm.cg_opts(prec_inner=bsm.F32R12)), L(st),
                                     5 * A, 1 << 40, 0) == bsm.EUNSUPPORTED
    # the multi-RHS and batch paths take plain FP32 links only
    assert bsm._lib.bsm_dslash_mrhs(L(su3), A, 2 * A, 3 * A, 4, bsm.FULL, 0, bsm.F32R12, 0) == bsm.EUNSUPPORTED


def test_too_large_lattice_is_unsupported(bsm):
    lat = bsm.lattice((2048, 1024, 1024, 2), 3)
    assert bsm.bsm_field_bytes(lat, bsm.FIELD_SPINOR, bsm.F32) == 0
    assert bsm._lib.bsm_dslash(ctypes.byref(lat), 256, 512, 1024, 0, 0, 0, 0) == bsm.EUNSUPPORTED


def test_strerror_covers_every_status(bsm):
    for s in range(0, -9, -1):
        assert bsm.bsm_strerror(s) not in ("", "unknown status")
    assert bsm.bsm_strerror(-99) == "unknown status"


def test_ptc_and_fgcr_validation(bsm):
    L = ctypes.byref
    A = 1 << 20
    big = 1 << 40
    good = bsm.lattice((4, 4, 4, 4), 3)
    adj = bsm.lattice((4, 4, 4, 4), 2, bsm.ADJ)
    su4 = bsm.lattice((4, 4, 4, 4), 4)
    assert bsm.bsm_ptc_workspace_bytes(good, 12, 2, 1) > bsm.bsm_ptc_workspace_bytes(good, 12, 2, 0) > 0
    for lat, C, nb in [(adj, 4, 1), (su4, 4, 1), (good, 0, 1), (good, 65, 1), (good, 4, 0)]:
        assert bsm.bsm_ptc_workspace_bytes(lat, C, nb, 0) == 0
    apply = bsm._lib.bsm_ptc_apply
    assert apply(L(adj), A, 2 * A, 3 * A, 4, 4 * A, 5 * A, 1, bsm.F32, 6 * A, big, 0) == bsm.EUNSUPPORTED
    # the status query rejects a missing or misaligned workspace before touching the GPU
    assert bsm._lib.bsm_ptc_status(None, None) == bsm.EINVAL
    assert bsm._lib.bsm_ptc_status(A + 4, None) == bsm.EINVAL
    assert apply(L(good), A, 2 * A, 3 * A, 4, 4 * A, 5 * A, 1, bsm.F64, 6 * A, big, 0) == bsm.EUNSUPPORTED
    assert apply(L(good), A, 2 * A, 3 * A, 0, 4 * A, 5 * A, 1, bsm.F32, 6 * A, big, 0) == bsm.EINVAL
    assert apply(L(good), A, 2 * A + 4, 3 * A, 4, 4 * A, 5 * A, 1, bsm.F32, 6 * A, big, 0) == bsm.EINVAL
    assert apply(L(good), A, 2 * A, 3 * A, 4, 4 * A, 4 * A + 64, 1, bsm.F32, 6 * A, big, 0) == bsm.EINVAL
    assert apply(L(good), A, 2 * A, 3 * A, 4, 4 * A, 5 * A, 1, bsm.F32, 6 * A, 1024, 0) == bsm.EWORKSPACE
    loss = ctypes.c_double()
    assert bsm._lib.bsm_ptc_loss_grad(L(good), A, 2 * A, 3 * A, 4, 4 * A, 5 * A, 1, 6 * A, 7 * A, None, 8 * A, big,
                                      0) == bsm.EINVAL
    assert bsm._lib.bsm_ptc_loss_grad(L(good), A, 2 * A, 3 * A, 4, 4 * A, 5 * A, 1, 6 * A, 7 * A, L(loss), 8 * A,
                                      1024, 0) == bsm.EWORKSPACE
    assert bsm._lib.bsm_ptc_adam_step(A, 2 * A, 3 * A, 4 * A, 0, 1e-3, 1, 0) == bsm.EINVAL
    assert bsm._lib.bsm_ptc_adam_step(A, 2 * A, 3 * A, 4 * A, 16, 1e-3, 0, 0) == bsm.EINVAL
    assert bsm._lib.bsm_ptc_pack(L(adj), A, 2 * A, 0) == bsm.EUNSUPPORTED
    assert bsm._lib.bsm_ptc_unpack(L(good), None, 2 * A, 0) == bsm.EINVAL

    def solve(opts, ws_bytes=big, W=A):
        st = bsm.FgcrStats()
        return bsm._lib.bsm_fgcr_solve(L(good), A, 2 * A, W, W, 3 * A, 4 * A, L(opts), L(st), 5 * A, ws_bytes, 0)

    assert bsm.bsm_fgcr_workspace_bytes(good, bsm.fgcr_opts(restart=0)) == 0
    assert bsm.bsm_fgcr_workspace_bytes(good, bsm.fgcr_opts(restart=8, precond=bsm.FGCR_PTC, channels=4)) > \
        bsm.bsm_fgcr_workspace_bytes(good, bsm.fgcr_opts(restart=8)) > 0
    # with the CG fallback the workspace holds either solver
    assert bsm.bsm_fgcr_workspace_bytes(good, bsm.fgcr_opts(restart=2, fallback=True)) >= max(
        bsm.bsm_fgcr_workspace_bytes(good, bsm.fgcr_opts(restart=2)),
        bsm.bsm_workspace_bytes(good, bsm.CALL_CG, bsm.F64))
    assert solve(bsm.fgcr_opts(fallback=True, fallback_max_iter=-1)) == bsm.EINVAL
    assert solve(bsm.fgcr_opts(tol=0.0)) == bsm.EINVAL
    assert solve(bsm.fgcr_opts(restart=65)) == bsm.EINVAL
    assert solve(bsm.fgcr_opts(precond=7)) == bsm.EINVAL
    assert solve(bsm.fgcr_opts(precond=bsm.FGCR_PTC, channels=4, ptc_prec=bsm.F64)) == bsm.EUNSUPPORTED
    assert solve(bsm.fgcr_opts(precond=bsm.FGCR_PTC, channels=4), W=None) == bsm.EINVAL
    assert solve(bsm.fgcr_opts(), ws_bytes=4096) == bsm.EWORKSPACE
    assert solve(bsm.fgcr_opts(prec_inner=9)) == bsm.EUNSUPPORTED
    assert solve(bsm.fgcr_opts(prec_inner=bsm.F32, inner_tol=1.5)) == bsm.EINVAL
    st = bsm.FgcrStats()
    assert bsm._lib.bsm_fgcr_solve(L(good), A, None, None, None, 3 * A, 4 * A, L(bsm.fgcr_opts(prec_inner=bsm.F32)),
                                   L(st), 5 * A, big, 0) == bsm.EINVAL   # FP32 cycles need FP32 links
    # FP32 cycles keep their 2 x restart basis vectors in FP32: half the bytes
    assert 0 < bsm.bsm_fgcr_workspace_bytes(good, bsm.fgcr_opts(prec_inner=bsm.F32)) < \
        bsm.bsm_fgcr_workspace_bytes(good, bsm.fgcr_opts())
    # the double-float outer operator: only with FP32 cycles (no FP64 links are passed then), and
    # two full-lattice double-float copies in the workspace
    assert solve(bsm.fgcr_opts(prec_outer=bsm.DF64)) == bsm.EUNSUPPORTED
    assert solve(bsm.fgcr_opts(prec_inner=bsm.F32, prec_outer=bsm.F32)) == bsm.EUNSUPPORTED
    assert solve(bsm.fgcr_opts(prec_inner=bsm.F32, prec_outer=7)) == bsm.EUNSUPPORTED
    assert bsm.bsm_fgcr_workspace_bytes(good, bsm.fgcr_opts(prec_inner=bsm.F32, prec_outer=bsm.DF64)) == \
        bsm.bsm_fgcr_workspace_bytes(good, bsm.fgcr_opts(prec_inner=bsm.F32)) + \
        2 * bsm.bsm_field_bytes(good, bsm.FIELD_SPINOR, bsm.F64)


def test_slab_arguments_are_checked(bsm):
    """time slabs: t0 and nt even, 2 <= nt, t0 + nt <= T, FP64/FP32 only"""
    glat = bsm.lattice((8, 4, 4, 4), 3, bsm.FUND, 0.1)
    A = 1 << 24
    for t0, nt in ((1, 4), (0, 3), (6, 4), (-2, 4), (0, 0)):
        assert bsm._lib.bsm_dslash_slab(bsm.slab(glat, t0, nt), A, 2 * A, 3 * A, 4 * A, 5 * A, 0, 0, bsm.F64,
                                        None) == bsm.EINVAL
        assert bsm._lib.bsm_face_pack(bsm.slab(glat, t0, nt), A, 2 * A, bsm.FACE_LO, 1, 0, bsm.F64,
                                      None) == bsm.EINVAL
        assert bsm.bsm_face_bytes(bsm.slab(glat, t0, nt), bsm.F64) == 0
    ok = bsm.slab(glat, 2, 4)
    assert bsm._lib.bsm_dslash_slab(ok, A, 2 * A, 3 * A, 4 * A, 5 * A, 0, 0, bsm.DF64, None) == bsm.EUNSUPPORTED
    assert bsm._lib.bsm_dslash_slab(ok, A, 2 * A, 3 * A, 4 * A, 5 * A, 2, 0, bsm.F64, None) == bsm.EINVAL
    assert bsm._lib.bsm_face_pack(ok, A, 2 * A, 7, 1, 0, bsm.F64, None) == bsm.EINVAL
    # one face: X Y Z / 2 sites x 2 spins x d colours, complex
    assert bsm.bsm_face_bytes(ok, bsm.F64) == 4 * 4 * 4 // 2 * 2 * 3 * 16
    assert bsm.bsm_face_bytes(ok, bsm.F32) == 4 * 4 * 4 // 2 * 2 * 3 * 8


def test_cg_batch_arguments_are_checked(bsm):
    lat = bsm.lattice((4, 4, 4, 4), 3, bsm.FUND, 0.1)
    A = 1 << 24
    fb = bsm.bsm_field_bytes(lat, bsm.FIELD_SPINOR, bsm.F64)

    def items(nrhs=2, lat_=lat, x=8 * A):
        return bsm.cg_batch_items([(lat_, A, 2 * A, 4 * A, x, nrhs)])

    assert bsm.bsm_cg_batch_workspace_bytes(items()) > 0
    assert bsm.bsm_cg_batch_workspace_bytes(items(nrhs=3)) == 0           # nrhs a power of two <= 16
    assert bsm.bsm_cg_batch_workspace_bytes(items(nrhs=32)) == 0
    assert bsm.bsm_cg_batch_workspace_bytes(items(lat_=bsm.lattice((4, 4, 4, 4), 3, bsm.ADJ, 0.1))) == 0
    assert bsm.bsm_cg_batch_workspace_bytes(items(x=4 * A + fb)) == 0      # b and x overlap
    ws = 16 * A
    opts = bsm.cg_opts(prec_inner=bsm.F32)
    for bad, want in ((bsm.cg_opts(prec_inner=bsm.F64), bsm.EUNSUPPORTED),
                      (bsm.cg_opts(prec_inner=bsm.F32, eo=False), bsm.EUNSUPPORTED),
                      (bsm.cg_opts(prec_inner=bsm.F32, tol=0.0), bsm.EINVAL),
                      (bsm.cg_opts(prec_inner=bsm.F32, prec_outer=bsm.F32), bsm.EUNSUPPORTED)):
        assert bsm._lib.bsm_cg_solve_batch(items(), 1, ctypes.byref(bad), None, ws, 1 << 40, None) == want
    assert bsm._lib.bsm_cg_solve_batch(items(), 1, ctypes.byref(opts), None, ws, 1024, None) == bsm.EWORKSPACE
    assert bsm._lib.bsm_cg_solve_batch(items(), 0, ctypes.byref(opts), None, ws, 1 << 40, None) == bsm.EINVAL
