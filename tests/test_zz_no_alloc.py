"""bsm_dirac_eo_noalloc: the allocation-free entry point for callers that
cannot allocate device memory themselves (their device memory belongs to
another allocator, or their environment offers no allocation call).  Its
result must equal bsm_dirac_eo's, computed with a caller workspace, and the
oracle's Schur operator, on consecutive calls (each reuses the library's
scratch array as the previous call left it), and calls after the first must
reserve no device memory.  Kept in a file that pytest collects last."""
import ctypes

import numpy as np
import pytest
import torch

import oracle as orc
from paper_1401_3733_gb300 import bsm, fields
from tests.gpu_helpers import TOL, gpu_links, gpu_spinor, half, rel, to_canon, zeros_field

pytestmark = pytest.mark.gpu

DIMS = (8, 8, 6, 8)
PHASE = (np.pi, 0, 0, 0)
OPS = {bsm.OP_DHAT: "dhat", bsm.OP_DHAT_DAG: "dhat_dag", bsm.OP_DHAT_DAG_DHAT: "dhat_dag_dhat"}


def with_workspace(lat, U, inp_e, op, prec):
    ws = torch.empty(bsm.bsm_workspace_bytes(lat, bsm.CALL_DIRAC_EO, prec), dtype=torch.uint8, device="cuda")
    out = zeros_field(lat, bsm.FIELD_SPINOR, prec)
    bsm.bsm_dirac_eo(lat, U, inp_e, half(lat, out, 0, prec), op, prec, ws)
    return to_canon(lat, out, prec)


@pytest.mark.parametrize("prec", [bsm.F64, bsm.F32, bsm.DF64, bsm.F32R12], ids=["f64", "f32", "df64", "f32r12"])
def test_noalloc_matches_dirac_eo_and_oracle_on_consecutive_calls(prec):
    lat = bsm.lattice(DIMS, 3, bsm.FUND, 0.05, PHASE)
    olat = orc.Lattice(DIMS, 3, orc.FUND, 0.05, PHASE)
    Uc = fields.gauge_field(DIMS, 3, "smooth", seed=7, eps=0.3)
    R = orc.links_to_rep(olat, Uc)
    U = gpu_links(lat, Uc, prec)
    for op, seed in [(bsm.OP_DHAT_DAG_DHAT, 71), (bsm.OP_DHAT, 72), (bsm.OP_DHAT_DAG, 73), (bsm.OP_DHAT, 74)]:
        psi = fields.gaussian_spinor(DIMS, 3, seed)
        inp = gpu_spinor(lat, psi, prec)
        out = zeros_field(lat, bsm.FIELD_SPINOR, prec)
        bsm.bsm_dirac_eo_noalloc(lat, U, half(lat, inp, 0, prec), half(lat, out, 0, prec), op, prec)
        got = to_canon(lat, out, prec)
        want = with_workspace(lat, U, half(lat, inp, 0, prec), op, prec)
        assert rel(got, want) <= TOL[prec], (OPS[op], rel(got, want))
        ref = orc.dhat(olat, R, psi, op)   # the oracle's Schur operator on the even sites
        assert rel(got, ref) <= TOL[prec], (OPS[op], rel(got, ref))


def test_noalloc_calls_after_the_first_reserve_no_device_memory():
    prec = bsm.F32
    lat = bsm.lattice(DIMS, 3, bsm.FUND, 0.05, PHASE)
    U = gpu_links(lat, fields.gauge_field(DIMS, 3, "smooth", seed=7, eps=0.3), prec)
    inp = gpu_spinor(lat, fields.gaussian_spinor(DIMS, 3, 75), prec)
    out = zeros_field(lat, bsm.FIELD_SPINOR, prec)
    args = (lat, U, half(lat, inp, 0, prec), half(lat, out, 0, prec), bsm.OP_DHAT_DAG_DHAT, prec)
    bsm.bsm_dirac_eo_noalloc(*args)   # the first call on the device may load the module
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    alloc0 = torch.cuda.memory_allocated()
    for _ in range(5):
        bsm.bsm_dirac_eo_noalloc(*args)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert torch.cuda.memory_allocated() == alloc0
    assert abs(free1 - free0) <= (2 << 20), (free0, free1)   # driver bookkeeping only


def test_noalloc_rejects_lattices_beyond_the_scratch_array():
    # 2 half spinors of a 32^4 SU(3) FP64 field need 2 * 100 MiB > 64 MiB;
    # the check happens on the host, before any launch
    lat = bsm.lattice((32, 32, 32, 32), 3, bsm.FUND, 0.1)
    need = 2 * bsm.bsm_field_bytes(lat, bsm.FIELD_HALF_SPINOR, bsm.F64)
    assert need > bsm.NOALLOC_SCRATCH_BYTES
    A = 1 << 24
    st = bsm._lib.bsm_dirac_eo_noalloc(ctypes.byref(lat), A, 2 * A, 3 * A, bsm.OP_DHAT, bsm.F64, None)
    assert st == bsm.EWORKSPACE
