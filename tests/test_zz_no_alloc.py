"""bsm_dirac_eo_noalloc: the allocation-free entry point for callers that
cannot allocate device memory themselves (their device memory belongs to
another allocator, or their environment offers no allocation call).  Its
result must equal bsm_dirac_eo's, computed with a caller workspace, on two
calls in a row (the second one reuses the library's scratch array as the
first call left it).  Kept in a file that pytest collects last."""
import ctypes

import numpy as np
import pytest
import torch

from paper_1401_3733_gb300 import bsm, fields
from tests.gpu_helpers import TOL, gpu_links, gpu_spinor, half, rel, to_canon, zeros_field

pytestmark = pytest.mark.gpu


def reference(lat, U, inp_e, op, prec):
    ws = torch.empty(bsm.bsm_workspace_bytes(lat, bsm.CALL_DIRAC_EO, prec), dtype=torch.uint8, device="cuda")
    out = zeros_field(lat, bsm.FIELD_SPINOR, prec)
    bsm.bsm_dirac_eo(lat, U, inp_e, half(lat, out, 0, prec), op, prec, ws)
    return to_canon(lat, out, prec)


@pytest.mark.parametrize("prec", [bsm.F64, bsm.F32], ids=["f64", "f32"])
def test_noalloc_matches_dirac_eo_on_consecutive_calls(prec):
    dims = (8, 8, 6, 8)
    lat = bsm.lattice(dims, 3, bsm.FUND, 0.05, (np.pi, 0, 0, 0))
    U = gpu_links(lat, fields.gauge_field(dims, 3, "smooth", seed=7, eps=0.3), prec)
    calls = [(bsm.OP_DHAT_DAG_DHAT, 71), (bsm.OP_DHAT, 72), (bsm.OP_DHAT_DAG, 73)]
    for op, seed in calls:   # consecutive calls share the scratch array
        psi = fields.gaussian_spinor(dims, 3, seed)
        inp = gpu_spinor(lat, psi, prec)
        out = zeros_field(lat, bsm.FIELD_SPINOR, prec)
        bsm.bsm_dirac_eo_noalloc(lat, U, half(lat, inp, 0, prec), half(lat, out, 0, prec), op, prec)
        got = to_canon(lat, out, prec)
        want = reference(lat, U, half(lat, inp, 0, prec), op, prec)
        assert rel(got, want) <= TOL[prec], (op, rel(got, want))


def test_noalloc_rejects_lattices_beyond_the_scratch_array():
    # 2 half spinors of a 32^4 SU(3) FP64 field need 2 * 100 MiB > 64 MiB;
    # the check happens on the host, before any launch
    lat = bsm.lattice((32, 32, 32, 32), 3, bsm.FUND, 0.1)
    need = 2 * bsm.bsm_field_bytes(lat, bsm.FIELD_HALF_SPINOR, bsm.F64)
    assert need > bsm.NOALLOC_SCRATCH_BYTES
    A = 1 << 24
    st = bsm._lib.bsm_dirac_eo_noalloc(ctypes.byref(lat), A, 2 * A, 3 * A, bsm.OP_DHAT, bsm.F64, None)
    assert st == bsm.EWORKSPACE
