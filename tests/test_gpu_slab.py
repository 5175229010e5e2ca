"""The time-slab decomposition of the hop on one GPU (Sec. II-C): the global
lattice is cut into slabs of time slices held in separate buffers of this
GPU's memory; each slab packs its two boundary faces (bsm_face_pack), the
faces are handed to the neighbouring slabs as a multi-GPU run would send
them, and each slab applies bsm_dslash_slab.  The slabs' outputs together
must equal the oracle's hop on the whole lattice, element by element."""
import numpy as np
import pytest
import torch

import oracle as orc
from paper_1401_3733_gb300 import bsm, fields
from tests.gpu_helpers import TOL, dev_c128, gpu_links, rel

pytestmark = pytest.mark.gpu

CASES = [
    ((8, 4, 4, 4), 3, bsm.FUND, (np.pi, 0.0, 0.0, 0.0), 2),
    ((12, 4, 2, 6), 2, bsm.FUND, (0.7, 0.3, 0.0, -1.1), 3),
    ((8, 2, 4, 2), 3, bsm.FUND, (np.pi, 0.0, 0.0, 0.0), 4),
    ((4, 4, 4, 2), 2, bsm.ADJ, (np.pi, 0.0, np.pi, 0.0), 2),
    ((6, 4, 2, 4), 4, bsm.ASYM, (0.0, 0.0, 0.0, 0.0), 3),
    ((16, 8, 8, 8), 3, bsm.FUND, (np.pi, 0.0, 0.0, 0.0), 2),
]
IDS = ["SU3F-2slabs", "SU2F-3slabs-twisted", "SU3F-4slabs-L2", "SU2adj-2slabs", "SU4AS-3slabs", "SU3F-16c8"]


def slab_hop(glat, links, psi, nslab, out_parity, dagger, prec):
    """the hop of parity out_parity through nslab slabs: canonical (V, 4, d) -> canonical"""
    T, X, Y, Z = glat.dims[:]
    S, d = X * Y * Z, bsm.bsm_rep_dim(glat.N, glat.rep)
    nt = T // nslab
    q = 1 - out_parity
    slabs, ins, outs, lat_s = [], [], [], []
    for k in range(nslab):
        sl = bsm.slab(glat, k * nt, nt)
        loc = bsm.lattice((nt, X, Y, Z), glat.N, glat.rep, glat.m0, tuple(glat.bc_phase))
        full = bsm.empty_field(loc, bsm.FIELD_SPINOR, prec)
        part = psi.reshape(T, S, 4, d)[k * nt:(k + 1) * nt].reshape(-1, 4, d)
        bsm.bsm_pack_spinor(loc, dev_c128(part), full, prec)
        nh = bsm.bsm_field_bytes(loc, bsm.FIELD_HALF_SPINOR, prec)
        slabs.append(sl)
        lat_s.append(loc)
        ins.append(full[q * nh:(q + 1) * nh])
        outs.append(torch.zeros_like(full))
    nf = bsm.bsm_face_bytes(slabs[0], prec)
    lo = [torch.empty(nf, dtype=torch.uint8, device="cuda") for _ in range(nslab)]
    hi = [torch.empty(nf, dtype=torch.uint8, device="cuda") for _ in range(nslab)]
    for k in range(nslab):
        bsm.bsm_face_pack(slabs[k], ins[k], lo[k], bsm.FACE_LO, q, dagger, prec)
        bsm.bsm_face_pack(slabs[k], ins[k], hi[k], bsm.FACE_HI, q, dagger, prec)
    # the exchange: a copy of each face into a buffer of its receiver
    recv_lo = [hi[(k - 1) % nslab].clone() for k in range(nslab)]
    recv_hi = [lo[(k + 1) % nslab].clone() for k in range(nslab)]
    res = []
    for k in range(nslab):
        nh = bsm.bsm_field_bytes(lat_s[k], bsm.FIELD_HALF_SPINOR, prec)
        bsm.bsm_dslash_slab(slabs[k], links, ins[k], recv_lo[k], recv_hi[k],
                            outs[k][out_parity * nh:(out_parity + 1) * nh], out_parity, dagger, prec)
        c = torch.empty((lat_s[k].dims[0] * S, 4, d), dtype=torch.complex128, device="cuda")
        bsm.bsm_unpack_spinor(lat_s[k], outs[k], c, prec)
        res.append(c)
    torch.cuda.synchronize()
    return torch.cat(res).cpu().numpy()


@pytest.mark.parametrize("prec", [bsm.F64, bsm.F32], ids=["f64", "f32"])
@pytest.mark.parametrize("dims,N,rep,phase,nslab", CASES, ids=IDS)
def test_slabs_with_exchanged_faces_equal_the_global_hop(dims, N, rep, phase, nslab, prec):
    olat = orc.Lattice(dims, N, rep, 0.1, phase)
    glat = bsm.lattice(dims, N, rep, 0.1, phase)
    U = fields.gauge_field(dims, N, "haar", seed=51)
    R = orc.links_to_rep(olat, U)
    psi = fields.gaussian_spinor(dims, olat.d, 52)
    links = gpu_links(glat, U, prec)
    odd = orc.parity_mask(dims)
    for p in (bsm.EVEN, bsm.ODD):
        for dagger in (0, 1):
            got = slab_hop(glat, links, psi, nslab, p, dagger, prec)
            want = orc.hop(olat, R, psi, orc.EVEN if p == bsm.EVEN else orc.ODD, dagger=bool(dagger))
            sel = odd if p == bsm.ODD else ~odd
            assert rel(got[sel], want[sel]) <= TOL[prec], (p, dagger, rel(got[sel], want[sel]))
            assert float(np.abs(got[~sel]).max()) == 0.0


def test_one_slab_is_the_periodic_lattice():
    """nt = T: the slab's faces go to itself, and the result is bsm_dslash's."""
    dims, N = (4, 4, 4, 4), 3
    olat = orc.Lattice(dims, N, bsm.FUND, 0.1, (np.pi, 0, 0, 0))
    glat = bsm.lattice(dims, N, bsm.FUND, 0.1, (np.pi, 0, 0, 0))
    U = fields.gauge_field(dims, N, "haar", seed=53)
    psi = fields.gaussian_spinor(dims, N, 54)
    got = slab_hop(glat, gpu_links(glat, U, bsm.F64), psi, 1, bsm.EVEN, 0, bsm.F64)
    want = orc.hop(olat, orc.links_to_rep(olat, U), psi, orc.EVEN)
    assert rel(got, want) <= 1e-13

