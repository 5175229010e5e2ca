"""Helpers shared by the GPU tests: move canonical numpy fields to the device
through the C ABI (pack, links_to_rep) and back (unpack), and compare."""
import numpy as np
import torch

from paper_1401_3733_gb300 import bsm

REP_CASES = [(2, bsm.FUND), (3, bsm.FUND), (4, bsm.FUND), (6, bsm.FUND), (8, bsm.FUND),
             (2, bsm.ADJ), (3, bsm.ADJ), (2, bsm.SYM), (3, bsm.SYM), (3, bsm.ASYM), (4, bsm.ASYM)]
REP_IDS = [f"SU{N}-{['F', 'ADJ', 'S', 'AS'][r]}" for N, r in REP_CASES]
# Relative L2 bars for the Dslash against the FP64 oracle.  BF16 keeps 8
# significand bits: each stored link and spinor value carries a relative
# rounding error of at most 2^-9 (rms about 2^-9/sqrt(3)), so an output
# summed from many such products sits near 3e-3; the bar allows 3x that.
# F32R12 rebuilds each link's third row from the stored two in FP32 (a few
# roundings more per link than F32), so it gets a slightly wider FP32 bar.
TOL = {bsm.F64: 1e-13, bsm.F32: 2e-6, bsm.DF64: 1e-13, bsm.BF16: 1e-2, bsm.F32R12: 2e-6}


def rel(a, b):
    return float(np.linalg.norm((a - b).reshape(-1)) / np.linalg.norm(b.reshape(-1)))


def dev_c128(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.complex128)).to("cuda")


def gpu_links(lat, U, prec):
    out = bsm.empty_field(lat, bsm.FIELD_LINKS, prec)
    bsm.bsm_links_to_rep(lat, dev_c128(U), out, prec)
    return out


def gpu_spinor(lat, psi, prec):
    out = bsm.empty_field(lat, bsm.FIELD_SPINOR, prec)
    bsm.bsm_pack_spinor(lat, dev_c128(psi), out, prec)
    return out


def to_canon(lat, dev, prec):
    V = int(np.prod(list(lat.dims)))
    d = bsm.bsm_rep_dim(lat.N, lat.rep)
    c = torch.empty((V, 4, d), dtype=torch.complex128, device="cuda")
    bsm.bsm_unpack_spinor(lat, dev, c, prec)
    torch.cuda.synchronize()
    return c.cpu().numpy()


def half(lat, field, parity, prec):
    n = bsm.bsm_field_bytes(lat, bsm.FIELD_HALF_SPINOR, prec)
    return field[parity * n:(parity + 1) * n]


def zeros_field(lat, kind, prec):
    t = bsm.empty_field(lat, kind, prec)
    t.zero_()
    return t
