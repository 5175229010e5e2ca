"""ctypes binding of the C ABI in include/bsm.h (libbsm_gb300.so).

Argument marshalling only: every step of the computation runs in the CUDA
library.  Device buffers are torch tensors (their data_ptr is passed), the
stream defaults to torch's current stream.  Importing this module raises
ImportError when the library has not been built, so there is no silent
fallback.  Function names follow the C entry points.
"""
from __future__ import annotations

import ctypes
import os

import torch

_LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "libbsm_gb300.so")
if not os.path.exists(_LIB_PATH):
    raise ImportError(f"{_LIB_PATH} is missing: build it with `python -c 'import __graft_entry__ as g; g.build()'`")
_lib = ctypes.CDLL(_LIB_PATH)

# enums of bsm.h
OK, EINVAL, EUNSUPPORTED, ECUDA, EWORKSPACE, ENOCONV, EBREAKDOWN, ENAN, ETIMEOUT = 0, -1, -2, -3, -4, -5, -6, -7, -8
FUND, ADJ, SYM, ASYM = 0, 1, 2, 3
F64, F32, DF64, BF16, F32R12 = 0, 1, 2, 3, 4
EVEN, ODD, FULL = 0, 1, 2
OP_DHAT, OP_DHAT_DAG, OP_DHAT_DAG_DHAT = 0, 1, 2
FIELD_LINKS, FIELD_SPINOR, FIELD_HALF_SPINOR, FIELD_FUND_CANON, FIELD_SPINOR_CANON = 0, 1, 2, 3, 4
CALL_DIRAC_EO, CALL_CG = 0, 1


class Lattice(ctypes.Structure):
    _fields_ = [("dims", ctypes.c_int32 * 4), ("N", ctypes.c_int32), ("rep", ctypes.c_int32),
                ("m0", ctypes.c_double), ("bc_phase", ctypes.c_double * 4)]


class CgOpts(ctypes.Structure):
    _fields_ = [("tol", ctypes.c_double), ("max_iter", ctypes.c_int32), ("prec_inner", ctypes.c_int32),
                ("delta", ctypes.c_double), ("use_x0", ctypes.c_int32), ("eo", ctypes.c_int32),
                ("check_every", ctypes.c_int32), ("prec_outer", ctypes.c_int32), ("use_graph", ctypes.c_int32)]


class CgStats(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int32), ("reliable_updates", ctypes.c_int32),
                ("true_res_normal", ctypes.c_double), ("true_res_full", ctypes.c_double),
                ("seconds", ctypes.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class BatchItem(ctypes.Structure):
    _fields_ = [("lat", Lattice), ("U_rep", ctypes.c_void_p), ("in_", ctypes.c_void_p), ("out", ctypes.c_void_p),
                ("nrhs", ctypes.c_int32)]


class BatchOpts(ctypes.Structure):
    _fields_ = [("op", ctypes.c_int32), ("prec", ctypes.c_int32), ("timeout_s", ctypes.c_double),
                ("barrier_extra", ctypes.c_int32)]


BATCH_D, BATCH_DHAT = 0, 1
FGCR_NONE, FGCR_PTC = 0, 1


class FgcrOpts(ctypes.Structure):
    _fields_ = [("tol", ctypes.c_double), ("max_iter", ctypes.c_int32), ("restart", ctypes.c_int32),
                ("precond", ctypes.c_int32), ("ptc_prec", ctypes.c_int32), ("channels", ctypes.c_int32),
                ("prec_inner", ctypes.c_int32), ("inner_tol", ctypes.c_double), ("eo", ctypes.c_int32),
                ("check_every", ctypes.c_int32), ("prec_outer", ctypes.c_int32), ("fallback", ctypes.c_int32),
                ("fallback_max_iter", ctypes.c_int32)]


class FgcrStats(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int32), ("cycles", ctypes.c_int32), ("true_res", ctypes.c_double),
                ("seconds", ctypes.c_double), ("fgcr_status", ctypes.c_int32), ("fallback_iters", ctypes.c_int32)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class Slab(ctypes.Structure):
    _fields_ = [("global_", Lattice), ("t0", ctypes.c_int32), ("nt", ctypes.c_int32)]


FACE_LO, FACE_HI = 0, 1


class CgBatchItem(ctypes.Structure):
    _fields_ = [("lat", Lattice), ("U_rep64", ctypes.c_void_p), ("U_rep32", ctypes.c_void_p), ("b", ctypes.c_void_p),
                ("x", ctypes.c_void_p), ("nrhs", ctypes.c_int32)]


class BsmError(RuntimeError):
    def __init__(self, status: int, what: str):
        msg = f"{what}: {bsm_strerror(status)} ({status})"
        if status == ECUDA:
            msg += f" [{bsm_last_cuda_error()}]"
        super().__init__(msg)
        self.status = status


_P = ctypes.c_void_p
_LP = ctypes.POINTER(Lattice)
_lib.bsm_rep_dim.argtypes = [ctypes.c_int32, ctypes.c_int32]
_lib.bsm_rep_dim.restype = ctypes.c_int
_lib.bsm_field_bytes.argtypes = [_LP, ctypes.c_int32, ctypes.c_int32]
_lib.bsm_field_bytes.restype = ctypes.c_size_t
_lib.bsm_workspace_bytes.argtypes = [_LP, ctypes.c_int32, ctypes.c_int32]
_lib.bsm_workspace_bytes.restype = ctypes.c_size_t
_lib.bsm_pack_spinor.argtypes = [_LP, _P, _P, ctypes.c_int32, _P]
_lib.bsm_unpack_spinor.argtypes = [_LP, _P, _P, ctypes.c_int32, _P]
_lib.bsm_links_to_rep.argtypes = [_LP, _P, _P, ctypes.c_int32, _P]
_lib.bsm_pack_spinor_mrhs.argtypes = [_LP, _P, _P, ctypes.c_int32, ctypes.c_int32, _P]
_lib.bsm_unpack_spinor_mrhs.argtypes = [_LP, _P, _P, ctypes.c_int32, ctypes.c_int32, _P]
_lib.bsm_dslash_mrhs_block.argtypes = [_LP, ctypes.c_int32, ctypes.c_int32]
_lib.bsm_dslash_mrhs_block.restype = ctypes.c_int
_lib.bsm_dslash_mrhs_set_block.argtypes = [_LP, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32]
_lib.bsm_dslash_mrhs_set_block.restype = ctypes.c_int
_lib.bsm_dslash_mrhs.argtypes = [_LP, _P, _P, _P, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, _P]
_lib.bsm_dslash.argtypes = [_LP, _P, _P, _P, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, _P]
_lib.bsm_dirac_eo.argtypes = [_LP, _P, _P, _P, ctypes.c_int32, ctypes.c_int32, _P, ctypes.c_size_t, _P]
_lib.bsm_dirac_eo_noalloc.argtypes = [_LP, _P, _P, _P, ctypes.c_int32, ctypes.c_int32, _P]
_lib.bsm_cg_solve.argtypes = [_LP, _P, _P, _P, _P, ctypes.POINTER(CgOpts), ctypes.POINTER(CgStats), _P,
                              ctypes.c_size_t, _P]
_lib.bsm_batch_workspace_bytes.argtypes = [ctypes.POINTER(BatchItem), ctypes.c_int32, ctypes.POINTER(BatchOpts)]
_lib.bsm_batch_workspace_bytes.restype = ctypes.c_size_t
_lib.bsm_dslash_batch.argtypes = [ctypes.POINTER(BatchItem), ctypes.c_int32, ctypes.POINTER(BatchOpts), _P,
                                  ctypes.c_size_t, _P]
_lib.bsm_dslash_batch.restype = ctypes.c_int
_lib.bsm_dslash_batch_async.argtypes = [ctypes.POINTER(BatchItem), ctypes.c_int32, ctypes.POINTER(BatchOpts), _P,
                                        ctypes.c_size_t, _P]
_lib.bsm_dslash_batch_async.restype = ctypes.c_int
_lib.bsm_dslash_batch_status.argtypes = [_P, _P]
_lib.bsm_dslash_batch_status.restype = ctypes.c_int
_lib.bsm_ptc_pack.argtypes = [_LP, _P, _P, _P]
_lib.bsm_ptc_unpack.argtypes = [_LP, _P, _P, _P]
_lib.bsm_ptc_workspace_bytes.argtypes = [_LP, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32]
_lib.bsm_ptc_workspace_bytes.restype = ctypes.c_size_t
_lib.bsm_ptc_apply.argtypes = [_LP, _P, _P, _P, ctypes.c_int32, _P, _P, ctypes.c_int32, ctypes.c_int32, _P,
                               ctypes.c_size_t, _P]
_lib.bsm_ptc_status.argtypes = [_P, _P]
_lib.bsm_ptc_status.restype = ctypes.c_int
_lib.bsm_ptc_loss_grad.argtypes = [_LP, _P, _P, _P, ctypes.c_int32, _P, _P, ctypes.c_int32, _P, _P,
                                   ctypes.POINTER(ctypes.c_double), _P, ctypes.c_size_t, _P]
_lib.bsm_ptc_adam_step.argtypes = [_P, _P, _P, _P, ctypes.c_int64, ctypes.c_double, ctypes.c_int32, _P]
_lib.bsm_fgcr_workspace_bytes.argtypes = [_LP, ctypes.POINTER(FgcrOpts)]
_lib.bsm_fgcr_workspace_bytes.restype = ctypes.c_size_t
_lib.bsm_fgcr_solve.argtypes = [_LP, _P, _P, _P, _P, _P, _P, ctypes.POINTER(FgcrOpts), ctypes.POINTER(FgcrStats),
                                _P, ctypes.c_size_t, _P]
_lib.bsm_cg_batch_workspace_bytes.argtypes = [ctypes.POINTER(CgBatchItem), ctypes.c_int32]
_lib.bsm_cg_batch_workspace_bytes.restype = ctypes.c_size_t
_lib.bsm_cg_solve_batch.argtypes = [ctypes.POINTER(CgBatchItem), ctypes.c_int32, ctypes.POINTER(CgOpts),
                                    ctypes.POINTER(CgStats), _P, ctypes.c_size_t, _P]
_lib.bsm_cg_solve_batch.restype = ctypes.c_int
_lib.bsm_batch_last_config.argtypes = [ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int32)]
_lib.bsm_batch_last_config.restype = ctypes.c_int
_SP = ctypes.POINTER(Slab)
_lib.bsm_face_bytes.argtypes = [_SP, ctypes.c_int32]
_lib.bsm_face_bytes.restype = ctypes.c_size_t
_lib.bsm_face_pack.argtypes = [_SP, _P, _P, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, _P]
_lib.bsm_face_pack.restype = ctypes.c_int
_lib.bsm_dslash_slab.argtypes = [_SP, _P, _P, _P, _P, _P, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, _P]
_lib.bsm_dslash_slab.restype = ctypes.c_int
_lib.bsm_strerror.argtypes = [ctypes.c_int]
_lib.bsm_strerror.restype = ctypes.c_char_p
_lib.bsm_last_cuda_error.argtypes = []
_lib.bsm_last_cuda_error.restype = ctypes.c_char_p
for _f in ("bsm_pack_spinor", "bsm_unpack_spinor", "bsm_links_to_rep", "bsm_dslash", "bsm_dirac_eo",
           "bsm_dirac_eo_noalloc", "bsm_cg_solve", "bsm_pack_spinor_mrhs", "bsm_unpack_spinor_mrhs",
           "bsm_dslash_mrhs", "bsm_ptc_pack", "bsm_ptc_unpack", "bsm_ptc_apply", "bsm_ptc_loss_grad",
           "bsm_ptc_adam_step", "bsm_fgcr_solve"):
    getattr(_lib, _f).restype = ctypes.c_int


def library_path() -> str:
    return _LIB_PATH


def lattice(dims, N, rep=FUND, m0=0.1, bc_phase=(0.0, 0.0, 0.0, 0.0)) -> Lattice:
    return Lattice((ctypes.c_int32 * 4)(*dims), N, rep, float(m0), (ctypes.c_double * 4)(*bc_phase))


def _ptr(t):
    if t is None:
        return None
    if isinstance(t, int):
        return t
    return t.data_ptr()


def _stream(stream):
    if stream is None:
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, torch.cuda.Stream):
        return stream.cuda_stream
    return stream


def _check(status, what):
    if status != OK:
        raise BsmError(status, what)


def bsm_strerror(status: int) -> str:
    return _lib.bsm_strerror(status).decode()


def bsm_last_cuda_error() -> str:
    return _lib.bsm_last_cuda_error().decode()


def bsm_rep_dim(N: int, rep: int) -> int:
    return _lib.bsm_rep_dim(N, rep)


def bsm_field_bytes(lat: Lattice, kind: int, prec: int = F64) -> int:
    return _lib.bsm_field_bytes(ctypes.byref(lat), kind, prec)


def bsm_workspace_bytes(lat: Lattice, call: int, prec: int) -> int:
    return _lib.bsm_workspace_bytes(ctypes.byref(lat), call, prec)


def empty_field(lat: Lattice, kind: int, prec: int = F64, device="cuda") -> torch.Tensor:
    """Uninitialised byte tensor sized for a field of `kind` (torch device
    allocations are at least 256-byte aligned)."""
    n = bsm_field_bytes(lat, kind, prec)
    if n == 0:
        raise BsmError(EINVAL, "bsm_field_bytes")
    return torch.empty(n, dtype=torch.uint8, device=device)


def bsm_pack_spinor(lat, canon, dev, prec, stream=None):
    _check(_lib.bsm_pack_spinor(ctypes.byref(lat), _ptr(canon), _ptr(dev), prec, _stream(stream)),
           "bsm_pack_spinor")


def bsm_unpack_spinor(lat, dev, canon, prec, stream=None):
    _check(_lib.bsm_unpack_spinor(ctypes.byref(lat), _ptr(dev), _ptr(canon), prec, _stream(stream)),
           "bsm_unpack_spinor")


def bsm_pack_spinor_mrhs(lat, canon, dev, nrhs, prec, stream=None):
    _check(_lib.bsm_pack_spinor_mrhs(ctypes.byref(lat), _ptr(canon), _ptr(dev), nrhs, prec, _stream(stream)),
           "bsm_pack_spinor_mrhs")


def bsm_unpack_spinor_mrhs(lat, dev, canon, nrhs, prec, stream=None):
    _check(_lib.bsm_unpack_spinor_mrhs(ctypes.byref(lat), _ptr(dev), _ptr(canon), nrhs, prec, _stream(stream)),
           "bsm_unpack_spinor_mrhs")


def bsm_dslash_mrhs(lat, U_rep, inp, out, nrhs, out_parity, dagger, prec, stream=None):
    _check(_lib.bsm_dslash_mrhs(ctypes.byref(lat), _ptr(U_rep), _ptr(inp), _ptr(out), nrhs, out_parity, int(dagger),
                                prec, _stream(stream)), "bsm_dslash_mrhs")


def bsm_dslash_mrhs_block(lat, nrhs, prec) -> int:
    return _lib.bsm_dslash_mrhs_block(ctypes.byref(lat), nrhs, prec)


MRHS_TENSOR_CORE_BLOCK = 16


def bsm_dslash_mrhs_set_block(lat, nrhs, prec, block):
    _check(_lib.bsm_dslash_mrhs_set_block(ctypes.byref(lat), nrhs, prec, block), "bsm_dslash_mrhs_set_block")


def bsm_links_to_rep(lat, U_fund, U_rep, prec, stream=None):
    _check(_lib.bsm_links_to_rep(ctypes.byref(lat), _ptr(U_fund), _ptr(U_rep), prec, _stream(stream)),
           "bsm_links_to_rep")


def bsm_dslash(lat, U_rep, inp, out, out_parity, dagger, prec, stream=None):
    _check(_lib.bsm_dslash(ctypes.byref(lat), _ptr(U_rep), _ptr(inp), _ptr(out), out_parity, int(dagger), prec,
                           _stream(stream)), "bsm_dslash")


def bsm_dirac_eo(lat, U_rep, in_e, out_e, op, prec, workspace, stream=None):
    nbytes = workspace.numel() * workspace.element_size() if workspace is not None else 0
    _check(_lib.bsm_dirac_eo(ctypes.byref(lat), _ptr(U_rep), _ptr(in_e), _ptr(out_e), op, prec, _ptr(workspace),
                             nbytes, _stream(stream)), "bsm_dirac_eo")


def bsm_dirac_eo_noalloc(lat, U_rep, in_e, out_e, op, prec, stream=None):
    """bsm_dirac_eo with the library's own fixed scratch array instead of a
    workspace, for callers that cannot allocate device memory."""
    _check(_lib.bsm_dirac_eo_noalloc(ctypes.byref(lat), _ptr(U_rep), _ptr(in_e), _ptr(out_e), op, prec,
                                     _stream(stream)), "bsm_dirac_eo_noalloc")


NOALLOC_SCRATCH_BYTES = 64 << 20


def batch_items(entries):
    """entries: iterable of (lattice, U_rep, in, out, nrhs) -> ctypes array."""
    entries = list(entries)
    arr = (BatchItem * len(entries))()
    for k, (lat, U, i, o, n) in enumerate(entries):
        arr[k] = BatchItem(lat, _ptr(U), _ptr(i), _ptr(o), n)
    return arr


def bsm_batch_workspace_bytes(items, opts: BatchOpts) -> int:
    return _lib.bsm_batch_workspace_bytes(items, len(items), ctypes.byref(opts))


def bsm_dslash_batch(items, opts: BatchOpts, workspace, stream=None, raise_on_error=True) -> int:
    nbytes = workspace.numel() * workspace.element_size() if workspace is not None else 0
    st = _lib.bsm_dslash_batch(items, len(items), ctypes.byref(opts), _ptr(workspace), nbytes, _stream(stream))
    if raise_on_error:
        _check(st, "bsm_dslash_batch")
    return st


def bsm_dslash_batch_async(items, opts: BatchOpts, workspace, stream=None) -> int:
    nbytes = workspace.numel() * workspace.element_size()
    st = _lib.bsm_dslash_batch_async(items, len(items), ctypes.byref(opts), _ptr(workspace), nbytes,
                                     _stream(stream))
    _check(st, "bsm_dslash_batch_async")
    return st


def bsm_dslash_batch_status(workspace, stream=None) -> int:
    return _lib.bsm_dslash_batch_status(_ptr(workspace), _stream(stream))


def bsm_cg_solve(lat, U_rep64, U_rep32, b, x, opts: CgOpts, workspace, stream=None, raise_on_error=True):
    """Returns (status, CgStats); raises BsmError on a nonzero status unless
    raise_on_error is False."""
    stats = CgStats()
    nbytes = workspace.numel() * workspace.element_size() if workspace is not None else 0
    st = _lib.bsm_cg_solve(ctypes.byref(lat), _ptr(U_rep64), _ptr(U_rep32), _ptr(b), _ptr(x), ctypes.byref(opts),
                           ctypes.byref(stats), _ptr(workspace), nbytes, _stream(stream))
    if raise_on_error:
        _check(st, "bsm_cg_solve")
    return st, stats


def cg_opts(tol=1e-10, max_iter=10000, prec_inner=F64, delta=0.1, use_x0=False, eo=True, check_every=8,
            prec_outer=F64, use_graph=False) -> CgOpts:
    return CgOpts(tol, max_iter, prec_inner, delta, int(use_x0), int(eo), check_every, prec_outer, int(use_graph))


# --- learned preconditioner (parallel-transport convolutions) and FGCR -------

def ptc_shapes(channels: int):
    """Shapes (complex entries) of W1 and W2 for `channels` hidden channels."""
    return (36, 4 * channels), (36 * channels, 4)


def bsm_ptc_pack(lat, psi, field, stream=None):
    _check(_lib.bsm_ptc_pack(ctypes.byref(lat), _ptr(psi), _ptr(field), _stream(stream)), "bsm_ptc_pack")


def bsm_ptc_unpack(lat, field, psi, stream=None):
    _check(_lib.bsm_ptc_unpack(ctypes.byref(lat), _ptr(field), _ptr(psi), _stream(stream)), "bsm_ptc_unpack")


def bsm_ptc_workspace_bytes(lat, channels, nbatch, train) -> int:
    return _lib.bsm_ptc_workspace_bytes(ctypes.byref(lat), channels, nbatch, int(train))


def bsm_ptc_apply(lat, U_rep32, W1, W2, channels, inp, out, nbatch, prec, workspace, stream=None):
    nbytes = workspace.numel() * workspace.element_size()
    _check(_lib.bsm_ptc_apply(ctypes.byref(lat), _ptr(U_rep32), _ptr(W1), _ptr(W2), channels, _ptr(inp), _ptr(out),
                              nbatch, prec, _ptr(workspace), nbytes, _stream(stream)), "bsm_ptc_apply")


def bsm_ptc_status(workspace, stream=None) -> int:
    return _lib.bsm_ptc_status(_ptr(workspace), _stream(stream))


def bsm_ptc_loss_grad(lat, U_rep32, W1, W2, channels, r, e, nbatch, G_W1, G_W2, workspace, stream=None) -> float:
    loss = ctypes.c_double(0.0)
    nbytes = workspace.numel() * workspace.element_size()
    _check(_lib.bsm_ptc_loss_grad(ctypes.byref(lat), _ptr(U_rep32), _ptr(W1), _ptr(W2), channels, _ptr(r), _ptr(e),
                                  nbatch, _ptr(G_W1), _ptr(G_W2), ctypes.byref(loss), _ptr(workspace), nbytes,
                                  _stream(stream)), "bsm_ptc_loss_grad")
    return loss.value


def bsm_ptc_adam_step(W, G, m, v, lr, step, stream=None):
    n = W.numel() * W.element_size() // 4
    _check(_lib.bsm_ptc_adam_step(_ptr(W), _ptr(G), _ptr(m), _ptr(v), n, float(lr), step, _stream(stream)),
           "bsm_ptc_adam_step")


def fgcr_opts(tol=1e-10, max_iter=1000, restart=16, precond=FGCR_NONE, ptc_prec=F32, channels=1, prec_inner=F64,
              inner_tol=0.0, eo=False, check_every=1, prec_outer=F64, fallback=False, fallback_max_iter=0) -> FgcrOpts:
    return FgcrOpts(tol, max_iter, restart, precond, ptc_prec, channels, prec_inner, inner_tol, int(eo), check_every,
                    prec_outer, int(fallback), fallback_max_iter)


def bsm_fgcr_workspace_bytes(lat, opts: FgcrOpts) -> int:
    return _lib.bsm_fgcr_workspace_bytes(ctypes.byref(lat), ctypes.byref(opts))


def bsm_fgcr_solve(lat, U_rep64, U_rep32, W1, W2, b, x, opts: FgcrOpts, workspace, stream=None,
                   raise_on_error=True):
    """Returns (status, FgcrStats)."""
    stats = FgcrStats()
    nbytes = workspace.numel() * workspace.element_size() if workspace is not None else 0
    st = _lib.bsm_fgcr_solve(ctypes.byref(lat), _ptr(U_rep64), _ptr(U_rep32), _ptr(W1), _ptr(W2), _ptr(b), _ptr(x),
                             ctypes.byref(opts), ctypes.byref(stats), _ptr(workspace), nbytes, _stream(stream))
    if raise_on_error:
        _check(st, "bsm_fgcr_solve")
    return st, stats


def slab(global_lat, t0, nt) -> Slab:
    return Slab(global_lat, t0, nt)


def bsm_face_bytes(sl, prec) -> int:
    return _lib.bsm_face_bytes(ctypes.byref(sl), prec)


def bsm_face_pack(sl, in_slab, face, side, in_parity, dagger, prec, stream=None):
    _check(_lib.bsm_face_pack(ctypes.byref(sl), _ptr(in_slab), _ptr(face), side, in_parity, int(dagger), prec,
                              _stream(stream)), "bsm_face_pack")


def bsm_dslash_slab(sl, U_rep, in_slab, face_lo, face_hi, out_slab, out_parity, dagger, prec, stream=None):
    _check(_lib.bsm_dslash_slab(ctypes.byref(sl), _ptr(U_rep), _ptr(in_slab), _ptr(face_lo), _ptr(face_hi),
                                _ptr(out_slab), out_parity, int(dagger), prec, _stream(stream)), "bsm_dslash_slab")


def cg_batch_items(entries):
    """entries: (lattice, U_rep64, U_rep32, b, x, nrhs) tuples -> ctypes array
    (b, x: nrhs FP64 full spinors one after the other, as one tensor each)"""
    arr = (CgBatchItem * len(entries))()
    for k, (lat, U64, U32, b, x, n) in enumerate(entries):
        arr[k] = CgBatchItem(lat, _ptr(U64), _ptr(U32), _ptr(b), _ptr(x), n)
    return arr


def bsm_cg_batch_workspace_bytes(items) -> int:
    return _lib.bsm_cg_batch_workspace_bytes(items, len(items))


def bsm_cg_solve_batch(items, opts: CgOpts, workspace, stream=None, raise_on_error=True):
    """Returns (status, [CgStats per system])."""
    nsys = sum(it.nrhs for it in items)
    stats = (CgStats * nsys)()
    nbytes = workspace.numel() * workspace.element_size() if workspace is not None else 0
    st = _lib.bsm_cg_solve_batch(items, len(items), ctypes.byref(opts), stats, _ptr(workspace), nbytes,
                                 _stream(stream))
    if raise_on_error:
        _check(st, "bsm_cg_solve_batch")
    return st, list(stats)


def bsm_batch_last_config():
    """(RHS per thread, chunks per work-queue grab) of the last batch call on this thread."""
    rb, grab = ctypes.c_int32(), ctypes.c_int32()
    _check(_lib.bsm_batch_last_config(ctypes.byref(rb), ctypes.byref(grab)), "bsm_batch_last_config")
    return rb.value, grab.value
