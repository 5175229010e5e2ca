"""The halo seam of the time-slab decomposition (Sec. II-C), on the CPU with
gloo ranks: each rank owns a slab of time slices of the global lattice, sends
the spin projections of its two boundary slices to its neighbours -- the
face, 2 spin x d colour complex per site: the upper half h of (1 + s g_0) psi,
whose lower half is s h in the chiral basis -- and receives theirs, together
with the links of the slice below it.  It then applies the oracle's hop to its
slab extended by one ghost slice on each side, a ghost holding the spinor
(h, s h) / 2 rebuilt from a received face (the oracle's (1 + s g_0) of it is
the sender's projection exactly) times the boundary phase when the face
crossed the lattice's time boundary.  The slabs gathered from all ranks must
equal the oracle's hop on the whole lattice, for both parities of the output
and its adjoint."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _face(psi_slice, s, gamma0):
    """upper half of (1 + s g_0) psi on one slice (sites, 4, d) -> (sites, 2, d)"""
    P = np.eye(4) + s * gamma0
    full = np.einsum("ij,njc->nic", P, psi_slice)
    assert np.allclose(full[:, 2:], s * full[:, :2], rtol=0, atol=1e-13)   # chiral basis: lower = s * upper
    return np.ascontiguousarray(full[:, :2])


def _ghost(face, s):
    return np.concatenate([face, s * face], axis=1) / 2


def _exchange(arr, to_rank, from_rank, rank):
    """send arr to to_rank, receive an array of the same shape from from_rank"""
    out = torch.empty_like(torch.from_numpy(arr))
    src = torch.from_numpy(np.ascontiguousarray(arr))
    if rank % 2 == 0:
        dist.send(src, to_rank)
        dist.recv(out, from_rank)
    else:
        dist.recv(out, from_rank)
        dist.send(src, to_rank)
    return out.numpy()


def _worker(rank, world, port, dims, N, rep, m0, phase, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import oracle as orc
    from paper_1401_3733_gb300 import fields

    T, X, Y, Z = dims
    nt, S = T // world, X * Y * Z
    t0 = rank * nt
    d = orc.rep_dim(N, rep)
    # every rank draws the global fields from the same seeds and keeps its slab
    U = fields.gauge_field(dims, N, "haar", seed=41).reshape(T, S, 4, N, N)[t0:t0 + nt]
    psi = fields.gaussian_spinor(dims, d, 42).reshape(T, S, 4, d)[t0:t0 + nt]
    up, down = (rank + 1) % world, (rank - 1) % world
    g0 = orc.gamma(0)
    ext = (nt + 2, X, Y, Z)
    elat = orc.Lattice(ext, N, rep, m0, (0.0,) + tuple(phase[1:]))   # the time phase travels with the faces
    # links of the slice below the slab (the backward time links of slice t0)
    U_below = _exchange(np.ascontiguousarray(U[nt - 1]), up, down, rank)
    U_ext = np.concatenate([U_below[None], U, np.broadcast_to(np.eye(N), (1, S, 4, N, N))], axis=0)
    R_ext = orc.links_to_rep(elat, U_ext.reshape(-1, 4, N, N))
    results = {}
    for dagger in (False, True):
        sf = 1.0 if dagger else -1.0           # sign of (1 + s g_0) in a forward term; backward: -sf
        # faces: the first slice goes down (forward term there), the last one up (backward term there)
        from_up = _exchange(_face(psi[0], sf, g0), down, up, rank)
        from_down = _exchange(_face(psi[nt - 1], -sf, g0), up, down, rank)
        ph = np.exp(1j * phase[0])
        lo = _ghost(from_down, -sf) * (np.conj(ph) if rank == 0 else 1.0)          # crossed t = T-1 -> 0 backwards
        hi = _ghost(from_up, sf) * (ph if rank == world - 1 else 1.0)              # crossed t = T-1 -> 0 forwards
        psi_ext = np.concatenate([lo[None], psi, hi[None]], axis=0).reshape(-1, 4, d)
        h = orc.hop(elat, R_ext, psi_ext, orc.FULL, dagger=dagger).reshape(nt + 2, S, 4, d)[1:nt + 1]
        results[dagger] = h.copy()
    out[rank] = results
    dist.destroy_process_group()


@pytest.mark.parametrize("world,dims,N,rep,phase", [
    (2, (8, 4, 4, 4), 3, 0, (np.pi, 0.0, 0.0, 0.0)),
    (3, (12, 4, 2, 4), 2, 0, (0.7, 0.3, 0.0, -1.1)),
    (2, (4, 2, 4, 2), 2, 1, (np.pi, 0.0, np.pi, 0.0)),
], ids=["2ranks-SU3F", "3ranks-SU2F-twisted", "2ranks-SU2adj-L2slabs"])
def test_slab_hop_with_exchanged_faces_equals_the_global_hop(world, dims, N, rep, phase):
    import oracle as orc
    from paper_1401_3733_gb300 import fields

    m0 = 0.1
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_worker, args=(world, port, dims, N, rep, m0, phase, out), nprocs=world, join=True)
        res = {r: out[r] for r in range(world)}
    lat = orc.Lattice(dims, N, rep, m0, phase)
    R = orc.links_to_rep(lat, fields.gauge_field(dims, N, "haar", seed=41))
    psi = fields.gaussian_spinor(dims, lat.d, 42)
    T, S = dims[0], int(np.prod(dims[1:]))
    for dagger in (False, True):
        want = orc.hop(lat, R, psi, orc.FULL, dagger=dagger).reshape(T, S, 4, lat.d)
        got = np.concatenate([res[r][dagger] for r in range(world)], axis=0)
        err = np.linalg.norm(got - want) / np.linalg.norm(want)
        assert err <= 1e-14, (dagger, err)
