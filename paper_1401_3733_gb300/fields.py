"""Seeded synthetic inputs: gauge links and fermion sources.

The paper benchmarks on "randomly-generated fields" (Sec. III); this module
makes them reproducibly.  It is shared by the tests, the smoke check and the
benchmark, and feeds the CUDA path and the CPU oracle alike.  It holds none
of the method's arithmetic (no representation map, no Dirac operator, no
solver): it only draws random numbers and shapes them into SU(N) matrices
and Gaussian spinors in the canonical host layout

    links    U[site, mu, a, b]        complex128, (V, 4, N, N)
    spinors  psi[site, spin, colour]  complex128, (V, 4, d)

with site = ((t*X + x)*Y + y)*Z + z and dims = (T, X, Y, Z).

Random numbers: SplitMix64 (Steele, Lea, Flood 2014) used as a counter-based
generator, value i of stream `seed` being mix64(key(seed) + (i+1)*golden);
53-bit uniforms; Box-Muller (1958) Gaussians.  Consumption order is the
row-major order of the output arrays (site, mu, row, column, re/im).
"""
from __future__ import annotations

import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def _mix64(z: np.ndarray) -> np.ndarray:
    z = (z ^ (z >> np.uint64(30))) * _M1
    z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


def splitmix64(seed: int, n: int, offset: int = 0) -> np.ndarray:
    """n 64-bit words of stream `seed`, starting at counter `offset`."""
    with np.errstate(over="ignore"):
        key = _mix64(np.array([np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + _GOLDEN], np.uint64))[0]
        ctr = np.arange(offset + 1, offset + n + 1, dtype=np.uint64)
        return _mix64(key + ctr * _GOLDEN)


def uniforms(seed: int, n: int, offset: int = 0) -> np.ndarray:
    """n doubles uniform in [0, 1) with 53 random bits."""
    return (splitmix64(seed, n, offset) >> np.uint64(11)).astype(np.float64) * 2.0 ** -53


def gaussians(seed: int, n: int) -> np.ndarray:
    """n independent N(0, 1) doubles (Box-Muller on consecutive word pairs)."""
    m = (n + 1) // 2
    w = splitmix64(seed, 2 * m).reshape(m, 2) >> np.uint64(11)
    u1 = (w[:, 0].astype(np.float64) + 1.0) * 2.0 ** -53   # (0, 1]
    u2 = w[:, 1].astype(np.float64) * 2.0 ** -53           # [0, 1)
    rad = np.sqrt(-2.0 * np.log(u1))
    out = np.empty((m, 2))
    out[:, 0] = rad * np.cos(2.0 * np.pi * u2)
    out[:, 1] = rad * np.sin(2.0 * np.pi * u2)
    return out.reshape(-1)[:n]


def complex_gaussians(seed: int, shape) -> np.ndarray:
    """Complex array whose real and imaginary parts are independent N(0,1)."""
    n = int(np.prod(shape))
    g = gaussians(seed, 2 * n).reshape(n, 2)
    return (g[:, 0] + 1j * g[:, 1]).reshape(shape)


def haar_su(seed: int, count: int, N: int) -> np.ndarray:
    """count Haar-random SU(N) matrices: QR of a complex Ginibre matrix with
    the phases of R's diagonal moved into Q (Mezzadri 2007), then divided by
    det^(1/N) (principal branch) to land in SU(N)."""
    Z = complex_gaussians(seed, (count, N, N)) / np.sqrt(2.0)
    Q, R = np.linalg.qr(Z)
    diag = np.diagonal(R, axis1=1, axis2=2)
    Q = Q * (diag / np.abs(diag))[:, None, :]
    det = np.linalg.det(Q)
    return Q / (det ** (1.0 / N))[:, None, None]


def traceless_hermitian(seed: int, count: int, N: int) -> np.ndarray:
    """count Gaussian traceless Hermitian matrices H = sum_a h_a T^a with
    h_a ~ N(0,1) over the generalised Gell-Mann generators (Tr T^a T^b =
    delta/2): H_ij = (h_s - i h_a)/2 above the diagonal and the Cartan part
    sum_l h_l diag(1,..,1,-l,0,..)/sqrt(2 l (l+1)) on it."""
    noff = N * (N - 1) // 2
    h = gaussians(seed, count * (N * N - 1)).reshape(count, N * N - 1)
    H = np.zeros((count, N, N), np.complex128)
    k = 0
    for i in range(N):
        for j in range(i + 1, N):
            H[:, i, j] = 0.5 * (h[:, k] - 1j * h[:, noff + k])
            H[:, j, i] = np.conj(H[:, i, j])
            k += 1
    for l in range(1, N):
        c = h[:, 2 * noff + l - 1] / np.sqrt(2.0 * l * (l + 1))
        for i in range(l):
            H[:, i, i] += c
        H[:, l, l] -= l * c
    return H


def smooth_su(seed: int, count: int, N: int, eps: float, chunk: int = 1 << 20) -> np.ndarray:
    """count SU(N) matrices U = exp(i eps H), H from traceless_hermitian."""
    import torch  # matrix exponential only; CPU, complex128

    H = traceless_hermitian(seed, count, N)
    out = np.empty_like(H)
    for s in range(0, count, chunk):
        h = torch.from_numpy(H[s:s + chunk])
        out[s:s + chunk] = torch.linalg.matrix_exp((1j * eps) * h).numpy()
    return out


def volume(dims) -> int:
    return int(np.prod(dims))


def gauge_field(dims, N: int, kind: str, seed: int = 0, eps: float = 0.3) -> np.ndarray:
    """Fundamental links (V, 4, N, N): kind = 'unit', 'haar' or 'smooth'."""
    V = volume(dims)
    if kind == "unit":
        return np.broadcast_to(np.eye(N, dtype=np.complex128), (V, 4, N, N)).copy()
    if kind == "haar":
        return haar_su(seed, V * 4, N).reshape(V, 4, N, N)
    if kind == "smooth":
        return smooth_su(seed, V * 4, N, eps).reshape(V, 4, N, N)
    raise ValueError(kind)


def gaussian_spinor(dims, d: int, seed: int) -> np.ndarray:
    """Gaussian source (V, 4, d): every real component N(0, 1)."""
    return complex_gaussians(seed, (volume(dims), 4, d))


def device_gaussian_spinors(dims, d: int, nrhs: int, seed: int, device="cuda"):
    """nrhs Gaussian sources (nrhs, V, 4, d) complex128 drawn on the device
    with torch's seeded Philox generator: for timing-only inputs too large to
    draw quickly on the host (every real component N(0, 1))."""
    import torch

    g = torch.Generator(device=device)
    g.manual_seed(seed)
    shape = (nrhs, volume(dims), 4, d, 2)
    v = torch.randn(shape, generator=g, device=device, dtype=torch.float64)
    return torch.view_as_complex(v)


def device_smooth_gauge_field(dims, N: int, seed: int, eps: float, device="cuda", chunk: int = 1 << 22):
    """Fundamental links (V, 4, N, N) complex128 on the device, U = exp(i eps H)
    with H = sum_a h_a T^a, h_a ~ N(0, 1) over the generalised Gell-Mann
    generators as in traceless_hermitian, but drawn with torch's seeded
    Philox generator on the device: for timing-scale lattices whose host
    generation would take minutes (a different random stream from
    gauge_field, the same distribution)."""
    import torch

    V = volume(dims)
    count = V * 4
    g = torch.Generator(device=device)
    g.manual_seed(seed)
    out = torch.empty((count, N, N), dtype=torch.complex128, device=device)
    noff = N * (N - 1) // 2
    for s0 in range(0, count, chunk):
        n = min(chunk, count - s0)
        h = torch.randn((n, N * N - 1), generator=g, device=device, dtype=torch.float64)
        H = torch.zeros((n, N, N), dtype=torch.complex128, device=device)
        k = 0
        for i in range(N):
            for j in range(i + 1, N):
                H[:, i, j] = torch.complex(0.5 * h[:, k], -0.5 * h[:, noff + k])
                H[:, j, i] = torch.conj(H[:, i, j])
                k += 1
        for l in range(1, N):
            c = h[:, 2 * noff + l - 1] / np.sqrt(2.0 * l * (l + 1))
            for i in range(l):
                H[:, i, i] += c
            H[:, l, l] -= l * c
        out[s0:s0 + n] = torch.linalg.matrix_exp((1j * eps) * H)
    return out.reshape(V, 4, N, N)


def gauge_transform(dims, N: int, seed: int) -> np.ndarray:
    """Haar-random g(x) in SU(N) for every site, (V, N, N)."""
    return haar_su(seed, volume(dims), N)


def site_coords(dims) -> np.ndarray:
    """(V, 4) integer coordinates (t, x, y, z) of each canonical site."""
    T, X, Y, Z = dims
    c = np.meshgrid(np.arange(T), np.arange(X), np.arange(Y), np.arange(Z), indexing="ij")
    return np.stack([a.reshape(-1) for a in c], axis=1)
