"""Pins for the FP64 CPU oracle: every check here compares the oracle with
something other than itself -- the Clifford algebra, group theory (the
homomorphism property, characters, the centre), the closed-form free Wilson
operator in momentum space, gamma5-hermiticity, gauge covariance, dense
linear algebra (numpy's eigvalsh/solve, an independent Schur complement) and
brute force on 2^4 lattices.  No GPU is involved."""
import itertools

import numpy as np
import pytest

import oracle as orc
from paper_1401_3733_gb300 import fields

pytestmark = pytest.mark.filterwarnings("ignore::RuntimeWarning")

REPS = [(2, orc.FUND), (3, orc.FUND), (4, orc.FUND), (6, orc.FUND),
        (2, orc.ADJ), (3, orc.ADJ), (2, orc.SYM), (3, orc.SYM),
        (3, orc.ASYM), (4, orc.ASYM)]
REP_IDS = [f"SU{N}-{['F', 'ADJ', 'S', 'AS'][r]}" for N, r in REPS]


def inner(a, b):
    return np.vdot(a.reshape(-1), b.reshape(-1))


def rel(a, b):
    return np.linalg.norm((a - b).reshape(-1)) / np.linalg.norm(b.reshape(-1))


# ----------------------------------------------------------------------------
# gamma matrices
# ----------------------------------------------------------------------------

def test_gamma_clifford_and_hermiticity():
    g = [orc.gamma(mu) for mu in range(5)]
    I4 = np.eye(4)
    for mu in range(4):
        assert np.allclose(g[mu], g[mu].conj().T, atol=0)
        for nu in range(4):
            assert np.allclose(g[mu] @ g[nu] + g[nu] @ g[mu], 2 * (mu == nu) * I4, atol=0)
        assert np.allclose(g[4] @ g[mu] + g[mu] @ g[4], 0, atol=0)
    assert np.allclose(g[4], np.diag([-1, -1, 1, 1]), atol=0)


# ----------------------------------------------------------------------------
# representation maps
# ----------------------------------------------------------------------------

def test_rep_dims():
    assert [orc.rep_dim(N, r) for N, r in REPS] == [2, 3, 4, 6, 3, 8, 3, 6, 3, 6]
    assert orc.rep_dim(2, orc.ASYM) == -1   # the trivial representation is excluded
    assert orc.rep_dim(1, orc.FUND) == -1


@pytest.mark.parametrize("N,rep", REPS, ids=REP_IDS)
def test_rep_group_properties(N, rep):
    U, W = fields.haar_su(11 + N, 2, N)
    RU, RW, RUW = (orc.rep_matrix(N, rep, M) for M in (U, W, U @ W))
    d = RU.shape[0]
    assert np.abs(RUW - RU @ RW).max() < 1e-14                   # homomorphism
    assert np.abs(RU @ RU.conj().T - np.eye(d)).max() < 1e-14    # unitarity
    assert abs(np.linalg.det(RU) - 1) < 1e-13                    # SU(N) is perfect
    assert np.abs(orc.rep_matrix(N, rep, np.eye(N)) - np.eye(d)).max() < 1e-15
    if rep == orc.ADJ:
        assert np.abs(RU.imag).max() < 1e-15                     # a real representation


@pytest.mark.parametrize("N,rep", REPS, ids=REP_IDS)
def test_rep_characters_and_centre(N, rep):
    U = fields.haar_su(5 * N + rep, 1, N)[0]
    tr, tr2 = np.trace(U), np.trace(U @ U)
    want = {orc.FUND: tr, orc.ADJ: abs(tr) ** 2 - 1,
            orc.SYM: (tr ** 2 + tr2) / 2, orc.ASYM: (tr ** 2 - tr2) / 2}[rep]
    assert abs(np.trace(orc.rep_matrix(N, rep, U)) - want) < 1e-13
    z = np.exp(2j * np.pi / N)
    Rz = orc.rep_matrix(N, rep, z * np.eye(N))
    d = Rz.shape[0]
    zc = {orc.FUND: z, orc.ADJ: 1.0, orc.SYM: z * z, orc.ASYM: z * z}[rep]
    assert np.abs(Rz - zc * np.eye(d)).max() < 1e-14


def test_su2_adjoint_is_so3():
    for U in fields.haar_su(3, 5, 2):
        R = orc.rep_matrix(2, orc.ADJ, U).real
        assert np.abs(R @ R.T - np.eye(3)).max() < 1e-14
        assert abs(np.linalg.det(R) - 1) < 1e-14


# ----------------------------------------------------------------------------
# free field: closed form in momentum space
# ----------------------------------------------------------------------------

def free_symbol(m0, p):
    """Textbook free Wilson operator in momentum space,
    D(p) = m0 + sum_mu (1 - cos p_mu) + i sum_mu gamma_mu sin p_mu."""
    D = (m0 + np.sum(1 - np.cos(p))) * np.eye(4, dtype=np.complex128)
    for mu in range(4):
        D = D + 1j * np.sin(p[mu]) * orc.gamma(mu)
    return D


@pytest.mark.parametrize("dims,phase", [
    ((4, 4, 4, 4), (np.pi, 0, 0, 0)),
    ((2, 2, 2, 2), (0, 0, 0, 0)),
    ((6, 4, 2, 4), (0.7, -1.1, 0.3, 2.0)),
    ((2, 4, 6, 2), (np.pi, np.pi, 0, 0.5)),
])
def test_free_field_plane_waves(dims, phase):
    N, rep, m0 = 3, orc.FUND, 0.13
    lat = orc.Lattice(dims, N, rep, m0, phase)
    R = orc.links_to_rep(lat, fields.gauge_field(dims, N, "unit"))
    xs = fields.site_coords(dims)
    rng = np.random.default_rng(7)
    for _ in range(4):
        n = np.array([rng.integers(0, L) for L in dims])
        p = (2 * np.pi * n + np.array(phase)) / np.array(dims)
        chi = rng.standard_normal((4, 3)) + 1j * rng.standard_normal((4, 3))
        wave = np.exp(1j * xs @ p)
        psi = wave[:, None, None] * chi[None]
        want = wave[:, None, None] * (free_symbol(m0, p) @ chi)[None]
        assert rel(orc.dirac(lat, R, psi), want) < 1e-14
        want_dag = wave[:, None, None] * (free_symbol(m0, p).conj().T @ chi)[None]
        assert rel(orc.dirac(lat, R, psi, dagger=True), want_dag) < 1e-14


@pytest.mark.parametrize("dims,phase,N,rep", [
    ((2, 2, 2, 2), (np.pi, 0, 0, 0), 2, orc.FUND),
    ((4, 2, 2, 2), (0.4, 0, 1.0, 0), 2, orc.ADJ),
])
def test_free_field_dense_spectrum(dims, phase, N, rep):
    """Eigenvalues of the dense D^+D against the closed form
    (m0 + sum(1-cos p))^2 + sum sin^2 p, each with multiplicity 4 d."""
    m0 = 0.1
    lat = orc.Lattice(dims, N, rep, m0, phase)
    R = orc.links_to_rep(lat, fields.gauge_field(dims, N, "unit"))
    M = orc.dense_dirac(lat, R)
    ev = np.linalg.eigvalsh(M.conj().T @ M)
    want = []
    for n in itertools.product(*[range(L) for L in dims]):
        p = (2 * np.pi * np.array(n) + np.array(phase)) / np.array(dims)
        want += [(m0 + np.sum(1 - np.cos(p))) ** 2 + np.sum(np.sin(p) ** 2)] * (4 * lat.d)
    assert np.abs(np.sort(ev) - np.sort(want)).max() < 2e-13


# ----------------------------------------------------------------------------
# interacting field: dense assembly, gamma5-hermiticity, gauge covariance
# ----------------------------------------------------------------------------

@pytest.mark.parametrize("N,rep", REPS[:7], ids=REP_IDS[:7])
def test_dense_equals_matrix_free(N, rep):
    dims = (2, 2, 2, 2) if N <= 3 else (2, 2, 2, 2)
    lat = orc.Lattice(dims, N, rep, 0.2, (np.pi, 0.3, 0, 0))
    R = orc.links_to_rep(lat, fields.gauge_field(dims, N, "haar", seed=21))
    M = orc.dense_dirac(lat, R)
    psi = fields.gaussian_spinor(dims, lat.d, 22)
    assert rel(orc.dirac(lat, R, psi), (M @ psi.reshape(-1)).reshape(psi.shape)) < 1e-14
    # the dagger flag is the adjoint matrix
    got = orc.dirac(lat, R, psi, dagger=True)
    assert rel(got, (M.conj().T @ psi.reshape(-1)).reshape(psi.shape)) < 1e-14


@pytest.mark.parametrize("N,rep", REPS, ids=REP_IDS)
def test_gamma5_hermiticity(N, rep):
    dims = (4, 2, 2, 4)
    lat = orc.Lattice(dims, N, rep, 0.05, (np.pi, 0, 0, 0))
    R = orc.links_to_rep(lat, fields.gauge_field(dims, N, "haar", seed=31))
    phi = fields.gaussian_spinor(dims, lat.d, 32)
    psi = fields.gaussian_spinor(dims, lat.d, 33)
    g5 = np.diag([-1.0, -1.0, 1.0, 1.0])
    G5 = lambda f: np.einsum("ab,sbc->sac", g5, f)
    lhs = inner(phi, G5(orc.dirac(lat, R, G5(psi))))
    rhs = inner(orc.dirac(lat, R, phi), psi)
    assert abs(lhs - rhs) / abs(rhs) < 1e-13
    # and the dagger flag is gamma5 D gamma5
    assert rel(orc.dirac(lat, R, psi, dagger=True), G5(orc.dirac(lat, R, G5(psi)))) < 1e-14


@pytest.mark.parametrize("N,rep", REPS, ids=REP_IDS)
def test_gauge_covariance(N, rep):
    """D[U^g] R(g) psi = R(g) D[U] psi with U^g_mu(x) = g(x) U_mu(x) g(x+mu)^+."""
    dims = (4, 2, 4, 2)
    lat = orc.Lattice(dims, N, rep, 0.1, (np.pi, 0, 0.9, 0))
    U = fields.gauge_field(dims, N, "haar", seed=41)
    g = fields.gauge_transform(dims, N, 42)
    xs = fields.site_coords(dims)
    Ug = np.empty_like(U)
    T, X, Y, Z = dims
    for mu in range(4):
        c = xs.copy()
        c[:, mu] = (c[:, mu] + 1) % dims[mu]
        fwd = ((c[:, 0] * X + c[:, 1]) * Y + c[:, 2]) * Z + c[:, 3]
        Ug[:, mu] = g @ U[:, mu] @ np.conj(np.transpose(g[fwd], (0, 2, 1)))
    Rg = orc.links_to_rep(lat, np.repeat(g[:, None], 4, axis=1))[:, 0]
    psi = fields.gaussian_spinor(dims, lat.d, 43)
    rot = lambda f: np.einsum("sab,sib->sia", Rg, f)
    lhs = orc.dirac(lat, orc.links_to_rep(lat, Ug), rot(psi))
    rhs = rot(orc.dirac(lat, orc.links_to_rep(lat, U), psi))
    assert rel(lhs, rhs) < 1e-13


# ----------------------------------------------------------------------------
# even-odd operator and solver
# ----------------------------------------------------------------------------

def _eo_setup(dims, N, rep, seed, m0=0.1, phase=(np.pi, 0, 0, 0)):
    lat = orc.Lattice(dims, N, rep, m0, phase)
    R = orc.links_to_rep(lat, fields.gauge_field(dims, N, "haar", seed=seed))
    odd = orc.parity_mask(dims)
    return lat, R, odd


@pytest.mark.parametrize("N,rep", [(2, orc.FUND), (3, orc.FUND), (2, orc.ADJ)])
def test_dhat_is_schur_complement(N, rep):
    """Dhat against the Schur complement D_ee - D_eo D_oo^-1 D_oe of the dense
    D, up to the normalisation: D_ee = D_oo = A, so Dhat = Schur."""
    dims = (2, 2, 2, 4)
    lat, R, odd = _eo_setup(dims, N, rep, 51)
    d = lat.d
    M = orc.dense_dirac(lat, R)
    rows = np.repeat(odd, 4 * d)
    Mee, Meo = M[~rows][:, ~rows], M[~rows][:, rows]
    Moe, Moo = M[rows][:, ~rows], M[rows][:, rows]
    S = Mee - Meo @ np.linalg.solve(Moo, Moe)
    psi = fields.gaussian_spinor(dims, d, 52)
    psi[odd] = 0
    for op, mat in [(orc.DHAT, S), (orc.DHAT_DAG, S.conj().T),
                    (orc.DHAT_DAG_DHAT, S.conj().T @ S)]:
        got = orc.dhat(lat, R, psi, op)
        assert np.abs(got[odd]).max() == 0
        want = mat @ psi[~odd].reshape(-1)
        assert rel(got[~odd].reshape(-1), want) < 1e-13


def test_lu_solve_against_numpy():
    rng = np.random.default_rng(3)
    A = rng.standard_normal((40, 40)) + 1j * rng.standard_normal((40, 40))
    b = rng.standard_normal(40) + 1j * rng.standard_normal(40)
    assert rel(orc.lu_solve(A, b), np.linalg.solve(A, b)) < 1e-12


@pytest.mark.parametrize("eo", [True, False])
@pytest.mark.parametrize("N,rep", [(2, orc.FUND), (3, orc.FUND), (2, orc.ADJ), (3, orc.ASYM)])
def test_cg_against_dense_lu(eo, N, rep):
    dims = (2, 2, 2, 2)
    lat, R, odd = _eo_setup(dims, N, rep, 61)
    b = fields.gaussian_spinor(dims, lat.d, 62)
    M = orc.dense_dirac(lat, R)
    x_lu = orc.lu_solve(M, b.reshape(-1)).reshape(b.shape)
    assert rel(x_lu, np.linalg.solve(M, b.reshape(-1)).reshape(b.shape)) < 1e-12
    x, it, res = orc.cg(lat, R, b, eo=eo, tol=1e-12, max_iter=2000)
    assert it > 0 and res <= 1e-12
    assert rel(x, x_lu) < 1e-9
    assert rel(orc.dirac(lat, R, x), b) < 1e-9


def test_cg_initial_guess_restart():
    dims = (2, 2, 2, 4)
    lat, R, _ = _eo_setup(dims, 2, orc.FUND, 71)
    b = fields.gaussian_spinor(dims, 2, 72)
    x1, it1, _ = orc.cg(lat, R, b, eo=True, tol=1e-6)
    x2, it2, res2 = orc.cg(lat, R, b, eo=True, tol=1e-11, x0=x1)
    x3, it3, _ = orc.cg(lat, R, b, eo=True, tol=1e-11)
    assert res2 <= 1e-11 and it2 < it3
    assert rel(x2, x3) < 1e-9


def test_cg_free_field_terminates_within_distinct_eigenvalues():
    """In exact arithmetic CG on a Hermitian positive-definite matrix ends
    within the number of distinct eigenvalues; the free eo operator on 4^4
    has only a few dozen."""
    dims, N = (4, 4, 4, 4), 2
    lat = orc.Lattice(dims, N, orc.FUND, 0.1, (np.pi, 0, 0, 0))
    R = orc.links_to_rep(lat, fields.gauge_field(dims, N, "unit"))
    odd = orc.parity_mask(dims)
    M = orc.dense_dirac(lat, R)
    rows = np.repeat(odd, 4 * lat.d)
    S = M[~rows][:, ~rows] - M[~rows][:, rows] @ np.linalg.solve(M[rows][:, rows], M[rows][:, ~rows])
    ev = np.sort(np.linalg.eigvalsh(S.conj().T @ S))
    distinct = 1 + int(np.sum(np.diff(ev) > 1e-9 * ev[-1]))
    b = fields.gaussian_spinor(dims, lat.d, 81)
    _, it, res = orc.cg(lat, R, b, eo=True, tol=1e-10, max_iter=1000)
    assert 0 < it <= distinct + 2, (it, distinct)
