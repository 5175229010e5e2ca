"""Mutation check of the oracle's pins.  Each case plants one plausible
mistake (a flipped sign, a dropped term or phase, a transposed or
mis-indexed operand, a wrong normalisation) into a temporary copy of
oracle.c, builds it on the CPU, routes the oracle wrappers through it and
asserts that at least one pin of test_oracle_pins fails.  A pin battery
that passes on a mutant would mean that mistake could hide in the oracle."""
import os
import shutil
import subprocess

import numpy as np
import pytest

import oracle as orc
from tests import test_oracle_pins as pins

SRC = os.path.join(os.path.dirname(orc.__file__), "oracle.c")
HDR = os.path.join(os.path.dirname(orc.__file__), "oracle.h")

# (name, text in oracle.c, replacement); the first occurrence is replaced
MUTATIONS = [
    ("forward projector sign",
     "(al == be ? 1.0 : 0.0) - sgn * g[mu][al][be]", "(al == be ? 1.0 : 0.0) + sgn * g[mu][al][be]"),
    ("backward projector sign",
     "(al == be ? 1.0 : 0.0) + sgn * g[mu][al][be]", "(al == be ? 1.0 : 0.0) - sgn * g[mu][al][be]"),
    ("backward link not daggered",
     "acc += P * conj(Rl[b * d + a]) * p[be * d + b]", "acc += P * Rl[b * d + a] * p[be * d + b]"),
    ("backward link transposed only",
     "acc += P * conj(Rl[b * d + a]) * p[be * d + b]", "acc += P * conj(Rl[a * d + b]) * p[be * d + b]"),
    ("forward link transposed",
     "acc += P * Rl[a * d + b] * p[be * d + b]", "acc += P * Rl[b * d + a] * p[be * d + b]"),
    ("backward link taken at x instead of x - mu",
     "const cplx *Rl = R + (sb * 4 + mu) * d * d;", "const cplx *Rl = R + (s * 4 + mu) * d * d;"),
    ("forward neighbour in the wrong sense",
     "const long sf = neighbour(L, s, mu, +1);", "const long sf = neighbour(L, s, mu, -1);"),
    ("direction mu = 3 dropped",
     "for (int mu = 0; mu < 4; ++mu) {\n      /* forward", "for (int mu = 0; mu < 3; ++mu) {\n      /* forward"),
    ("forward boundary phase dropped",
     "(c[mu] == L->dims[mu] - 1) ? cexp(I * L->phase[mu]) : 1.0", "(c[mu] == L->dims[mu] - 1) ? 1.0 : 1.0"),
    ("backward boundary phase with the wrong sign",
     "(c[mu] == 0) ? cexp(-I * L->phase[mu]) : 1.0", "(c[mu] == 0) ? cexp(I * L->phase[mu]) : 1.0"),
    ("hopping term without the 1/2",
     "out[k] = A * in[k] - 0.5 * out[k];", "out[k] = A * in[k] - out[k];"),
    ("gamma_k with the opposite sign (other chirality)",
     "-I * sigma[mu][a][b]", "I * sigma[mu][a][b]"),
    ("Cartan generator normalisation",
     "1.0 / sqrt(2.0 * l * (l + 1))", "1.0 / sqrt(1.0 * l * (l + 1))"),
    ("adjoint built with U^T instead of U^+",
     "? conj(U[j * N + i]) /* U^+ */", "? U[j * N + i] /* U^+ */"),
    ("two-index basis with swapped symmetry",
     "(sym ? 1.0 : -1.0) / sqrt(2.0)", "(sym ? -1.0 : 1.0) / sqrt(2.0)"),
    ("adjoint without the factor 2",
     "(rep == ORC_ADJ ? 2.0 : 1.0) * trace(N, t3)", "trace(N, t3)"),
    ("Schur complement coefficient 1/(2A)",
     "- out[s * 4 * d + k] / (4.0 * A);", "- out[s * 4 * d + k] / (2.0 * A);"),
    ("eo source with 1/(4A)",
     "b[s * 4 * d + k] + t1[s * 4 * d + k] / (2.0 * A)", "b[s * 4 * d + k] + t1[s * 4 * d + k] / (4.0 * A)"),
    ("eo reconstruction sign",
     "(b[s * 4 * d + k] + 0.5 * t1[s * 4 * d + k]) / A", "(b[s * 4 * d + k] - 0.5 * t1[s * 4 * d + k]) / A"),
    ("CG beta inverted",
     "const double beta = rr_new / rr;", "const double beta = rr / rr_new;"),
    ("CG residual update sign",
     "r[k] -= alpha * Mp[k];", "r[k] += alpha * Mp[k];"),
    ("dense assembly overwrites instead of adding",
     "M[row * n + (sb * 4 + be) * d + b] += -0.5 * phb * Pp * Ub;",
     "M[row * n + (sb * 4 + be) * d + b] = -0.5 * phb * Pp * Ub;"),
    ("LU elimination drops the right-hand side update",
     "b[i] -= f * b[k];", "(void)f;"),
]


def battery():
    """The pin checks a mutant has to get past (a fast subset of the pins)."""
    F, ADJ, S, AS = orc.FUND, orc.ADJ, orc.SYM, orc.ASYM
    yield lambda: pins.test_gamma_clifford_and_hermiticity()
    for N, r in [(3, F), (3, ADJ), (3, S), (4, AS)]:
        yield lambda N=N, r=r: pins.test_rep_group_properties(N, r)
        yield lambda N=N, r=r: pins.test_rep_characters_and_centre(N, r)
    yield lambda: pins.test_free_field_plane_waves((6, 4, 2, 4), (0.7, -1.1, 0.3, 2.0))
    yield lambda: pins.test_free_field_plane_waves((2, 4, 6, 2), (np.pi, np.pi, 0, 0.5))
    yield lambda: pins.test_dense_equals_matrix_free(2, F)
    yield lambda: pins.test_gamma5_hermiticity(3, F)
    yield lambda: pins.test_gauge_covariance(3, F)
    yield lambda: pins.test_gauge_covariance(2, ADJ)
    yield lambda: pins.test_dhat_is_schur_complement(2, F)
    yield lambda: pins.test_lu_solve_against_numpy()
    yield lambda: pins.test_cg_against_dense_lu(True, 2, F)
    yield lambda: pins.test_cg_against_dense_lu(False, 2, F)


def test_battery_passes_on_the_real_oracle():
    for check in battery():
        check()


@pytest.mark.parametrize("name,old,new", MUTATIONS, ids=[m[0] for m in MUTATIONS])
def test_planted_mistake_is_caught(tmp_path, name, old, new):
    src = open(SRC).read()
    assert src.count(old) >= 1, f"mutation anchor not found: {old!r}"
    (tmp_path / "oracle.c").write_text(src.replace(old, new, 1))
    shutil.copy(HDR, tmp_path / "oracle.h")
    so = tmp_path / "libmut.so"
    subprocess.run(["gcc", "-std=c11", "-O1", "-fPIC", "-shared", "-o", str(so),
                    str(tmp_path / "oracle.c"), "-lm"], check=True)
    prev = orc.use_library(str(so))
    failed = []
    try:
        for i, check in enumerate(battery()):
            try:
                check()
            except (AssertionError, ValueError, ZeroDivisionError, np.linalg.LinAlgError):
                failed.append(i)
                break
    finally:
        orc.restore_library(prev)
    assert failed, f"no pin caught the planted mistake: {name}"
