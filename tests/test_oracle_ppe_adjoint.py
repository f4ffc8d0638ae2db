"""Pins of the oracle's pressure-equation assembly and transpose solve (the
adjoint of the pressure solve).

  * the dense matrix assembled column by column from the oracle's operator
    reproduces the oracle's own solve: A p = b on the unknown rows (a matrix
    assembled by rows instead of columns fails: A is not symmetric);
  * the transpose solve satisfies the adjoint identity <p_bar, A^-1 b> =
    <A^-T p_bar, b> with the oracle's own b and p, and a solve with A instead
    of A^T does not.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2607_28872_b300 import scenarios as S


@pytest.fixture(scope="module")
def system():
    sc = S.small_tank(dim=2, kind="SIGMA", L=0.2, H=0.06, d0=0.01, seed=2, with_wave=True)
    return O.ppe_system(sc, rtol=1e-13)


def test_assembly_reproduces_the_solve(system):
    rows, A, b, p = system
    assert rows.size > 50
    assert np.abs(A @ p - b).max() < 1e-10 * np.abs(b).max()
    asym = np.abs(A - A.T).max() / np.abs(A).max()
    assert asym > 1e-3                                   # not symmetric
    assert np.abs(A.T @ p - b).max() > 1e-4 * np.abs(b).max()


def test_transpose_solve_adjoint_identity(system):
    rows, A, b, p = system
    rng = np.random.default_rng(7)
    pb = rng.normal(size=rows.size)
    bb = O.ppe_adjoint(A, pb)
    lhs, rhs = pb @ p, bb @ b
    assert abs(lhs - rhs) < 1e-10 * (np.abs(pb) @ np.abs(p))
    wrong = np.linalg.solve(A, pb)
    assert abs(wrong @ b - lhs) > 1e-4 * (np.abs(pb) @ np.abs(p))
