"""Pins for the CPU oracle: it is checked against things other than itself.

Hand-worked closed forms (tests/golden), an exact-rational brute force of the
probabilistic definition, the paper's tie-free Alg. 1 / Alg. 2, invariants
that the mathematics fixes (sum of C = n/2, row sums = local depth, bounds),
metamorphic relations, and planted mistakes that the pins must catch.
"""
from fractions import Fraction
import os

import numpy as np
import pytest

import oracle
from paper_2307_16652_gb300 import inputs
from tests import pald_exact as ex

pytestmark = pytest.mark.filterwarnings("ignore::RuntimeWarning")


def _as_f32(rows):
    return np.array([[float(v) for v in r] for r in rows], dtype=np.float32)


def _check_exact(D, U, C, atol=1e-14):
    """u exact and C within FP64 rounding of the exact-rational brute force."""
    u_ex, C_ex = ex.exact_pald(D.tolist())
    assert np.array_equal(U, np.array(u_ex)), "u differs from the exact definition"
    C_ex = np.array([[float(v) for v in r] for r in C_ex])
    assert np.allclose(C, C_ex, rtol=1e-14, atol=atol), "C differs from the exact definition"


# --------------------------------------------------------------------------
# hand-worked closed forms


def test_golden_cases(golden_dir):
    cases = ex.load_golden(os.path.join(golden_dir, "hand_worked.txt"))
    assert len(cases) >= 5
    for case in cases:
        D = _as_f32(case["D"])
        U, C = oracle.focus_and_cohesion(D, threads=2)
        assert np.array_equal(U, np.array(case["u"], dtype=np.int64)), case["name"]
        expect = np.array([[float(v) for v in r] for r in case["C"]])
        assert np.allclose(C, expect, rtol=0, atol=1e-15), case["name"]


def test_golden_cases_agree_with_exact_enumeration(golden_dir):
    """The fixtures themselves against the rational brute force."""
    for case in ex.load_golden(os.path.join(golden_dir, "hand_worked.txt")):
        u, C = ex.exact_pald(case["D"])
        assert u == [[int(v) for v in r] for r in case["u"]], case["name"]
        assert C == case["C"], case["name"]


# --------------------------------------------------------------------------
# brute force on tiny inputs


@pytest.mark.parametrize("seed", range(6))
def test_bruteforce_tie_heavy(seed):
    rng = np.random.default_rng(1000 + seed)
    for _ in range(40):
        n = int(rng.integers(2, 9))
        D = inputs.small_tie_heavy(rng, n, hi=int(rng.choice([1, 2, 3, 5])), dup=bool(rng.integers(0, 2)))
        U, C = oracle.focus_and_cohesion(D, threads=1)
        _check_exact(D, U, C)


def test_bruteforce_euclidean():
    rng = np.random.default_rng(77)
    for _ in range(30):
        n = int(rng.integers(2, 9))
        D = inputs.small_points_matrix(rng, n)
        U, C = oracle.focus_and_cohesion(D, threads=1)
        _check_exact(D, U, C)


def test_all_equal_and_all_zero():
    for n in (2, 3, 5, 8):
        D = np.ones((n, n), dtype=np.float32)
        np.fill_diagonal(D, 0)
        U, C = oracle.focus_and_cohesion(D)
        _check_exact(D, U, C)
        # every focus is the whole set; c_xx = 1/n, off-diagonal c_xz = 1/(2n)(n-2)/(n-1)
        assert np.all(U[~np.eye(n, dtype=bool)] == n)
        assert np.allclose(np.diag(C), 1.0 / n)
        if n > 2:
            off = C[~np.eye(n, dtype=bool)]
            assert np.allclose(off, (n - 2) / (2.0 * n * (n - 1)))
    Z = np.zeros((4, 4), dtype=np.float32)        # four coincident points
    U, C = oracle.focus_and_cohesion(Z)
    _check_exact(Z, U, C)
    assert np.all(U == 4) and np.allclose(C, 1.0 / 8.0)


# --------------------------------------------------------------------------
# the paper's own algorithms on tie-free inputs


@pytest.mark.parametrize("n", [5, 17, 40])
def test_tie_free_matches_pairwise_and_triplet_algorithms(n):
    rng = np.random.default_rng(n)
    D = inputs.small_points_matrix(rng, n, dim=4)
    off = ~np.eye(n, dtype=bool)
    vals = D[off]
    assert len(np.unique(vals)) == len(vals) // 2, "input must be tie-free"
    U, C = oracle.focus_and_cohesion(D)
    U1, C1 = ex.pairwise_alg(D)
    U2, C2 = ex.triplet_alg(D)
    assert np.array_equal(U[off], U1[off]) and np.array_equal(U[off], U2[off])
    assert np.allclose(C * (n - 1), C1, rtol=1e-12, atol=1e-14)            # incl. diagonal
    assert np.allclose((C * (n - 1))[off], C2[off], rtol=1e-12, atol=1e-14)


# --------------------------------------------------------------------------
# invariants fixed by the mathematics


def _invariants(D, U, C):
    n = D.shape[0]
    off = ~np.eye(n, dtype=bool)
    assert np.array_equal(U, U.T)
    assert U[off].min() >= 2 and U[off].max() <= n
    assert np.array_equal(np.diag(U), (D <= 0).sum(axis=1))
    assert C.min() >= 0
    # each unordered pair's focus hands out exactly one unit between x and y:
    # the sum of all cohesion values is n/2
    assert abs(C.sum() - n / 2.0) < 1e-9 * n
    ld = C.sum(axis=1)
    assert ld.min() >= 0 and ld.max() <= 1 + 1e-12
    # c_zx = 0 whenever z is not in any focus of x closer ... weaker but cheap:
    # c_xz > 0 requires d_xz <= d_xy for some y != x, i.e. z is not the
    # unique farthest point from x
    return ld


@pytest.mark.parametrize("maker", ["plain", "tie", "dup"])
def test_invariants(maker):
    rng = np.random.default_rng(5)
    if maker == "plain":
        D = inputs.plain_matrix(96)
    elif maker == "tie":
        D = inputs.tie_heavy_matrix(97, hi=6)
    else:
        D = inputs.small_tie_heavy(rng, 60, hi=3, dup=True)
    U, C = oracle.focus_and_cohesion(D)
    ld = _invariants(D, U, C)
    # row sums are the local depths of eq. (LD), evaluated on their own
    for x in (0, 7, D.shape[0] - 1):
        assert abs(ld[x] - float(ex.local_depth_exact(D.tolist(), x))) < 1e-12


def test_rows_match_full():
    D = inputs.tie_heavy_matrix(150, hi=9)
    U, C = oracle.focus_and_cohesion(D)
    rows = np.array([0, 3, 77, 149])
    Ur, Cr = oracle.rows(D, rows)
    assert np.array_equal(Ur, U[rows])
    assert np.array_equal(Cr, C[rows])
    C2 = oracle.cohesion_from_u(D, U)
    assert np.array_equal(C2, C)


# --------------------------------------------------------------------------
# metamorphic relations


def test_monotone_map_and_power_of_two_scaling():
    D = inputs.tie_heavy_matrix(120, hi=20)
    U, C = oracle.focus_and_cohesion(D)
    U2, C2 = oracle.focus_and_cohesion(D * D)          # exact for integers <= 20
    assert np.array_equal(U, U2) and np.array_equal(C, C2)
    P = inputs.plain_matrix(128)
    U, C = oracle.focus_and_cohesion(P)
    U3, C3 = oracle.focus_and_cohesion(P * np.float32(0.125))
    assert np.array_equal(U, U3) and np.array_equal(C, C3)


def test_permutation_equivariance():
    rng = np.random.default_rng(3)
    D = inputs.tie_heavy_matrix(90, hi=7)
    p = rng.permutation(90)
    U, C = oracle.focus_and_cohesion(D)
    Up, Cp = oracle.focus_and_cohesion(D[np.ix_(p, p)])
    assert np.array_equal(Up, U[np.ix_(p, p)])
    assert np.allclose(Cp, C[np.ix_(p, p)], rtol=1e-13, atol=1e-15)


# --------------------------------------------------------------------------
# planted mistakes: every mutant of the oracle must fail one of the pins


def _pins_pass(mutant):
    cases = ex.load_golden(os.path.join(os.path.dirname(__file__), "golden", "hand_worked.txt"))
    try:
        for case in cases:
            D = _as_f32(case["D"])
            U, C = oracle.focus_and_cohesion(D, threads=1, mutant=mutant)
            if not np.array_equal(U, np.array(case["u"], dtype=np.int64)):
                return False
            expect = np.array([[float(v) for v in r] for r in case["C"]])
            if not np.allclose(C, expect, rtol=0, atol=1e-15):
                return False
        rng = np.random.default_rng(11)
        for _ in range(20):
            n = int(rng.integers(3, 8))
            D = inputs.small_tie_heavy(rng, n, hi=3, dup=bool(rng.integers(0, 2)))
            U, C = oracle.focus_and_cohesion(D, threads=1, mutant=mutant)
            u_ex, C_ex = ex.exact_pald(D.tolist())
            if not np.array_equal(U, np.array(u_ex)):
                return False
            if not np.allclose(C, np.array([[float(v) for v in r] for r in C_ex]), atol=1e-14):
                return False
        return True
    except Exception:
        return False


@pytest.mark.parametrize("mutant", range(1, 10))
def test_planted_mistakes_are_caught(mutant):
    assert oracle._lib(mutant).pald_oracle_mutant() == mutant
    assert not _pins_pass(mutant), f"mutant {mutant} slipped through the pins"


def test_unmutated_oracle_passes_mutant_harness():
    assert _pins_pass(0)
