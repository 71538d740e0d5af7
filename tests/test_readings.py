"""Exact-arithmetic checks of the evaluation orders the library uses instead of the plain chain of Eq. 1.

Each grouping must give the same matrix as the plain coupled chain N (N (... (N M))) for every symmetric
M, since all factors are polynomials in M. Checked in exact rational arithmetic (sympy) on small dense
matrices, so that a wrong coefficient cannot hide behind rounding.
"""
import pytest

sympy = pytest.importorskip("sympy")


def rational_symmetric(n, seed):
    import random
    rnd = random.Random(seed)
    M = sympy.zeros(n, n)
    for i in range(n):
        for j in range(i, n):
            v = sympy.Rational(rnd.randint(-9, 9), rnd.randint(1, 7))
            M[i, j] = M[j, i] = v
    return M


@pytest.mark.parametrize("p", [1, 2, 3, 4])
def test_coupled_update_groupings_equal_the_plain_chain(p):
    n = 4
    I = sympy.eye(n)
    for seed in range(3):
        M = rational_symmetric(n, 10 * p + seed)
        N = ((p + 1) * I - M) / p
        plain = M
        for _ in range(p):
            plain = N * plain
        if p == 3:
            # N^3 M = L R, L = 4M - M^2, R = (16 I - 8 M + M^2) / 27
            S = M * M
            L = 4 * M - S
            R = (16 * I - 8 * M + S) / 27
            grouped = L * R
        elif p == 4:
            N2 = N * N
            grouped = (N2 * N2) * M
        else:
            grouped = plain
        assert (grouped - plain).applyfunc(sympy.simplify) == sympy.zeros(n, n)
        # The next N of the fused epilogue: ((p + 1) I - M') / p.
        Nn = ((p + 1) * I - grouped) / p
        assert Nn == ((p + 1) * I - plain) / p


def test_newton_schulz_is_the_p1_coupled_step():
    # p = 1: C' = C (2I - A C) is Eq. 1 with p = 1, C' = 2C - C^2 A, when C commutes with A.
    n = 3
    A = rational_symmetric(n, 5)
    C = 2 * A + A * A  # a polynomial in A
    assert C * (2 * sympy.eye(n) - A * C) == 2 * C - C * C * A
