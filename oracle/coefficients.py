"""Exact candidate-stencil coefficients and linear weights of the NENO6 scheme.

Test infrastructure (part of the oracle): derived here in exact rational
arithmetic, then rounded once to binary64.

Sec. 2, Eqs. (definitionEq) and (approximatepolynomial): the point values
f_j act as cell averages of a primitive function h; on a candidate stencil of
r_k points h is approximated by a polynomial of degree r_k - 1 whose cell
averages match f_j, and the numerical flux is that polynomial at x_{i+1/2}.
With dx = 1 and x_i = 0 the flux is sum_j c_j f_j, where the c_j solve

    sum_j c_j * int_{o_j - 1/2}^{o_j + 1/2} xi^l dxi = (1/2)^l,  l = 0..r_k-1,

o_j being the cell offsets of the stencil relative to i.

Candidate stencils of incremental width (Fig. 1 of the paper, whose image is
missing from the source; the assignment below is the one that reproduces the
paper's Table "Convergencesmooth" digit for digit):
    S0 = {i-1, i, i+1}, S1 = {i, i+1, i+2}, S2 = {i-2, i-1, i},
    S3 = {i, i+1, i+2, i+3}.

Optimal linear weights d_k of TENO6-opt / NENO6: printed in Sec. 2.2 and
repeated in Sec. 4.  With them the linear scheme is fourth order (Sec. 4.1
states the fourth-order constraint).  The weights that reproduce the unique
sixth-order six-point scheme are derived below (for the sixth-order test
mode only).
"""
from fractions import Fraction

STENCIL_OFFSETS = {
    0: (-1, 0, 1),
    1: (0, 1, 2),
    2: (-2, -1, 0),
    3: (0, 1, 2, 3),
}

# Sec. 2.2: d_0..d_3 as printed (decimal strings, rounded once by float()).
PAPER_D = ("0.4294317718960898", "0.1727270875843552", "0.0855682281039113",
           "0.312272912415645")


def _cell_moment(o, l):
    """int_{o-1/2}^{o+1/2} xi^l dxi, exactly."""
    a = Fraction(2 * o - 1, 2)
    b = Fraction(2 * o + 1, 2)
    return (b ** (l + 1) - a ** (l + 1)) / (l + 1)


def _solve(A, b):
    """Gaussian elimination in exact arithmetic on a square system."""
    n = len(A)
    M = [list(row) + [rhs] for row, rhs in zip(A, b)]
    for col in range(n):
        piv = next(r for r in range(col, n) if M[r][col] != 0)
        M[col], M[piv] = M[piv], M[col]
        for r in range(n):
            if r != col and M[r][col] != 0:
                fac = M[r][col] / M[col][col]
                M[r] = [x - fac * y for x, y in zip(M[r], M[col])]
    return [M[r][n] / M[r][r] for r in range(n)]


def reconstruction_coefficients(offsets):
    """Exact c_j with h(x_{i+1/2}) = sum_j c_j f_j for polynomials of degree
    len(offsets)-1 (Eqs. definitionEq / approximatepolynomial)."""
    r = len(offsets)
    A = [[_cell_moment(o, l) for o in offsets] for l in range(r)]
    b = [Fraction(1, 2) ** l for l in range(r)]
    return _solve(A, b)


def candidate_coefficients_exact():
    return {k: reconstruction_coefficients(off) for k, off in STENCIL_OFFSETS.items()}


def candidate_coefficients():
    """4x4 binary64 table; row k holds S_k's coefficients in stencil order
    (S0..S2 use the first three entries)."""
    ex = candidate_coefficients_exact()
    out = [[0.0] * 4 for _ in range(4)]
    for k, cs in ex.items():
        for l, c in enumerate(cs):
            out[k][l] = float(c)
    return out


def sixth_order_weights_exact():
    """d_k with sum_k d_k S_k equal to the six-point sixth-order scheme over
    offsets -2..3 (solved exactly; the 6x4 system is consistent)."""
    full = reconstruction_coefficients((-2, -1, 0, 1, 2, 3))
    ex = candidate_coefficients_exact()
    rows = []
    for p in range(-2, 4):
        row = []
        for k in range(4):
            off = STENCIL_OFFSETS[k]
            row.append(ex[k][off.index(p)] if p in off else Fraction(0))
        rows.append(row)
    # Pick four independent rows, solve, then verify all six.
    import itertools
    for pick in itertools.combinations(range(6), 4):
        A = [rows[i] for i in pick]
        try:
            d = _solve(A, [full[i] for i in pick])
        except (StopIteration, ZeroDivisionError):
            continue
        if all(sum(a * x for a, x in zip(rows[i], d)) == full[i] for i in range(6)):
            return d
    raise RuntimeError("no consistent sixth-order weights")


def linear_weights(kind="paper"):
    if kind == "paper":
        return [float(s) for s in PAPER_D]
    if kind == "sixth":
        return [float(x) for x in sixth_order_weights_exact()]
    raise ValueError(kind)
