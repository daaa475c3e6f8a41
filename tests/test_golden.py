"""Values the paper states, stored as fixtures under tests/golden/ (each file
cites its passage), checked on the CPU:

* the worked example of Section 3.1: every derivative of x1^3 x2^7 x3^2 from
  the exact oracle equals a_j times the common factor x1^2 x2^6 x3 times the
  derivative of the Speelpenning product x1 x2 x3, and the value is the
  common factor times the product;
* the multiplication counts of Sections 3.1 and 3.2 (d - 2 per variable for
  the powers, k - 1 per common factor, 3k - 6 for the Speelpenning
  derivatives, 5k - 4 per thread of the second kernel, 6k - 5 per monomial)
  against an instrumented model of the paper's procedure -- forward products
  in the locations L_2 .. L_k, one backward product Q -- whose outputs are
  checked against the exact oracle.
"""
import os
from fractions import Fraction

import numpy as np
import pytest

import synth
from oracle import exact as E

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
ONE = (Fraction(1), Fraction(0))


def rows(name):
    with open(os.path.join(GOLDEN, name)) as fh:
        return [ln.split() for ln in fh if ln.strip() and not ln.startswith("#")]


def fr(v):
    """A complex double-double [4] as an exact pair of Fractions."""
    return (Fraction(float(v[0])) + Fraction(float(v[1])), Fraction(float(v[2])) + Fraction(float(v[3])))


def fr_exact(z):
    a, b, e = z
    s = Fraction(2) ** e
    return (a * s, b * s)


def cmul(x, y):
    return (x[0] * y[0] - x[1] * y[1], x[0] * y[1] + x[1] * y[0])


def cpow(x, e):
    r = ONE
    for _ in range(e):
        r = cmul(r, x)
    return r


# ----------------------------------------------------------------------------
# Section 3.1, the worked example
# ----------------------------------------------------------------------------

def test_worked_example_common_factor_section3_1():
    (row,) = rows("common_factor_section3_1.txt")
    text = " ".join(row).split("|")
    a = [int(t) for t in text[0].split()]
    cf = [int(t) for t in text[1].split()]
    speel = [int(t) - 1 for t in text[2].split()]
    assert cf == [e - 1 for e in a] and speel == list(range(len(a)))
    n = len(a)
    s = synth.from_monomials(n, [[(speel, a)]], [[1.0, 0.0, 0.0, 0.0]])
    pts = synth.points(1201, n, 3)
    for q in range(pts.shape[1]):
        x = [fr(pts[v, q]) for v in range(n)]
        f, J = E.evaluate_point(s, pts, q)
        common = ONE
        for v in range(n):
            common = cmul(common, cpow(x[v], cf[v]))
        product = ONE
        for v in speel:
            product = cmul(product, x[v])
        assert fr_exact(f[0]) == cmul(common, product)
        for i in range(n):
            d_speel = ONE  # d/dx_i of x_1 x_2 x_3: the product without x_i
            for v in speel:
                if v != i:
                    d_speel = cmul(d_speel, x[v])
            want = cmul((Fraction(a[i]), Fraction(0)), cmul(common, d_speel))
            assert fr_exact(J[0][i]) == want


# ----------------------------------------------------------------------------
# Sections 3.1 and 3.2, the multiplication counts
# ----------------------------------------------------------------------------

class CountingMul:
    """Complex multiplication of exact pairs that counts its calls."""

    def __init__(self):
        self.n = 0

    def __call__(self, x, y):
        self.n += 1
        return cmul(x, y)


def powers_model(mul, x, d):
    """x^0 .. x^(d-1) of one variable: x^2 .. x^(d-1) by repeated
    multiplication (Section 3.1, first stage of the first kernel)."""
    p = [ONE, x]
    for _ in range(2, d):
        p.append(mul(p[-1], x))
    return p


def common_factor_model(mul, quantities):
    """The product of the k quantities x_{i_j}^(a_j - 1) (Section 3.1,
    second stage of the first kernel)."""
    cf = quantities[0]
    for q in quantities[1:]:
        cf = mul(cf, q)
    return cf


def second_kernel_model(mul, xs, cf, coef_value, coef_derivs):
    """The procedure of Section 3.2 for k >= 3 variables, with the locations
    L_1 .. L_{k+1} and the backward product Q; returns (derivatives of the
    monomial times their coefficients, value times its coefficient,
    multiplications spent on the Speelpenning derivatives, locations used)."""
    k = len(xs)
    L = [None] * (k + 2)  # L[1] .. L[k+1]
    n0 = mul.n
    L[2] = xs[0]
    for r in range(1, k - 1):  # the forward products x_1 ... x_{r+1} into L_{r+2}
        L[r + 2] = mul(L[r + 1], xs[r])
    Q = xs[k - 1]
    L[k - 1] = mul(L[k - 1], Q)  # derivative by x_{k-1}
    for r in range(1, k - 2):
        Q = mul(Q, xs[k - r - 1])  # Q = x_k x_{k-1} ... x_{k-r}
        L[k - r - 1] = mul(L[k - r - 1], Q)  # derivative by x_{k-r-1}
    Q = mul(Q, xs[1])
    L[1] = Q  # derivative by x_1
    speelpenning = mul.n - n0
    for j in range(1, k + 1):  # monomial derivatives: times the common factor
        L[j] = mul(L[j], cf)
    L[k + 1] = mul(L[k], xs[k - 1])  # the value: derivative by x_k times x_k
    for j in range(1, k + 1):
        L[j] = mul(L[j], coef_derivs[j - 1])
    L[k + 1] = mul(L[k + 1], coef_value)
    used = sum(1 for v in L[1:] if v is not None)
    return L[1:k + 1], L[k + 1], speelpenning, used


@pytest.mark.parametrize("row", rows("operation_counts_section3.txt"), ids=lambda r: f"k{r[0]}_d{r[1]}")
def test_operation_counts_sections3_1_3_2(row):
    k, d, speel_n, kernel2_n, cf_n, pow_n, mono_n, locations = (int(t) for t in row)
    rng = np.random.Generator(np.random.PCG64(1201 + 100 * k + d))
    n = k + 3
    pos = sorted(rng.choice(n, size=k, replace=False).tolist())
    a = rng.integers(1, d + 1, size=k).tolist()
    a[int(rng.integers(0, k))] = d  # d is the largest exponent
    coef = synth.random_cdd(rng, 1)
    s = synth.from_monomials(n, [[(pos, a)]], coef)
    pts = synth.points(1202 + k, n, 1)
    x = [fr(pts[v, 0]) for v in range(n)]
    c = fr(coef[0])

    mul = CountingMul()
    powers = {v: powers_model(mul, x[v], d) for v in pos}
    assert mul.n == k * max(d - 2, 0) and max(d - 2, 0) == pow_n
    mul.n = 0
    cf = common_factor_model(mul, [powers[v][aj - 1] for v, aj in zip(pos, a)])
    assert mul.n == cf_n == k - 1
    mul.n = 0
    coef_derivs = [cmul(c, (Fraction(aj), Fraction(0))) for aj in a]  # reading R2
    derivs, value, speel, used = second_kernel_model(mul, [x[v] for v in pos], cf, c, coef_derivs)
    assert speel == speel_n == 3 * k - 6
    assert mul.n == kernel2_n == 5 * k - 4
    assert used == locations == k + 1
    assert cf_n + kernel2_n == mono_n == 6 * k - 5

    f, J = E.evaluate_point(s, pts, 0)
    assert value == fr_exact(f[0])
    for j, v in enumerate(pos):
        assert derivs[j] == fr_exact(J[0][v])
