"""The kernels evaluate the smoothness indicators of the reconstruction
(Sec. 2.1, Eq. GHYZP) and of the limiter (Sec. 2.2) in rewritten forms that
are equal in exact arithmetic to the paper's. This checks, without a GPU,
that the identities hold symbolically and that every decimal constant the
kernel source carries for them equals its exact value to the digits given.
The parity tests compare the kernels' results with the oracle's on the GPU.
"""
import os
import re

import pytest

sympy = pytest.importorskip("sympy")
from sympy import Rational as R, sqrt, symbols, expand  # noqa: E402

SRC = os.path.join(os.path.dirname(__file__), os.pardir, "paper_2207_05258_gb300", "csrc",
                   "hweno_math.cuh")


def kernel_text():
    with open(SRC) as f:
        return f.read()


def literal_after(text, anchor, index=0):
    """The index-th decimal literal Real(x) in the statement that starts at
    the line containing `anchor`."""
    start = text.index(anchor)
    stmt = text[start:text.index(";", start)]
    lits = re.findall(r"Real\((-?[0-9.]+)\)", stmt)
    return float(lits[index]), lits[index]


def close(lit, exact, digits):
    """The decimal literal agrees with the exact value to `digits`
    significant digits (compared at 30 digits, not in double)."""
    x = sympy.Float(lit, 30)
    e = sympy.N(exact, 30)
    assert abs(x - e) <= sympy.Float(10) ** (1 - digits) * abs(e), (lit, e)


fm, f0, fp, Hm, H0, Hp = symbols("fm f0 fp Hm H0 Hp")
sHp, dHp, lap, dif = Hm + Hp, Hm - Hp, fm - 2 * f0 + fp, fm - fp
# the quintic's coefficients with dx absorbed into H (Sec. 2.1)
a1 = R(19, 192) * sHp + R(79, 48) * H0 + R(27, 64) * dif
a2 = R(3, 8) * dHp + R(5, 4) * lap
a3 = -(R(11, 24) * sHp + R(17, 6) * H0) - R(15, 8) * dif
a4 = -R(1, 4) * dHp - R(1, 2) * lap
a5 = R(1, 4) * sHp + H0 + R(3, 4) * dif


def test_first_square_of_beta0_is_the_derivative_value():
    assert expand(a1 + a3 / 4 + a5 / 16 - H0) == 0


def test_reconstruction_indicator_constants():
    text = kernel_text()
    K2, K3, K4 = sqrt(R(13, 3)), sqrt(R(781, 20)), sqrt(R(1421461, 2275))
    e2 = a2 + R(63, 130) * a4
    e3 = a3 + R(8825, 10934) * a5
    # E2 = sqrt(13/3) e2 in dHp, lap
    assert expand(e2 - (R(33, 130) * dHp + R(131, 130) * lap)) == 0
    for i, c in enumerate((K2 * R(33, 130), K2 * R(131, 130))):
        _, lit = literal_after(text, "const Real E2 = Real(0.528", i)
        close(lit, c, 19)
    # E3 = sqrt(781/20) e3 in sHp, H_i, dif
    c3 = (R(-16831, 65604), R(-33232, 16401), R(-27765, 21868))
    assert expand(e3 - (c3[0] * sHp + c3[1] * H0 + c3[2] * dif)) == 0
    for i, c in enumerate(c3):
        _, lit = literal_after(text, "const Real E3 =", i)
        close(lit, K3 * c, 19)
    # A4 = sqrt(1421461/2275) a4
    for i, c in enumerate((-R(1, 4), -R(1, 2))):
        _, lit = literal_after(text, "const Real A4 = Real(-6.249", i)
        close(lit, K4 * c, 19)
    # sqrt(13/3) on the inner sums of beta_1, beta_2
    _, lit = literal_after(text, "const Real kH =")
    close(lit, K2, 19)


def test_limiter_indicator_constants():
    text = kernel_text()
    um, u0, up, Vm, Vp = symbols("um u0 up Vm Vp")
    sV, dV, lapu, du = Vm + Vp, Vm - Vp, um - 2 * u0 + up, up - um
    q0 = R(3, 4) * du - R(1, 4) * sV
    a2l = R(1, 4) * dV + lapu
    a3l = R(1, 4) * sV - R(1, 4) * du
    a4l = -R(1, 4) * dV - R(1, 2) * lapu
    e2l = a2l + R(63, 130) * a4l
    assert expand(e2l - (R(67, 520) * dV + R(197, 260) * lapu)) == 0
    K2, K3, K4 = sqrt(R(13, 3)), sqrt(R(781, 20)), sqrt(R(1421461, 2275))
    for i, c in enumerate((K2 * R(67, 520), K2 * R(197, 260))):
        _, lit = literal_after(text, "const Real E2 = Real(0.268", i)
        close(lit, c, 19)
    _, lit = literal_after(text, "const Real A3 =")
    close(lit, K3 / 4, 19)
    _, lit = literal_after(text, "const Real e1 = q0 +")
    close(lit, R(1, 4) / K3, 19)
    # e1 = a1 + a3/4 with a1 = q0 and a3 = A3 / sqrt(781/20)
    assert expand((q0 + a3l / 4) - (q0 + (K3 * a3l) * (R(1, 4) / K3))) == 0
    for i, c in enumerate((-R(1, 4), -R(1, 2))):
        _, lit = literal_after(text, "const Real A4 = Real(-6.249", i)
        close(lit, K4 * c, 19)


def test_derivative_flux_is_the_sum_of_the_two_sides():
    fpm, fp0, fpp, Hpm, Hp0, Hpp, fm0, fm1, fm2, Hm0, Hm1, Hm2 = symbols(
        "fpm fp0 fpp Hpm Hp0 Hpp fm0 fm1 fm2 Hm0 Hm1 Hm2")
    Dp = R(1, 4) * (fpm - 8 * fp0 + 7 * fpp) + (Hpm - 2 * Hp0 - 5 * Hpp) / 12
    Dm = -(R(1, 4) * (fm2 - 8 * fm1 + 7 * fm0) + (-Hm2 + 2 * Hm1 + 5 * Hm0) / 12)
    text = kernel_text()
    start = text.index("their sum as one linear form")
    stmt = text[start:text.index(";", start)]
    terms = re.findall(r"([+-]?)\s*Real\(([0-9.]+(?:\s*/\s*[0-9.]+)?)\)\s*\*\s*(\w+)", stmt)
    assert len(terms) == 12
    names = dict(fpm=fpm, fp0=fp0, fpp=fpp, Hpm=Hpm, Hp0=Hp0, Hpp=Hpp, fm0=fm0, fm1=fm1,
                 fm2=fm2, Hm0=Hm0, Hm1=Hm1, Hm2=Hm2)
    total = 0
    for sign, coef, var in terms:
        num = sympy.nsimplify(coef.replace(" ", ""))
        total += (-1 if sign == "-" else 1) * num * names[var]
    assert expand(total - (Dp + Dm)) == 0


def test_adjoint_uses_the_same_indicator_constants():
    """The reverse passes take beta_0 in the same rewritten form; their named
    constants equal the exact values as well."""
    path = os.path.join(os.path.dirname(SRC), "hweno_adjoint.cuh")
    with open(path) as f:
        text = f.read()
    K2, K3, K4 = sqrt(R(13, 3)), sqrt(R(781, 20)), sqrt(R(1421461, 2275))
    want = dict(E2d=K2 * R(33, 130), E2l=K2 * R(131, 130), E3s=K3 * R(-16831, 65604),
                E3h=K3 * R(-33232, 16401), E3d=K3 * R(-27765, 21868), A4d=-K4 / 4, A4l=-K4 / 2)
    for name, exact in want.items():
        m = re.search(r"\b%s = (-?[0-9.]+)" % name, text)
        assert m, name
        close(m.group(1), exact, 19)
