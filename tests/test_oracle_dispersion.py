"""Pins of the oracle's free-field dispersion solver (Sec. 2, App. A) against what
the paper prints: the Wilson relation solved for cosh(aE) in closed form, the
Brillouin relation as a quadratic in cosh(aE), the small-(am, ap) expansions
Eqs. free_wils, free_bril, over_wils, over_bril (the residual must shrink like
the sixth power of the scale), and the rho = (3 - sqrt 3)/2 cancellation of the
(am)^4 term of the overlap relations."""
import math

import numpy as np
import pytest

from oracle import dispersion

MOMENTA = [(0.0, 0.0, 0.0), (0.3, 0.0, 0.0), (0.4, 0.4, 0.0), (0.5, 0.5, 0.5), (1.1, 0.2, -0.7)]


@pytest.mark.parametrize("p", MOMENTA)
@pytest.mark.parametrize("am", [0.0, 0.1, 0.75])
def test_wilson_closed_form(p, am):
    """Sec. 2: 2 cosh(aE) [4 + am - sum cos p_i] = 1 + sum sin^2 p_i + [4 + am - sum cos p_i]^2."""
    w = 4.0 + am - sum(math.cos(x) for x in p)
    ch = (1.0 + sum(math.sin(x) ** 2 for x in p) + w * w) / (2.0 * w)
    assert dispersion.energy(p, am, "wil") == pytest.approx(math.acosh(ch), abs=1e-12)


@pytest.mark.parametrize("p", MOMENTA)
@pytest.mark.parametrize("am", [0.0, 0.1, 0.75])
def test_brillouin_quadratic(p, am):
    """Sec. 2 / App. A: the Brillouin relation as A cosh^2 + B cosh + C = 0 (the printed equation
    collected in powers of cosh); the oracle's energy is the arcosh of one of its roots."""
    c = [math.cos(x) for x in p]
    s = [math.sin(x) for x in p]
    ssum = sum(s[i] ** 2 * np.prod([(c[j] + 2.0) ** 2 for j in range(3) if j != i]) for i in range(3))
    p2 = np.prod([(ci + 2.0) ** 2 for ci in c])
    p1 = np.prod([ci + 1.0 for ci in c])
    m2 = 2.0 + am
    a = ssum / 729 - p2 / 729 + p1 ** 2 / 64
    b = 4 * ssum / 729 + 2 * p1 ** 2 / 64 - p1 * m2 / 4
    cc = 4 * ssum / 729 + p2 / 729 + p1 ** 2 / 64 - p1 * m2 / 4 + m2 ** 2
    e = dispersion.energy(p, am, "bri")
    ch = math.cosh(e)
    assert abs(a * ch * ch + b * ch + cc) <= 1e-12 * max(1.0, abs(b * ch), abs(cc))
    if abs(a) > 1e-12:
        roots = [(-b - math.sqrt(b * b - 4 * a * cc)) / (2 * a), (-b + math.sqrt(b * b - 4 * a * cc)) / (2 * a)]
        assert min(abs(ch - r) for r in roots) <= 1e-10


def _series(kind, overlap, am, p, rho=1.0):
    """(aE)^2 - (ap)^2 through O(a^5) (Eqs. free_wils, free_bril, over_wils, over_bril)."""
    pp = sum(x * x for x in p)
    quartic = sum(p[i] ** 2 * p[j] ** 2 for i in range(3) for j in range(i + 1, 3)) + sum(x ** 4 for x in p)
    if overlap:
        const = am ** 2 - (2 * rho ** 2 - 6 * rho + 3) / (6 * rho ** 2) * am ** 4
        if kind == "wil":
            return const - 2.0 / 3.0 * am ** 2 * pp - 2.0 / 3.0 * quartic
        return const
    const = am ** 2 - am ** 3 + 11.0 / 12.0 * am ** 4 - 5.0 / 6.0 * am ** 5
    if kind == "wil":
        return const + (-2.0 / 3.0 * am ** 2 + 7.0 / 6.0 * am ** 3) * pp + (-2.0 / 3.0 + am / 2.0) * quartic
    return const + am ** 3 / 12.0 * pp + am / 12.0 * quartic


@pytest.mark.parametrize("kind", ["wil", "bri"])
@pytest.mark.parametrize("overlap", [False, True])
@pytest.mark.parametrize("rho", [1.0, 0.7])
def test_small_momentum_expansions(kind, overlap, rho):
    """The residual against the printed expansion falls like scale^6 (halving the scale of
    am and ap divides it by about 64; a wrong coefficient at order 4 or 5 would give 16 or 32)."""
    if not overlap and rho != 1.0:
        pytest.skip("rho only enters the overlap relations")
    direction, m_ratio = np.array([0.9, 0.5, -0.3]), 0.8
    errs = []
    for scale in (0.08, 0.04, 0.02):
        p = tuple(scale * direction)
        am = scale * m_ratio
        e = dispersion.energy(p, am, kind, overlap=overlap, rho=rho)
        lhs = e * e - sum(x * x for x in p)
        errs.append(abs(lhs - _series(kind, overlap, am, p, rho)))
    assert errs[0] / errs[1] > 40 and errs[1] / errs[2] > 40, errs


@pytest.mark.parametrize("kind", ["wil", "bri"])
def test_magic_rho_removes_am4(kind):
    """Sec. 2: at rho = (3 - sqrt 3)/2 the (am)^4 term of the overlap relations vanishes, so at
    ap = 0 the residual (aE)^2 - (am)^2 is O((am)^6) there and O((am)^4) at rho = 1."""
    magic = (3.0 - math.sqrt(3.0)) / 2.0
    for am in (0.1, 0.05):
        e_magic = dispersion.energy((0.0, 0.0, 0.0), am, kind, overlap=True, rho=magic)
        e_one = dispersion.energy((0.0, 0.0, 0.0), am, kind, overlap=True, rho=1.0)
        assert abs(e_magic ** 2 - am ** 2) < 2 * am ** 6
        assert abs(e_one ** 2 - (am ** 2 - (2 - 6 + 3) / 6.0 * am ** 4)) < 2 * am ** 6
        assert abs(e_one ** 2 - am ** 2) > 0.1 * am ** 4
