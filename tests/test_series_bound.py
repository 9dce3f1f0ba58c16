"""The FP32 collision sums the rational terms of the path-length coefficients from power
series when |x|max < 0.02 (c1 from 2/(2+x), c from the Gauss-Legendre ratio, the Omega+
Boole bracket of b in t = k x), truncated after x^6.  This checks, on the CPU, that the
truncated forms reproduce the oracle's exact coefficients and path lengths far below FP32
rounding on near-equilibrium states of both lattices."""
import numpy as np
import pytest

import oracle as O

THRESHOLD = 0.02


def truncated(f, x, beta, b_variant):
    M = {k: np.sum(f * x ** k) for k in range(2, 7)}
    xm = np.minimum(x, 0.0)
    S = {k: np.sum(f * x ** 2 * xm ** (k - 2)) for k in range(3, 7)}
    b1 = 0.5 * M[2]
    c1 = M[2] - M[3] / 2 + M[4] / 4 - M[5] / 8 + M[6] / 16
    c = M[2] - M[3] / 2 + M[4] / 3 - M[5] / 4 + M[6] / 5
    root = lambda a, b, cc: 2 * cc / (b + np.sqrt(b * b - 4 * a * cc))
    aL = root(S[3] / 2, b1, c1)
    kk = aL if b_variant == O.B_PRINTED else aL * beta
    P = {m: M[m] - S[m] for m in range(3, 7)}
    bsum = 1.25 * P[3] + kk * (-0.625 * P[4] + kk * (0.375 * P[5] + kk * (-0.25 * P[6])))
    b = b1 - (2 / 15) * aL * beta ** 2 * bsum
    h = root(beta ** 2 * S[3] / 6, b, c)
    hb = h * beta
    a = beta ** 2 * (S[3] / 6 - hb * S[4] / 12 + hb ** 2 * S[5] / 20 - hb ** 3 * S[6] / 5)
    return dict(c1=c1, c=c, b=b, alpha_lower=aL, alpha_higher=root(a, b, c))


@pytest.mark.parametrize("D", [2, 3])
@pytest.mark.parametrize("b_variant", [O.B_DERIVED, O.B_PRINTED])
def test_truncated_series_reproduce_the_closed_form(D, b_variant):
    rng = np.random.default_rng(71 + D + 5 * b_variant)
    worst = {}
    n = 0
    while n < 800:
        u = rng.uniform(-0.1, 0.1, D)
        f = O.equilibrium(D, 1.0, u) * (1 + 10 ** rng.uniform(-4, np.log10(THRESHOLD)) * (2 * rng.random(3 ** D) - 1))
        r, uu = O.moments(D, f)
        feq = O.equilibrium(D, r, uu)
        x = O.departure(f, feq)
        if np.max(np.abs(x)) >= THRESHOLD:
            continue
        n += 1
        beta = rng.uniform(0.6, 0.9999)
        info = O.alpha(f, feq, beta, cutoff=False, b_variant=b_variant)
        got = truncated(f, x, beta, b_variant)
        ref = dict(c1=info.c1, c=info.c, b=info.b, alpha_lower=info.alpha_lower, alpha_higher=info.alpha_higher)
        scale = dict(c1=info.c1, c=info.c, b=info.b1, alpha_lower=2.0, alpha_higher=2.0)
        for k in ref:
            worst[k] = max(worst.get(k, 0.0), abs(got[k] - ref[k]) / abs(scale[k]))
    assert worst["c1"] < 1e-9 and worst["c"] < 1e-9 and worst["b"] < 1e-8, worst
    assert worst["alpha_lower"] < 1e-9 and worst["alpha_higher"] < 1e-8, worst
