"""The FP32 collision sums the rational terms of the path-length coefficients from power
series when |x|max < 0.04 (c1 from 2/(2+x), c from the Gauss-Legendre ratio, the Omega+
Boole bracket of b in t = k x), truncated after x^6, and after x^4 when |x|max < 0.005.
This checks, on the CPU, that the truncated forms reproduce the oracle's exact
coefficients and path lengths below FP32 rounding on near-equilibrium states of both
lattices."""
import numpy as np
import pytest

import oracle as O

THRESHOLD = 0.04
SHORT_THRESHOLD = 0.005


def truncated(f, x, beta, b_variant, top=6):
    """The coefficients from the power sums M_k = <f, x^k> and S_k = <f, x^k>_{Omega-},
    k <= top (the higher ones taken as zero)."""
    M = {k: np.sum(f * x ** k) if k <= top else 0.0 for k in range(2, 7)}
    xm = np.minimum(x, 0.0)
    S = {k: np.sum(f * x ** 2 * xm ** (k - 2)) if k <= top else 0.0 for k in range(3, 7)}
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
@pytest.mark.parametrize("threshold,top,bounds", [
    # the dropped x^7.. terms at |x|max < 0.04: the path length moves by < 4e-8 of 2, half
    # an FP32 ulp
    (THRESHOLD, 6, dict(c1=4e-9, c=2e-8, b=6e-8, alpha_lower=4e-9, alpha_higher=5e-8)),
    # x^5 and x^6 dropped: |M5| <= |x|max^3 M2 = 1.25e-7 M2, so c1 and c move by at most
    # 1.6e-8 and 3.2e-8 of themselves, b by at most (2/15) 2 (0.375 (2x)^2 + ...) 2 x^3
    # ~ 0.8 |x|max^3 = 1e-7 of b1, and the path lengths stay below FP32 rounding
    (SHORT_THRESHOLD, 4, dict(c1=2e-8, c=4e-8, b=1e-7, alpha_lower=6e-8, alpha_higher=6e-8)),
])
def test_truncated_series_reproduce_the_closed_form(D, b_variant, threshold, top, bounds):
    rng = np.random.default_rng(71 + D + 5 * b_variant + top)
    worst = {}
    n = 0
    while n < 800:
        u = rng.uniform(-0.1, 0.1, D)
        # half the states at the top decade of |x|max, where the truncation bites most
        lo = np.log10(threshold) - (0.5 if n % 2 else 4.0)
        f = O.equilibrium(D, 1.0, u) * (1 + 10 ** rng.uniform(lo, np.log10(threshold)) * (2 * rng.random(3 ** D) - 1))
        r, uu = O.moments(D, f)
        feq = O.equilibrium(D, r, uu)
        x = O.departure(f, feq)
        if np.max(np.abs(x)) >= threshold:
            continue
        n += 1
        beta = rng.uniform(0.6, 0.9999)
        info = O.alpha(f, feq, beta, cutoff=False, b_variant=b_variant)
        got = truncated(f, x, beta, b_variant, top)
        ref = dict(c1=info.c1, c=info.c, b=info.b, alpha_lower=info.alpha_lower, alpha_higher=info.alpha_higher)
        scale = dict(c1=info.c1, c=info.c, b=info.b1, alpha_lower=2.0, alpha_higher=2.0)
        for k in ref:
            worst[k] = max(worst.get(k, 0.0), abs(got[k] - ref[k]) / abs(scale[k]))
    assert all(worst[k] < bounds[k] for k in bounds), worst
