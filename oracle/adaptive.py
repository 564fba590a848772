"""Adaptive-ABFT fault-coverage model and mode policy (Sec. 3.1.2, the
fault-coverage formulas FC_single / FC_full and Alg. alg-abft), written out in
plain Python from the paper.  Test infrastructure: only the tests, the smoke
check and the benchmark's CPU baseline use this package.

Model: errors of type 0D, 1D and 2D arrive as independent Poisson processes
with rates lambda_0D, lambda_1D, lambda_2D (per second); in one detection
interval of length T (one iteration of the decomposition) their counts are
Poisson(lambda T).  The matrix has S = (n / b)^2 blocks and each error strikes
a block uniformly at random.  Single-side checksums correct every 0D error as
long as no two strike the same block and there is no 1D or 2D error; full
checksums correct 0D and 1D errors under the same condition and no 2D error.

Reading of the product in the paper's formulas: the probability that k errors
strike k distinct blocks is prod_{i=0}^{k-1} (S - i) / S.  The paper prints
the product up to i = k, which would leave even a single error uncovered with
probability 1/S; the upper index is taken as k - 1.

The sums run over k = 0 .. S as printed; terms whose Poisson weight is below
1e-300 are not added (a numerical cut, not a change of the model).
"""
import math

NONE, SINGLE, FULL = 0, 1, 2


def _poisson_terms(mu, kmax):
    """[e^-mu mu^k / k!  for k = 0 .. K], K <= kmax, stopping once the terms
    past the mode fall below 1e-300."""
    out = []
    t = math.exp(-mu)
    k = 0
    while k <= kmax:
        if t == 0.0 and k > mu:
            break
        out.append(t)
        k += 1
        t = t * mu / k
        if t < 1e-300 and k > mu:
            break
    return out


def distinct_blocks(S, k):
    """prod_{i=0}^{k-1} (S - i) / S: k errors strike k distinct blocks."""
    p = 1.0
    for i in range(k):
        p *= (S - i) / S
    return p


def fc_single(S, mu0, mu1, mu2):
    """FC_single = (sum_{k=0}^{S} Pois(k; mu0) prod_{i<k} (S-i)/S) e^-mu1 e^-mu2,
    mu_t = lambda_t T."""
    s = 0.0
    for k, w in enumerate(_poisson_terms(mu0, S)):
        s += w * distinct_blocks(S, k)
    return s * math.exp(-mu1) * math.exp(-mu2)


def fc_full(S, mu0, mu1, mu2):
    """FC_full = (sum_{k=0}^{S} sum_{j=0}^{S-k} Pois(k; mu0) Pois(j; mu1)
    prod_{i<k+j} (S-i)/S) e^-mu2."""
    p0 = _poisson_terms(mu0, S)
    s = 0.0
    for k, w0 in enumerate(p0):
        for j, w1 in enumerate(_poisson_terms(mu1, S - k)):
            s += w0 * w1 * distinct_blocks(S, k + j)
    return s * math.exp(-mu2)


def adaptive_modes(n, nb, lambdas, fc_desired, step_seconds):
    """Alg. alg-abft without its clock loop: per step, NONE when every rate is
    zero, else SINGLE when FC_single >= FC_desired, else FULL when FC_full >=
    FC_desired, else FULL (the strongest check; the paper would lower the
    clock here, which is out of scope).  Returns (modes, coverage per step)."""
    S = (-(-n // nb)) ** 2
    l0, l1, l2 = lambdas
    modes, cov = [], []
    for T in step_seconds:
        if l0 <= 0.0 and l1 <= 0.0 and l2 <= 0.0:
            modes.append(NONE)
            cov.append(1.0)
            continue
        fs = fc_single(S, l0 * T, l1 * T, l2 * T)
        if fs >= fc_desired:
            modes.append(SINGLE)
            cov.append(fs)
            continue
        ff = fc_full(S, l0 * T, l1 * T, l2 * T)
        modes.append(FULL)
        cov.append(ff)
    return modes, cov
