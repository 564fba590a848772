"""Enhanced algorithmic slack prediction (Sec. 3.2.1, the per-iteration time
formula with p = 4 and weights 1/2, 1/4, 1/8, 1/8) and the per-iteration work
of the blocked Cholesky, written out in plain Python.  Test infrastructure:
only the tests, the smoke check and the benchmark's CPU baseline use this
package.

The prediction of an operation's time at iteration k is the weighted sum,
over the previous iterations k - 1 .. k - 4 (nearest first), of the measured
time at that iteration scaled by the ratio of the operation's work at k to
its work there.  Readings: an iteration whose work is zero, or whose time is
not measured (negative), is skipped; when fewer than four neighbours are
usable (the first iterations), their weights are renormalized to sum to one,
so that an operation running at constant efficiency is predicted exactly; no
usable neighbour gives NaN.

Work per iteration (what the implementation performs): PD kb^3 / 3 flops,
PU m kb^2, TMU 2 kb E with E the elements of the trailing matrix's lower
block triangle (diagonal blocks full), verification E + m kb elements.
"""
import math

WEIGHTS = (0.5, 0.25, 0.125, 0.125)


def predict(T, W):
    """Predicted time per iteration from measured times T and work W."""
    out = []
    for k in range(len(T)):
        num = 0.0
        wsum = 0.0
        for i in range(1, 5):
            j = k - i
            if j < 0:
                break
            if not (W[j] > 0.0) or not (T[j] >= 0.0):
                continue
            num += WEIGHTS[i - 1] * (W[k] / W[j]) * T[j]
            wsum += WEIGHTS[i - 1]
        out.append(num / wsum if wsum > 0.0 else math.nan)
    return out


def chol_work(n, nb, op, k):
    """Work of operation op ('pd', 'pu', 'tmu', 'verify') at iteration k,
    counted element by element over the trailing block triangle."""
    K0 = k * nb
    if n <= 0 or nb <= 0 or k < 0 or K0 >= n:
        return 0.0
    kb = min(nb, n - K0)
    m = n - K0 - kb
    E = 0
    for i in range(m):            # row i of the trailing matrix
        last_col = (i // nb + 1) * nb
        E += min(last_col, m)     # columns 0 .. end of its diagonal block
    if op == "pd":
        return kb ** 3 / 3.0
    if op == "pu":
        return float(m * kb * kb)
    if op == "tmu":
        return 2.0 * kb * E
    if op == "verify":
        return float(E + m * kb)
    return 0.0
