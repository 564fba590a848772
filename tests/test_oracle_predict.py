"""The per-iteration time prediction (Sec. 3.2.1) and the Cholesky work
model: the oracle pinned by what the formula and the algorithm fix, and the
library's host functions checked against the oracle."""
import math

import numpy as np
import pytest

from oracle import predict as P


def test_weights_are_the_papers():
    assert P.WEIGHTS == (0.5, 0.25, 0.125, 0.125)
    assert sum(P.WEIGHTS) == 1.0


def test_constant_efficiency_is_predicted_exactly():
    """T_j = c W_j at every iteration: every prediction equals c W_k (the
    weights sum to one, and the renormalized early ones too)."""
    W = [1000.0 * (30 - k) ** 2 + 7.0 for k in range(30)]
    T = [3.5e-6 * w for w in W]
    pred = P.predict(T, W)
    assert math.isnan(pred[0])
    for k in range(1, 30):
        assert pred[k] == pytest.approx(T[k], rel=1e-12)


def test_hand_worked_example():
    # k = 4 uses all four neighbours: 1/2 (8/4) 2 + 1/4 (8/2) 5 + 1/8 (8/1) 1 + 1/8 (8/8) 3
    W = [8.0, 1.0, 2.0, 4.0, 8.0]
    T = [3.0, 1.0, 5.0, 2.0, 0.0]
    pred = P.predict(T, W)
    assert pred[4] == 0.5 * 2 * 2 + 0.25 * 4 * 5 + 0.125 * 8 * 1 + 0.125 * 1 * 3
    # k = 2: neighbours 1 and 0 with weights 1/2, 1/4 renormalized by 3/4
    assert pred[2] == pytest.approx((0.5 * 2 * 1 + 0.25 * (2 / 8) * 3) / 0.75, rel=1e-15)


def test_skips_iterations_without_work_or_measurement():
    W = [0.0, 4.0, 4.0, 4.0, 4.0, 4.0]
    T = [9.0, 2.0, -1.0, 2.0, 2.0, 2.0]
    pred = P.predict(T, W)
    # k = 5 uses j = 4, 3, 1 (j = 2 unmeasured): constant 2 over weights 1/2 1/4 1/8
    assert pred[5] == pytest.approx(2.0, rel=1e-15)
    assert math.isnan(P.predict([1.0], [0.0])[0])


def test_only_four_neighbours_are_used():
    W = [1.0] * 10
    T = [100.0] * 5 + [1.0] * 5
    assert P.predict(T, W)[9] == pytest.approx(1.0, rel=1e-15)
    assert P.predict(T, W)[8] == pytest.approx(0.875 + 0.125 * 100.0, rel=1e-15)


def brute_force_elements(n, nb, k):
    """Elements (i, j), i, j >= T0 with block(j) <= block(i), by enumeration."""
    T0 = min((k + 1) * nb, n)
    return sum(1 for i in range(T0, n) for j in range(T0, n) if (j - T0) // nb <= (i - T0) // nb)


@pytest.mark.parametrize("n,nb,k", [(10, 3, 0), (10, 3, 1), (17, 4, 2), (64, 16, 0), (65, 16, 3)])
def test_work_model_counts_the_block_triangle(n, nb, k):
    E = brute_force_elements(n, nb, k)
    K0 = k * nb
    kb = min(nb, n - K0)
    m = n - K0 - kb
    assert P.chol_work(n, nb, "tmu", k) == 2.0 * kb * E
    assert P.chol_work(n, nb, "verify", k) == E + m * kb
    assert P.chol_work(n, nb, "pu", k) == m * kb * kb
    assert P.chol_work(n, nb, "pd", k) == kb ** 3 / 3.0
    assert P.chol_work(n, nb, "tmu", (n + nb - 1) // nb) == 0.0


def test_library_predictor_matches_the_oracle():
    from paper_2301_03166_b300 import abft
    rng = np.random.default_rng(5)
    W = rng.uniform(0.0, 10.0, 40)
    W[[3, 17]] = 0.0
    T = rng.uniform(0.0, 2.0, 40)
    T[[8, 20]] = -1.0
    got = abft.predict_step_times(T, W)
    want = np.array(P.predict(list(T), list(W)))
    assert np.array_equal(np.isnan(got), np.isnan(want))
    ok = ~np.isnan(want)
    assert np.allclose(got[ok], want[ok], rtol=1e-14, atol=0.0)


@pytest.mark.parametrize("n,nb", [(1000, 128), (777, 64), (2048, 256)])
def test_library_work_model_matches_the_oracle(n, nb):
    from paper_2301_03166_b300 import abft
    for k in range((n + nb - 1) // nb + 1):
        for op in ("pd", "pu", "tmu", "verify"):
            assert abft.chol_step_work(n, nb, op, k) == P.chol_work(n, nb, op, k), (op, k)
