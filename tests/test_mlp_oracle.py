"""Pin of the perceptron oracle: analytic gradient = central finite differences."""
import numpy as np

from oracle import mlp_oracle as M


def test_gradient_matches_finite_differences():
    rng = np.random.default_rng(3)
    dims = [5, 7, 6, 4]
    n = sum(dims[l] * dims[l + 1] + dims[l + 1] for l in range(len(dims) - 1))
    p = rng.normal(scale=0.5, size=n)
    x = rng.normal(size=(9, 5))
    t = rng.normal(size=(9, 4))
    loss, g = M.loss_and_grad(p, dims, x, t)
    h = 1e-6
    for idx in rng.choice(n, 25, replace=False):
        e = np.zeros(n)
        e[idx] = h
        fd = (M.loss_and_grad(p + e, dims, x, t)[0] - M.loss_and_grad(p - e, dims, x, t)[0]) / (2 * h)
        assert abs(fd - g[idx]) <= 1e-7 * max(1.0, abs(fd)), idx


def test_bf16_rounding_is_round_to_nearest_even():
    x = np.array([1.0, 1.0 + 2 ** -8, 1.0 + 3 * 2 ** -9, -3.140625, 1e-3], dtype=np.float32)
    r = M.bf16_round(x)
    assert r[0] == 1.0
    assert r[1] == 1.0 + 2 ** -7 or r[1] == 1.0       # tie -> even mantissa
    assert r[1] == 1.0                                  # 1 + 2^-8 is a tie; even is 1.0
    assert r[2] == 1.0 + 2 ** -7                        # above the tie -> up
    assert r[3] == -3.140625
    assert abs(r[4] - 1e-3) <= 1e-3 * 2 ** -8
