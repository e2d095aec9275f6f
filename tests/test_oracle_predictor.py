"""Pins of the predictor oracle (hierarchical grid interpolation, int8
network, residual round trip, entropy, straight-through gradients).

References independent of the oracle's code: exact predictions of linear
fields (an odd-sized grid has no clamping, so every fine point is predicted
exactly), hand-worked small examples, the round trip residual -> bins,
closed-form entropies, and torch autograd on the same forward pass for the
training gradients."""
import math

import numpy as np
import pytest
import torch

import oracle.predictor as PR


def test_linear_field_is_predicted_exactly():
    N = 17  # last coarse point is 16 for every stride: no clamping
    I, J, K = np.meshgrid(np.arange(N), np.arange(N), np.arange(N), indexing="ij")
    bins = (3 * I - 5 * J + 7 * K + 11).astype(np.int32).ravel()
    res = PR.residuals(bins, N)
    _, level = PR.predict(bins, N)
    assert np.all(res[level > 0] == 0)
    assert np.array_equal(res[level == 0], bins[level == 0])


def test_levels_and_classes_partition_the_grid():
    N = 20
    seen = np.zeros(N ** 3, dtype=int)
    for (lv, cls), (I, J, K) in PR.point_sets(N).items():
        s = PR.level_stride(lv)
        assert np.all((I % s == 0) & (J % s == 0) & (K % s == 0))
        odd = ((I // s) % 2) | (((J // s) % 2) << 1) | (((K // s) % 2) << 2)
        assert np.all(odd == cls)
        seen[(I * N + J) * N + K] += 1
    I, J, K = PR.anchor_points(N)
    seen[(I * N + J) * N + K] += 1
    assert np.all(seen == 1)


def test_hand_worked_predictions():
    N = 10
    b = np.zeros((N, N, N), dtype=np.int32)
    b[0, 0, 0], b[2, 0, 0] = 10, 15          # (1,0,0): stride 1, class 1
    b[0, 2, 0], b[2, 2, 0] = -7, 100         # (1,1,0): stride 1, class 3 with the above
    b[8, 0, 0] = 41                           # (9,0,0): the +1 neighbour clamps to 8
    b[0, 0, 4], b[0, 0, 8] = 2, 3             # (0,0,6): stride 2, class 4; (0,0,4): stride 4
    pred, level = PR.predict(b.ravel(), N)
    at = lambda i, j, k: pred[(i * N + j) * N + k]
    assert at(1, 0, 0) == (10 + 15 + 1) >> 1 == 13
    assert at(1, 1, 0) == (10 + 15 - 7 + 100 + 2) >> 2 == 30
    assert at(9, 0, 0) == (41 + 41 + 1) >> 1 == 41
    assert at(0, 0, 6) == (b[0, 0, 4] + b[0, 0, 8] + 1) >> 1 == 3   # stride 2 between 4 and 8
    assert at(0, 0, 4) == (10 + 3 + 1) >> 1 == 7                    # stride 4: corners (0,0,0), (0,0,8)
    assert level[(1 * N + 0) * N + 0] == 3 and level[(0 * N + 0) * N + 4] == 1


def test_negative_sums_round_down():
    N = 9
    b = np.zeros((N, N, N), dtype=np.int32)
    b[0, 0, 0], b[2, 0, 0] = -3, 0
    pred, _ = PR.predict(b.ravel(), N)
    assert pred[(1 * N) * N] == math.floor((-3 + 0 + 1) / 2) == -1


@pytest.mark.parametrize("N", [9, 16, 23])
def test_round_trip_interpolation_and_network(N):
    rng = np.random.default_rng(N)
    bins = rng.integers(-(1 << 30) + 1, 1 << 30, N ** 3).astype(np.int32)
    for params in (None, _random_params(rng)):
        res = PR.residuals(bins, N, params)
        assert np.array_equal(PR.reconstruct(res, N, params), bins)


def _random_params(rng, s_in=(2, 1, 0)):
    return PR.Params(rng.integers(-128, 128, (3, 7, 16, 27)), rng.integers(-5000, 5000, (3, 7, 16)),
                     rng.integers(-128, 128, (3, 7, 16)), rng.integers(-5000, 5000, (3, 7)), s_in, 8, 6)


def test_zero_network_is_interpolation():
    rng = np.random.default_rng(1)
    N = 16
    bins = rng.integers(-1000, 1000, N ** 3).astype(np.int32)
    assert np.array_equal(PR.residuals(bins, N, PR.Params.zeros((3, 2, 1))), PR.residuals(bins, N))


def test_single_path_network_closed_form():
    # W1 routes stencil input 13 (the floor-aligned coarse point itself) to
    # hidden unit 0 with weight 1; W2 passes h_0 with weight 1.  With s_in = 0,
    # s1 = s2 = 1: o = (clamp((x + 1) >> 1, 0, 127) + 1) >> 1, x = clamp(c13 - base).
    N = 9
    rng = np.random.default_rng(2)
    bins = rng.integers(-300, 300, N ** 3).astype(np.int32)
    W1 = np.zeros((3, 7, 16, 27), dtype=np.int64)
    W1[:, :, 0, 13] = 1
    W2 = np.zeros((3, 7, 16), dtype=np.int64)
    W2[:, :, 0] = 1
    p = PR.Params(W1, np.zeros((3, 7, 16)), W2, np.zeros((3, 7)), (0, 0, 0), 1, 1)
    base, level = PR.predict(bins, N)
    got, _ = PR.predict(bins, N, p)
    b3 = bins.reshape(N, N, N)
    for e in np.flatnonzero(level > 0)[:400]:
        i, j, k = np.unravel_index(e, (N, N, N))
        s = PR.level_stride(level[e])
        f = [(c // (2 * s)) * (2 * s) for c in (i, j, k)]
        x = min(127, max(-128, int(b3[f[0], f[1], f[2]]) - int(base[e])))
        h = min(127, max(0, (x + 1) // 2))
        assert got[e] == base[e] + (h + 1) // 2


def test_entropy_closed_forms():
    assert PR.entropy_bits(np.zeros(100)) == 0.0
    assert abs(PR.entropy_bits(np.arange(64).repeat(3)) - 6.0) < 1e-12
    assert abs(PR.entropy_bits(np.array([0, 0, 0, 1])) - (-(0.75 * math.log2(0.75) + 0.25 * math.log2(0.25)))) < 1e-12


def test_training_gradients_match_autograd():
    rng = np.random.default_rng(5)
    n = 2000
    x = rng.integers(-128, 128, (n, 27))
    base = rng.integers(-500, 500, n)
    target = base + rng.integers(-300, 300, n)
    w1 = rng.normal(0, 20, (16, 27))
    b1 = rng.normal(0, 2000, 16)
    w2 = rng.normal(0, 40, 16)
    b2 = rng.normal(0, 50, ())
    s1, s2 = 8, 6
    loss, g, _ = PR.train_forward_backward(x, base, target, w1, b1, w2, b2, s1, s2)
    T = lambda a: torch.tensor(a, dtype=torch.float64, requires_grad=True)
    tw1, tb1, tw2, tb2 = T(w1), T(b1), T(w2), T(b2)

    def ste(v, lo, hi):  # rint with identity gradient inside [lo, hi], clamp outside
        r = torch.round(v)
        inside = ((r >= lo) & (r <= hi)).double()
        return torch.clamp(r, lo, hi).detach() + (v - v.detach()) * inside

    W1q, B1q = ste(tw1, -128, 127), ste(tb1, -PR.B1_LIM, PR.B1_LIM)
    W2q, B2q = ste(tw2, -128, 127), ste(tb2, -PR.B1_LIM, PR.B1_LIM)
    X = torch.tensor(x, dtype=torch.float64)
    z = X @ W1q.T + B1q
    u = (z + 2.0 ** (s1 - 1)) / 2.0 ** s1
    hu = u + (torch.floor(u) - u).detach()
    on = ((hu > 0) & (hu < 127)).double()
    h = torch.clamp(hu, 0, 127).detach() + (hu - hu.detach()) * on
    v = (h @ W2q + B2q + 2.0 ** (s2 - 1)) / 2.0 ** s2
    o = v + (torch.floor(v) - v).detach()
    r = torch.tensor(target, dtype=torch.float64) - (torch.tensor(base, dtype=torch.float64) + o)
    L = (r * r).sum()
    assert abs(L.item() - loss) <= 1e-9 * max(1.0, loss)
    (L / n).backward()
    for name, tt in (("w1", tw1), ("b1", tb1), ("w2", tw2), ("b2", tb2)):
        np.testing.assert_allclose(g[name], tt.grad.numpy(), rtol=1e-9, atol=1e-12)
