"""Pins of the learned-warm-start oracle (CPU): BF16 rounding against its definition and a
library conversion, backpropagation against finite differences, Adam's first step against
its closed form, the expanded warm-start loss against the decoded residual it stands for."""
import numpy as np
import pytest
import torch

from oracle import learned as O


def test_bf16_round_ties_to_even_and_specials():
    one = 1.0
    ulp = 2.0 ** -7                      # spacing of BF16 numbers in [1, 2)
    cases = {
        one: one,
        one + ulp / 2: one,              # tie -> even mantissa (0)
        one + 1.5 * ulp: one + 2 * ulp,  # tie -> even mantissa (2)
        one + 0.75 * ulp: one + ulp,
        -(one + 0.25 * ulp): -one,
        float("nan"): 0.0,
        float("inf"): 0.0,
    }
    for x, want in cases.items():
        got = O.bf16_round(np.array([x]))[0]
        assert got == want or np.isclose(got, want, rtol=2 ** -8), (x, got, want)
    assert O.bf16_bits(np.array([1.0]))[0] == 0x3F80
    assert O.bf16_bits(np.array([-2.0]))[0] == 0xC000
    assert O.from_bf16_bits(np.array([0x3F80, 0x4049]))[1] == 3.140625


def test_bf16_round_matches_torch_on_random_floats():
    rng = np.random.default_rng(0)
    x = np.concatenate([rng.standard_normal(20000) * 10.0 ** rng.integers(-20, 20, 20000),
                        rng.standard_normal(1000)]).astype(np.float32).astype(np.float64)
    ours = O.bf16_round(x)
    ref = torch.from_numpy(x.astype(np.float32)).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(ours, ref)


def _net(rng, dims):
    Ws = [rng.standard_normal((dims[l + 1], dims[l])) / np.sqrt(dims[l]) for l in range(len(dims) - 1)]
    bs = [0.1 * rng.standard_normal(dims[l + 1]) for l in range(len(dims) - 1)]
    return Ws, bs


def test_backprop_matches_central_differences():
    rng = np.random.default_rng(1)
    dims = [5, 7, 6, 3]
    Ws, bs = _net(rng, dims)
    X = rng.standard_normal((4, dims[0]))
    T = rng.standard_normal((4, dims[-1]))

    def loss(Ws_, bs_):
        Y, _ = O.mlp_forward(Ws_, bs_, X, bf16=False)
        return 0.5 * np.sum((Y - T) ** 2)

    Y, hs = O.mlp_forward(Ws, bs, X, bf16=False)
    gW, gb = O.mlp_backward(Ws, hs, Y - T, bf16=False)
    h = 1e-6
    for l in range(len(Ws)):
        for idx in [(0, 0), (dims[l + 1] - 1, dims[l] - 1), (1, 2)]:
            Wp = [w.copy() for w in Ws]
            Wm = [w.copy() for w in Ws]
            Wp[l][idx] += h
            Wm[l][idx] -= h
            fd = (loss(Wp, bs) - loss(Wm, bs)) / (2 * h)
            assert abs(fd - gW[l][idx]) <= 1e-6 * max(1.0, abs(fd)), (l, idx, fd, gW[l][idx])
        bp = [b.copy() for b in bs]
        bm = [b.copy() for b in bs]
        bp[l][0] += h
        bm[l][0] -= h
        fd = (loss(Ws, bp) - loss(Ws, bm)) / (2 * h)
        assert abs(fd - gb[l][0]) <= 1e-6 * max(1.0, abs(fd))


def test_bf16_network_rounds_hidden_activations():
    rng = np.random.default_rng(2)
    Ws, bs = _net(rng, [8, 16, 4])
    X = O.bf16_round(rng.standard_normal((3, 8)))
    _, hs = O.mlp_forward(Ws, bs, X, bf16=True)
    assert np.array_equal(hs[1], O.bf16_round(hs[1]))
    assert np.all(hs[1] >= 0)


def test_adam_first_step_closed_form():
    rng = np.random.default_rng(3)
    W = rng.standard_normal(50)
    g = rng.standard_normal(50)
    lr, eps = 1e-3, 1e-8
    W1, m, v = O.adam(W, np.zeros(50), np.zeros(50), g, 1, lr, 0.9, 0.999, eps)
    # m_hat = g and v_hat = g^2 at t = 1
    assert np.allclose(W1, W - lr * g / (np.abs(g) + eps), rtol=0, atol=1e-15)
    assert np.allclose(m, 0.1 * g) and np.allclose(v, 0.001 * g * g)


def test_ws_loss_equals_decoded_residual_and_its_gradient():
    rng = np.random.default_rng(4)
    D, r, B = 300, 12, 5
    Phi = rng.standard_normal((D, r)) / 4.0
    mu = rng.standard_normal(D)
    Zs = mu[None, :] + rng.standard_normal((B, D))
    alpha, E, w_sigma = 0.7, 3.0, 2.0
    G = Phi.T @ Phi
    R = Phi.T @ (Zs - mu[None, :]).T
    dd = np.sum((Zs - mu[None, :]) ** 2, axis=1)
    s = rng.standard_normal(B)
    Out = rng.standard_normal((B, 1 + r + 3))
    dO, ls, ll = O.ws_loss(Out, G, R, dd, s, alpha, E, w_sigma, r)
    # the expanded form equals the decoded residual (no clipping)
    Z0 = O.decode(Phi, mu, alpha * Out[:, 1:1 + r] / alpha, alpha, np.full(D, -np.inf), np.full(D, np.inf))
    direct = np.mean(np.sum((Z0 - Zs) ** 2, axis=1)) / (2 * E)
    assert abs(ll - direct) <= 1e-10 * direct
    assert abs(ls - np.mean(0.5 * w_sigma * (Out[:, 0] - s) ** 2)) <= 1e-12
    assert np.all(dO[:, 1 + r:] == 0)

    def total(Ov):
        _, a, b = O.ws_loss(Ov, G, R, dd, s, alpha, E, w_sigma, r)
        return a + b

    h = 1e-6
    for idx in [(0, 0), (1, 1), (4, r), (2, 5)]:
        P = Out.copy()
        M = Out.copy()
        P[idx] += h
        M[idx] -= h
        fd = (total(P) - total(M)) / (2 * h)
        assert abs(fd - dO[idx]) <= 1e-6 * max(1.0, abs(fd))
    # the least-squares latent is a stationary point
    ell_ls = np.linalg.solve(G, R)            # (r, B)
    Out2 = Out.copy()
    Out2[:, 1:1 + r] = ell_ls.T / alpha
    dO2, _, _ = O.ws_loss(Out2, G, R, dd, s, alpha, E, w_sigma, r)
    assert np.max(np.abs(dO2[:, 1:1 + r])) <= 1e-10


def test_decode_clips_into_bounds():
    rng = np.random.default_rng(5)
    D, r = 40, 3
    Phi = rng.standard_normal((D, r))
    mu = rng.standard_normal(D)
    lo = np.full(D, -0.5)
    hi = np.full(D, 0.5)
    lo[:10] = -np.inf
    Z = O.decode(Phi, mu, rng.standard_normal((2, r)), 1.3, lo, hi)
    assert np.all(Z <= 0.5) and np.all(Z[:, 10:] >= -0.5)
    ell = rng.standard_normal((2, r))
    Z = O.decode(Phi, mu, ell, 1.3, lo, hi)
    raw = mu[None, :] + 1.3 * (ell @ Phi.T)
    free = (raw > lo[None, :]) & (raw < hi[None, :])
    assert np.allclose(Z[free], raw[free], rtol=1e-15, atol=1e-15)


def test_standardize_gives_zero_mean_unit_variance():
    rng = np.random.default_rng(6)
    F = 3.0 + 2.0 * rng.standard_normal((7, 500))
    mu, istd = O.row_stats(F, 1e-12)
    X = (F - mu[:, None]) * istd[:, None]
    assert np.allclose(X.mean(axis=1), 0, atol=1e-12)
    assert np.allclose(X.std(axis=1), 1, atol=1e-12)
    assert np.array_equal(O.standardize(F, mu, istd), O.bf16_round(X.T))


def test_planted_mistake_is_caught():
    """Backprop with the ReLU mask dropped disagrees with central differences."""
    rng = np.random.default_rng(10)
    dims = [4, 6, 2]
    Ws, bs = _net(rng, dims)
    bs[0] -= 0.5                       # some hidden units inactive
    X = rng.standard_normal((5, 4))
    Y, hs = O.mlp_forward(Ws, bs, X, bf16=False)
    assert np.any(hs[1] == 0)
    wrong = (Y @ Ws[1]).T @ hs[0]      # first-layer gradient without the mask
    gW, _ = O.mlp_backward(Ws, hs, Y, bf16=False)
    assert not np.allclose(wrong, gW[0])
