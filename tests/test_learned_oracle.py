"""Pins of the learned-proposal oracle (oracle/mlp.py) against things other than itself:
finite differences of its own forward (pins the backward), numpy's Chebyshev Vandermonde matrix
(pins the basis), torch's BF16 conversion (pins the rounding), projector identities (pin the
target) and a hand-worked histogram (pins the features)."""
import math

import numpy as np
import pytest

from oracle import mlp as om


def test_bf16_rounding_matches_torch():
    torch = pytest.importorskip("torch")
    x = np.random.default_rng(0).standard_normal(4096) * np.exp(np.random.default_rng(1).uniform(-20, 20, 4096))
    ref = torch.tensor(x, dtype=torch.float32).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(om.bf16(x), ref)


def test_chebyshev_basis_spans_numpy_vandermonde():
    n, b = 200, 10.0
    Q = om.chebyshev_basis(n, b)
    x = (-b + (np.arange(n) + 0.5) * 2 * b / n) / b
    V = np.polynomial.chebyshev.chebvander(x, om.NCHEB - 1)
    assert np.abs(Q.T @ Q - np.eye(om.NCHEB)).max() < 1e-12
    # Gram-Schmidt in order: Q^T V is upper triangular with a positive diagonal, and Q Q^T V = V
    M = Q.T @ V
    assert np.abs(np.tril(M, -1)).max() < 1e-9 * np.abs(M).max()
    assert np.all(np.diag(M) > 0)
    assert np.abs(Q @ M - V).max() < 1e-9 * np.abs(V).max()


def test_target_is_a_projector_for_bases_inside_the_span():
    Q = om.chebyshev_basis(128, 10.0)
    A = np.random.default_rng(2).standard_normal((om.NCHEB, 7))
    Z, _ = np.linalg.qr(Q @ A)
    G = om.target(Q, Z)
    assert np.abs(G @ G - G).max() < 1e-12
    assert abs(np.trace(G) - 7) < 1e-12


def test_features_hand_worked():
    centres = np.array([[-5.0, 0.0, 4.99], [0.01, -4.9, 5.0], [7.0, 1.0, -9.0]])
    loga = np.array([math.log(0.5), math.log(4.0), math.log(100.0)])
    c = np.array([1.0, 2.0, 1.0])
    f = om.features(centres, loga, c, 5.0, math.log(0.5), math.log(20.0))
    # mode 0: x = -5 -> bin 0, 0.01 -> bin 32, 7 -> clipped to bin 63; weights 1, 2, 1 of 4
    assert f[0, 0] == 0.25 and f[0, 32] == 0.5 and f[0, 63] == 0.25
    # log a: log 0.5 -> bin 0; log 4 -> floor((log 8)/(log 40) * 64) = 36; log 100 -> 63
    q = int(math.floor(math.log(8.0) / math.log(40.0) * 64))
    assert f[0, 64 + 0] == 0.25 and f[0, 64 + q] == 0.5 and f[0, 64 + 63] == 0.25
    for l in range(3):
        assert abs(f[l, :64].sum() - 1) < 1e-15 and abs(f[l, 64:].sum() - 1) < 1e-15


def test_backward_matches_finite_differences():
    rng = np.random.default_rng(3)
    params = om.init_params(4)
    X = rng.uniform(0, 0.05, (2, 128))
    Q = om.chebyshev_basis(96, 10.0)
    Z, _ = np.linalg.qr(rng.standard_normal((96, 20)))
    G = np.stack([om.target(Q, Z)] * 2)

    def loss_of(p):
        Y, _ = om.forward(p, X, round_bf16=False)
        return om.loss_and_grad_output(Y, G)[0]

    Y, cache = om.forward(params, X, round_bf16=False)
    _, dY = om.loss_and_grad_output(Y, G)
    grads = om.backward(params, cache, dY, round_bf16=False)
    h = 1e-6
    for layer, which, idx in [(0, 0, (5, 17)), (1, 0, (100, 3)), (2, 1, (44,)), (3, 0, (2000, 500)),
                              (3, 1, (77,)), (0, 1, (9,))]:
        p_plus = [(W.copy(), b.copy()) for W, b in params]
        p_minus = [(W.copy(), b.copy()) for W, b in params]
        p_plus[layer][which][idx] += h
        p_minus[layer][which][idx] -= h
        fd = (loss_of(p_plus) - loss_of(p_minus)) / (2 * h)
        an = grads[layer][which][idx]
        assert abs(fd - an) <= 1e-6 * max(1.0, abs(an)), (layer, which, idx, fd, an)


def test_adam_first_step_moves_by_lr_times_sign():
    params = [(np.array([[1.0, -2.0]]), np.array([0.5]))]
    grads = [(np.array([[0.3, -4.0]]), np.array([1e-3]))]
    state = {}
    om.adam_step(params, grads, state, 0.01)
    # step 1: mhat = g, vhat = g^2, update = lr g / (|g| + 1e-8) ~ lr sign(g)
    assert np.allclose(params[0][0], [[0.99, -1.99]], atol=1e-9)
    assert np.allclose(params[0][1], [0.49], atol=1e-6)
