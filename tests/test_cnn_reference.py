"""The CPU convolution reference pinned to brute-force sums and to the
adjoint identities that define its gradients."""
import numpy as np
import pytest

from oracle import cnn_reference as ref


def brute_conv(x, w, b, stride, pad):
    N, H, W, C = x.shape
    K, R, S, _ = w.shape
    P, Q = (H + 2 * pad - R) // stride + 1, (W + 2 * pad - S) // stride + 1
    y = np.zeros((N, P, Q, K))
    for n in range(N):
        for p in range(P):
            for q in range(Q):
                for k in range(K):
                    s = b[k]
                    for r in range(R):
                        for t in range(S):
                            h, v = p * stride + r - pad, q * stride + t - pad
                            if 0 <= h < H and 0 <= v < W:
                                s += float(np.dot(x[n, h, v], w[k, r, t]))
                    y[n, p, q, k] = s
    return y


@pytest.mark.parametrize("stride,pad,R", [(1, 1, 3), (2, 1, 3), (2, 0, 3), (1, 0, 1)])
def test_forward_is_the_cross_correlation(stride, pad, R):
    rng = np.random.default_rng(stride * 10 + pad)
    x = rng.standard_normal((2, 7, 6, 3))
    w = rng.standard_normal((4, R, R, 3))
    b = rng.standard_normal(4)
    want = brute_conv(x, w, b, stride, pad)
    assert np.allclose(ref.conv_forward(x, w, b, stride, pad, False), want, atol=1e-12)
    assert np.allclose(ref.conv_forward(x, w, b, stride, pad, True), np.maximum(want, 0), atol=1e-12)


@pytest.mark.parametrize("stride,pad", [(1, 1), (2, 1), (2, 0)])
def test_gradients_are_the_adjoints(stride, pad):
    # conv is affine in x and in (w, b): <dy, conv(x, w, 0)> = <dx, x> and
    # <dy, conv(x, w, b)> = <dw, w> + <db, b>
    rng = np.random.default_rng(stride + 7 * pad)
    x = rng.standard_normal((2, 9, 8, 3))
    w = rng.standard_normal((5, 3, 3, 3))
    b = rng.standard_normal(5)
    y = brute_conv(x, w, np.zeros(5), stride, pad)
    dy = rng.standard_normal(y.shape)
    dx, dw, db = ref.conv_grads(x, w, b, stride, pad, dy)
    lhs = float((dy * y).sum())
    assert np.isclose(lhs, float((dx * x).sum()), rtol=1e-12)
    assert np.isclose(lhs, float((dw * w).sum()), rtol=1e-12)
    assert np.allclose(db, dy.sum(axis=(0, 1, 2)), atol=1e-12)
    # one filter-gradient entry by brute force
    k, r, t, c = 2, 1, 2, 0
    s = 0.0
    for n in range(2):
        for p in range(y.shape[1]):
            for q in range(y.shape[2]):
                h, v = p * stride + r - pad, q * stride + t - pad
                if 0 <= h < 9 and 0 <= v < 8:
                    s += dy[n, p, q, k] * x[n, h, v, c]
    assert np.isclose(dw[k, r, t, c], s, rtol=1e-12)
