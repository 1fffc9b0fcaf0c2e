"""Oracle of the policy network -- TEST INFRASTRUCTURE ONLY.

Float64 numpy restatement of the 12 -> 64 -> 64 -> 5 ReLU network and of the
gradient of its training loss, written out layer by layer from the chain
rule.  Only the test suite imports it (to check the CUDA training kernels'
gradients); the CUDA library shares no code with it.

Parameter vector layout (floats): W1 [64 x 12], b1 [64], W2 [64 x 64],
b2 [64], W3 [5 x 64], b3 [5], then the input normalisation mu [12], sd [12].
Loss of one sample: log(1 + exp(y0)) - t0 * y0 + wkc * (y1 - t1)^2 / 2
+ wmode * (log(sum_c exp(y_{2+c})) - y_{2+t2}) (binary cross-entropy on the
logit y0, a squared error on y1, and the softmax cross-entropy of the mode
logits y2..y4 against the class t2), averaged over the samples.
"""
import numpy as np

K_IN, K_H1, K_H2, K_OUT = 12, 64, 64, 5
K_MODES = 3
O_W1 = 0
O_B1 = O_W1 + K_H1 * K_IN
O_W2 = O_B1 + K_H1
O_B2 = O_W2 + K_H2 * K_H1
O_W3 = O_B2 + K_H2
O_B3 = O_W3 + K_OUT * K_H2
N_TRAINED = O_B3 + K_OUT
O_MU = N_TRAINED
O_SD = O_MU + K_IN
N_TOTAL = O_SD + K_IN


def unpack(P):
    P = np.asarray(P, dtype=np.float64)
    return (P[O_W1:O_B1].reshape(K_H1, K_IN), P[O_B1:O_W2], P[O_W2:O_B2].reshape(K_H2, K_H1),
            P[O_B2:O_W3], P[O_W3:O_B3].reshape(K_OUT, K_H2), P[O_B3:N_TRAINED], P[O_MU:O_SD],
            P[O_SD:N_TOTAL])


def forward(P, X):
    """Network outputs Y [n x 5] for raw inputs X [n x 12]."""
    W1, b1, W2, b2, W3, b3, mu, sd = unpack(P)
    Z = (np.asarray(X, np.float64) - mu) / sd
    H1 = np.maximum(Z @ W1.T + b1, 0.0)
    H2 = np.maximum(H1 @ W2.T + b2, 0.0)
    return H2 @ W3.T + b3


def _mode_ce(Ym, T2):
    """Softmax cross-entropy per sample of the mode logits Ym [n x 3]."""
    mx = Ym.max(axis=1)
    lse = mx + np.log(np.exp(Ym - mx[:, None]).sum(axis=1))
    return lse - Ym[np.arange(Ym.shape[0]), np.asarray(T2).astype(np.int64)]


def loss(P, X, T0, T1, T2, wkc, wmode):
    Y = forward(P, X)
    y0, y1 = Y[:, 0], Y[:, 1]
    softplus = np.maximum(y0, 0) + np.log1p(np.exp(-np.abs(y0)))
    return float(np.mean(softplus - np.asarray(T0) * y0 + 0.5 * wkc * (y1 - np.asarray(T1)) ** 2
                         + wmode * _mode_ce(Y[:, 2:2 + K_MODES], T2)))


def loss_and_grad(P, X, T0, T1, T2, wkc, wmode):
    """Mean loss and its gradient with respect to the trained parameters."""
    W1, b1, W2, b2, W3, b3, mu, sd = unpack(P)
    X = np.asarray(X, np.float64)
    T0 = np.asarray(T0, np.float64)
    T1 = np.asarray(T1, np.float64)
    n = X.shape[0]
    Z = (X - mu) / sd
    A1 = Z @ W1.T + b1
    H1 = np.maximum(A1, 0.0)
    A2 = H1 @ W2.T + b2
    H2 = np.maximum(A2, 0.0)
    Y = H2 @ W3.T + b3
    y0, y1 = Y[:, 0], Y[:, 1]
    Ym = Y[:, 2:2 + K_MODES]
    T2i = np.asarray(T2).astype(np.int64)
    softplus = np.maximum(y0, 0) + np.log1p(np.exp(-np.abs(y0)))
    L = float(np.mean(softplus - T0 * y0 + 0.5 * wkc * (y1 - T1) ** 2 + wmode * _mode_ce(Ym, T2i)))
    # output error: d/dy0 softplus(y0) = sigmoid(y0); d/dy of the softmax
    # cross-entropy = softmax(y) - one_hot(t2)
    Em = np.exp(Ym - Ym.max(axis=1, keepdims=True))
    Sm = Em / Em.sum(axis=1, keepdims=True)
    Sm[np.arange(n), T2i] -= 1.0
    dY = np.concatenate([(1.0 / (1.0 + np.exp(-y0)) - T0)[:, None], (wkc * (y1 - T1))[:, None], wmode * Sm],
                        axis=1) / n
    gW3 = dY.T @ H2
    gb3 = dY.sum(axis=0)
    dA2 = (dY @ W3) * (A2 > 0)
    gW2 = dA2.T @ H1
    gb2 = dA2.sum(axis=0)
    dA1 = (dA2 @ W2) * (A1 > 0)
    gW1 = dA1.T @ Z
    gb1 = dA1.sum(axis=0)
    g = np.concatenate([gW1.ravel(), gb1, gW2.ravel(), gb2, gW3.ravel(), gb3])
    return L, g


def init_params(rng, mu=None, sd=None):
    """He-style random initialisation (float64) with the given normalisation."""
    P = np.zeros(N_TOTAL)
    P[O_W1:O_B1] = rng.normal(0, np.sqrt(2.0 / K_IN), K_H1 * K_IN)
    P[O_W2:O_B2] = rng.normal(0, np.sqrt(2.0 / K_H1), K_H2 * K_H1)
    P[O_W3:O_B3] = rng.normal(0, np.sqrt(1.0 / K_H2), K_OUT * K_H2)
    P[O_MU:O_SD] = 0.0 if mu is None else mu
    P[O_SD:N_TOTAL] = 1.0 if sd is None else sd
    return P
