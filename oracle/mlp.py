"""FP64 reference of the parameter-predicting MLP (no counterpart in the paper;
the nearest passage is the adaptive choice of N_p and N_S from the DOS
suggested in Sec. 6) - oracle side.

Network: x (n_in) -> tanh(W1 x + b1) (n_h) -> tanh(W2 h1 + b2) (n_h) -> W3 h2 + b3
(n_out = 3: log N_p, log n_s, kernel logit).  Loss for a batch of B samples
with targets t: mean over samples of (z0 - t0)^2 + (z1 - t1)^2 plus the binary
cross entropy of sigmoid(z2) against t2 in {0, 1}:
    L = (1/B) sum_b [ (z0-t0)^2 + (z1-t1)^2 + softplus(z2) - t2 z2 ].
Weights are row-major (out x in).
"""
import numpy as np


def init_params(n_in, n_h, n_out, seed):
    rs = np.random.default_rng(seed)
    return dict(
        W1=rs.uniform(-1, 1, (n_h, n_in)) * np.sqrt(3.0 / n_in), b1=np.zeros(n_h),
        W2=rs.uniform(-1, 1, (n_h, n_h)) * np.sqrt(3.0 / n_h), b2=np.zeros(n_h),
        W3=rs.uniform(-1, 1, (n_out, n_h)) * np.sqrt(3.0 / n_h), b3=np.zeros(n_out))


def forward(P, X):
    a1 = X @ P["W1"].T + P["b1"]
    h1 = np.tanh(a1)
    a2 = h1 @ P["W2"].T + P["b2"]
    h2 = np.tanh(a2)
    z = h2 @ P["W3"].T + P["b3"]
    return z, (X, h1, h2)


def softplus(x):
    return np.logaddexp(0.0, x)


def loss(P, X, T):
    z, _ = forward(P, X)
    B = X.shape[0]
    per = (z[:, 0] - T[:, 0]) ** 2 + (z[:, 1] - T[:, 1]) ** 2 + softplus(z[:, 2]) - T[:, 2] * z[:, 2]
    return float(per.sum() / B)


def loss_and_grad(P, X, T):
    """Loss and its gradient (dict like P) by backpropagation."""
    z, (X, h1, h2) = forward(P, X)
    B = X.shape[0]
    dz = np.zeros_like(z)
    dz[:, 0] = 2.0 * (z[:, 0] - T[:, 0]) / B
    dz[:, 1] = 2.0 * (z[:, 1] - T[:, 1]) / B
    dz[:, 2] = (1.0 / (1.0 + np.exp(-z[:, 2])) - T[:, 2]) / B
    g = {}
    g["W3"] = dz.T @ h2
    g["b3"] = dz.sum(axis=0)
    dh2 = dz @ P["W3"]
    da2 = dh2 * (1.0 - h2 ** 2)
    g["W2"] = da2.T @ h1
    g["b2"] = da2.sum(axis=0)
    dh1 = da2 @ P["W2"]
    da1 = dh1 * (1.0 - h1 ** 2)
    g["W1"] = da1.T @ X
    g["b1"] = da1.sum(axis=0)
    per = (z[:, 0] - T[:, 0]) ** 2 + (z[:, 1] - T[:, 1]) ** 2 + softplus(z[:, 2]) - T[:, 2] * z[:, 2]
    return float(per.sum() / B), g


def adam_step(P, G, state, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update (Kingma and Ba, 2015) in place; state holds m, v, t."""
    state["t"] = state.get("t", 0) + 1
    t = state["t"]
    for k in P:
        m = state.setdefault("m_" + k, np.zeros_like(P[k]))
        v = state.setdefault("v_" + k, np.zeros_like(P[k]))
        m[...] = beta1 * m + (1 - beta1) * G[k]
        v[...] = beta2 * v + (1 - beta2) * G[k] ** 2
        mh = m / (1 - beta1 ** t)
        vh = v / (1 - beta2 ** t)
        P[k] = P[k] - lr * mh / (np.sqrt(vh) + eps)
    return P
