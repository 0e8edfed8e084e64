"""FP64 CPU reference of the learned warm-start network (test infrastructure only).

The network maps the features z = (sigma, ell, sqrt(lambda_1), ..., sqrt(lambda_M)) of an SG
system to its chaos-coefficient field X (N x P, flattened): after the input standardisation
z_hat = (z - mu) / sd it is
    h1 = tanh(W1 z_hat + b1),  h2 = tanh(W2 h1 + b2),  y = W3 h2 + b3,
trained on the mean squared error  L = sum_{b,j} (y_bj - t_bj)^2 / (B D).
Gradients follow the chain rule through these three layers.  Weights are stored row-major with
shape (out, in).  Nothing here is shared with the CUDA library.
"""

import numpy as np


def forward(params, Z, mu, sd):
    W1, b1, W2, b2, W3, b3 = params
    Zh = (Z - mu) / sd
    H1 = np.tanh(Zh @ W1.T + b1)
    H2 = np.tanh(H1 @ W2.T + b2)
    Y = H2 @ W3.T + b3
    return Y, (Zh, H1, H2)


def loss_and_grads(params, Z, T, mu, sd):
    """Mean squared error and its gradient with respect to (W1, b1, W2, b2, W3, b3)."""
    W1, b1, W2, b2, W3, b3 = params
    Y, (Zh, H1, H2) = forward(params, Z, mu, sd)
    B, D = Y.shape
    R = Y - T
    loss = float(np.sum(R * R) / (B * D))
    dY = 2.0 * R / (B * D)
    gW3 = dY.T @ H2
    gb3 = dY.sum(axis=0)
    dH2 = dY @ W3
    dA2 = dH2 * (1.0 - H2 * H2)
    gW2 = dA2.T @ H1
    gb2 = dA2.sum(axis=0)
    dH1 = dA2 @ W2
    dA1 = dH1 * (1.0 - H1 * H1)
    gW1 = dA1.T @ Zh
    gb1 = dA1.sum(axis=0)
    return loss, [gW1, gb1, gW2, gb2, gW3, gb3]


def adam_step(params, grads, m, v, t, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam step (Kingma & Ba 2015) with bias correction; t counts from 1."""
    out = []
    for i, (p, g) in enumerate(zip(params, grads)):
        m[i] = beta1 * m[i] + (1 - beta1) * g
        v[i] = beta2 * v[i] + (1 - beta2) * g * g
        mh = m[i] / (1 - beta1 ** t)
        vh = v[i] / (1 - beta2 ** t)
        out.append(p - lr * mh / (np.sqrt(vh) + eps))
    return out
