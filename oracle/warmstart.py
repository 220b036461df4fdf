"""FP64 reference for the learned warm-start network: an MLP with GELU hidden layers, its
mean-squared-error loss, the gradient by backpropagation, and the Adam update.

TEST INFRASTRUCTURE ONLY.

Network: h_1 = GELU(W_1 u + b_1), h_2 = GELU(W_2 h_1 + b_2), p = W_3 h_2 + b_3 (linear output),
GELU(z) = z Phi(z) (the exact erf form).  Loss over a batch of B rows:
L = (1 / (B n_out)) sum_b ||p_b - t_b||^2.
Adam (Kingma & Ba, "Adam: a method for stochastic optimization", cited by the paper for the
surrogate training of Section 4.2): with gradient g at step t,
m <- beta1 m + (1 - beta1) g,  v <- beta2 v + (1 - beta2) g^2,
mhat = m / (1 - beta1^t),  vhat = v / (1 - beta2^t),  w <- w - lr mhat / (sqrt(vhat) + eps).
"""
import numpy as np

from .nn import act_value, act_d1


def forward(params, U):
    """U: (B, n_in).  Returns (P, cache) with P: (B, n_out)."""
    W1, b1, W2, b2, W3, b3 = params
    Z1 = U @ W1.T + b1
    H1 = act_value("gelu", Z1)
    Z2 = H1 @ W2.T + b2
    H2 = act_value("gelu", Z2)
    P = H2 @ W3.T + b3
    return P, (U, Z1, H1, Z2, H2)


def loss(params, U, T):
    P, _ = forward(params, U)
    return float(np.mean((P - T) ** 2))


def grad(params, U, T):
    """Gradient of `loss` with respect to (W1, b1, W2, b2, W3, b3), by backpropagation."""
    W1, b1, W2, b2, W3, b3 = params
    P, (U, Z1, H1, Z2, H2) = forward(params, U)
    B, n_out = T.shape
    dP = 2.0 * (P - T) / (B * n_out)
    dW3 = dP.T @ H2
    db3 = dP.sum(axis=0)
    dH2 = dP @ W3
    dZ2 = dH2 * act_d1("gelu", Z2)
    dW2 = dZ2.T @ H1
    db2 = dZ2.sum(axis=0)
    dH1 = dZ2 @ W2
    dZ1 = dH1 * act_d1("gelu", Z1)
    dW1 = dZ1.T @ U
    db1 = dZ1.sum(axis=0)
    return [dW1, db1, dW2, db2, dW3, db3]


def adam_step(params, grads, state, t, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update (in place) at step t >= 1; state = (m list, v list)."""
    m, v = state
    for i, (w, g) in enumerate(zip(params, grads)):
        m[i] = beta1 * m[i] + (1.0 - beta1) * g
        v[i] = beta2 * v[i] + (1.0 - beta2) * g * g
        mhat = m[i] / (1.0 - beta1 ** t)
        vhat = v[i] / (1.0 - beta2 ** t)
        w -= lr * mhat / (np.sqrt(vhat) + eps)
    return params, (m, v)


def init_state(params):
    return [np.zeros_like(p) for p in params], [np.zeros_like(p) for p in params]
