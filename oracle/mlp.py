"""Plain NumPy restatement of the warm-start network (oracle for the GPU kernels).

MLP with GELU hidden activations (GELU(z) = z Phi(z), Phi the standard normal CDF),
mean-squared-error loss and Adam (Kingma & Ba, 2015).  FP64 here; the GPU kernels run
in FP32.  Test infrastructure only."""
import numpy as np
from scipy.special import erf


def gelu(z):
    return 0.5 * z * (1.0 + erf(z / np.sqrt(2.0)))


def gelu_grad(z):
    return 0.5 * (1.0 + erf(z / np.sqrt(2.0))) + z * np.exp(-0.5 * z * z) / np.sqrt(2.0 * np.pi)


def forward(params, X):
    """params: list of (W [fan_in, fan_out], b [fan_out]); returns output and cache."""
    cache = []
    H = X
    for li, (W, b) in enumerate(params):
        Z = H @ W + b
        last = li == len(params) - 1
        cache.append((H, Z))
        H = Z if last else gelu(Z)
    return H, cache


def loss_and_grads(params, X, T):
    Y, cache = forward(params, X)
    n = Y.size
    loss = np.mean((Y - T) ** 2)
    dH = 2.0 * (Y - T) / n
    grads = [None] * len(params)
    for li in range(len(params) - 1, -1, -1):
        Hin, Z = cache[li]
        dZ = dH if li == len(params) - 1 else dH * gelu_grad(Z)
        grads[li] = (Hin.T @ dZ, dZ.sum(0))
        dH = dZ @ params[li][0].T
    return loss, grads


def adam(w, g, m1, m2, step, lr, b1=0.9, b2=0.999, eps=1e-8):
    m1 = b1 * m1 + (1 - b1) * g
    m2 = b2 * m2 + (1 - b2) * g * g
    w = w - lr * (m1 / (1 - b1**step)) / (np.sqrt(m2 / (1 - b2**step)) + eps)
    return w, m1, m2
