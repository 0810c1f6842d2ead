"""Multilayer perceptron and subspace-projector loss for the learned warm start
(TEST INFRASTRUCTURE ONLY).

Written out in float64 NumPy with the library's precision choices made explicit so that the
GPU kernels can be compared with it:

  * layer l:  z_l = bf16(h_{l-1}) @ bf16(W_l) + b_l,  h_l = tanh(z_l) (hidden layers),
              the last layer is linear.  bf16() rounds to the nearest bfloat16 (ties to even):
              weights and layer inputs are stored in bfloat16, sums and biases are not.
  * output:   one sample's output of length k*n is k column vectors of length n (vector j is
              entries j*n .. j*n+n-1), Y = [y_1 ... y_k] (n x k).
  * loss:     the squared Frobenius distance of orthogonal projectors, written without the
              n x n matrices:  ||Y Y^T - V V^T||_F^2 = ||Y^T Y||_F^2 - 2 ||V^T Y||_F^2 + ||V^T V||_F^2,
              for V (n x k) with orthonormal columns (the reference subspace).  It is invariant
              under Y -> Y R for orthogonal R (rotations and sign flips of the predicted
              vectors) and its gradient is dL/dY = 4 Y (Y^T Y) - 4 V (V^T Y).
  * the batch loss is the mean over samples divided by k.

Backward propagation is the chain rule written out layer by layer; the bfloat16 roundings are
treated as identity in the derivative (straight-through), as the kernels do.
"""
import numpy as np


def bf16(x):
    """Round float64/float32 values to the nearest bfloat16 (ties to even), returned as float64."""
    f = np.asarray(x, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    rounding = ((u >> 16) & 1) + 0x7FFF
    r = ((u + rounding) >> 16) << 16
    out = r.astype(np.uint32).view(np.float32).astype(np.float64)
    return np.where(np.isfinite(f), out, f.astype(np.float64))


def forward(Ws, bs, x, rounding=True):
    """Ws[l]: (in_l, out_l), bs[l]: (out_l,), x: (batch, in_0).  Returns (outputs, cache).
    rounding=False drops the bfloat16 roundings (exact float64 network)."""
    r = bf16 if rounding else (lambda a: a)
    hs = [np.asarray(x, dtype=np.float64)]
    zs = []
    for l, (W, b) in enumerate(zip(Ws, bs)):
        z = r(hs[-1]) @ r(W) + b
        zs.append(z)
        hs.append(np.tanh(z) if l < len(Ws) - 1 else z)
    return hs[-1], (hs, zs)


def projector_loss(out, Vs, k):
    """Mean over samples of ||Y Y^T - V V^T||_F^2 / k and its gradient with respect to out.
    out: (batch, k*n); Vs: (batch, n, k) with orthonormal columns."""
    B = out.shape[0]
    n = out.shape[1] // k
    loss = 0.0
    g = np.zeros_like(out)
    for s in range(B):
        Y = out[s].reshape(k, n).T          # n x k, vector j = entries j*n .. j*n+n-1
        V = Vs[s]
        YtY = Y.T @ Y
        VtY = V.T @ Y
        loss += (np.sum(YtY * YtY) - 2.0 * np.sum(VtY * VtY) + np.sum((V.T @ V) ** 2)) / k
        dY = (4.0 * Y @ YtY - 4.0 * V @ VtY) / k
        g[s] = dY.T.reshape(-1)
    return loss / B, g / B


def backward(Ws, bs, cache, gout, rounding=True):
    """Gradients (dWs, dbs) of the loss whose gradient with respect to the output is gout."""
    r = bf16 if rounding else (lambda a: a)
    hs, zs = cache
    L = len(Ws)
    dWs, dbs = [None] * L, [None] * L
    d = gout
    for l in range(L - 1, -1, -1):
        if l < L - 1:
            d = d * (1.0 - np.tanh(zs[l]) ** 2)
        dWs[l] = r(hs[l]).T @ r(d)
        dbs[l] = d.sum(axis=0)
        if l > 0:
            d = r(d) @ r(Ws[l]).T
    return dWs, dbs


def adam_step(p, g, m, v, t, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update (Kingma and Ba 2015, Algorithm 1) of the float parameter array p."""
    m[:] = beta1 * m + (1 - beta1) * g
    v[:] = beta2 * v + (1 - beta2) * g * g
    mh = m / (1 - beta1 ** t)
    vh = v / (1 - beta2 ** t)
    p[:] = p - lr * mh / (np.sqrt(vh) + eps)
    return p
