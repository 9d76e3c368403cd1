"""FP64 reference of the troubled-cell indicator network (test infrastructure).

Network: 24 -> 64 -> 64 -> 64 -> 1, ReLU hidden layers, one logit out; a cell is
flagged when the logit is positive (sigmoid > 1/2).  Parameters are one flat FP32
vector in the order W1 [64x24], b1 [64], W2 [64x64], b2, W3 [64x64], b3, W4 [1x64],
b4 [1] (row-major, W[out][in]).  The weights the network computes with are the
bfloat16 roundings (round to nearest even) of the master values.
Loss: binary cross-entropy on the logit with a weight on positive labels.
Pinned in the tests by central differences of the loss (gradient), hand-computable
networks (forward), torch's float32 -> bfloat16 conversion (rounding) and the
first-step property of bias-corrected Adam.
"""
import numpy as np

SIZES = [(64, 24), (64, 64), (64, 64), (1, 64)]
N_PARAMS = sum(o * i + o for o, i in SIZES)


def bf16(x):
    """Round FP32 values to bfloat16 (nearest, ties to even), returned as float64."""
    f = np.ascontiguousarray(np.asarray(x, dtype=np.float32))
    b = f.view(np.uint32).astype(np.uint64)
    lsb = (b >> 16) & 1
    r = ((b + 0x7FFF + lsb) >> 16) << 16
    out = (r & 0xFFFFFFFF).astype(np.uint32).view(np.float32).astype(np.float64)
    return out.reshape(np.shape(x))


def unpack(theta):
    theta = np.asarray(theta, dtype=np.float64)
    out, o = [], 0
    for (n_out, n_in) in SIZES:
        W = theta[o:o + n_out * n_in].reshape(n_out, n_in)
        o += n_out * n_in
        b = theta[o:o + n_out]
        o += n_out
        out.append((W, b))
    return out


def forward(theta, X, weights_bf16=True, act_bf16=False):
    """Logits [n] and the activations needed by backward.  act_bf16 rounds the input
    and every hidden activation to bfloat16 (what tensor-core inference sees)."""
    layers = unpack(bf16(theta) if weights_bf16 else theta)
    A = [bf16(X) if act_bf16 else np.asarray(X, dtype=np.float64)]
    for li, (W, b) in enumerate(layers):
        Z = A[-1] @ W.T + b
        if li < len(layers) - 1:
            H = np.maximum(Z, 0.0)
            A.append(bf16(H) if act_bf16 else H)
        else:
            A.append(Z[:, 0])
    return A[-1], A


def loss_and_grad(theta, X, y, pos_weight=1.0, weights_bf16=True):
    """Mean weighted BCE-with-logits and its gradient w.r.t. the (bf16-rounded) parameters."""
    z, A = forward(theta, X, weights_bf16)
    layers = unpack(bf16(theta) if weights_bf16 else theta)
    y = np.asarray(y, dtype=np.float64)
    n = X.shape[0]
    sig = 1.0 / (1.0 + np.exp(-z))
    # L_i = -pw y log s - (1-y) log(1-s) ;  dL/dz = s (pw y + 1 - y) - pw y
    logs = -np.logaddexp(0.0, -z)
    log1ms = -np.logaddexp(0.0, z)
    loss = float(np.mean(-pos_weight * y * logs - (1 - y) * log1ms))
    dZ = ((sig * (pos_weight * y + 1 - y) - pos_weight * y) / n)[:, None]
    grads = [None] * len(layers)
    for li in range(len(layers) - 1, -1, -1):
        W, _ = layers[li]
        Ain = A[li]
        grads[li] = (dZ.T @ Ain, dZ.sum(axis=0))
        if li > 0:
            dA = dZ @ W
            dZ = dA * (A[li] > 0)
    flat = np.concatenate([np.concatenate([g[0].ravel(), g[1].ravel()]) for g in grads])
    return loss, flat


def init(seed):
    """He-uniform weights, zero biases (a reference initialisation for tests)."""
    rng = np.random.default_rng(seed)
    parts = []
    for (n_out, n_in) in SIZES:
        lim = np.sqrt(6.0 / n_in)
        parts.append(rng.uniform(-lim, lim, size=n_out * n_in))
        parts.append(np.zeros(n_out))
    return np.concatenate(parts).astype(np.float32)


def adam(theta, m, v, g, t, lr, b1=0.9, b2=0.999, eps=1e-8):
    m = b1 * m + (1 - b1) * g
    v = b2 * v + (1 - b2) * g * g
    mh = m / (1 - b1 ** t)
    vh = v / (1 - b2 ** t)
    return theta - lr * mh / (np.sqrt(vh) + eps), m, v
