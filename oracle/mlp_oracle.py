"""FP64 reference of the chemistry-surrogate MLP -- TEST INFRASTRUCTURE ONLY.

The network maps the chemistry operator's inputs (log10 nH, log10 y, log10 T, log10 N, log10 dt),
normalised, to normalised targets; architecture 5 -> 64 -> 64 -> 3 with SiLU activations:
    z1 = W1 x + b1,  h1 = silu(z1),  z2 = W2 h1 + b2,  h2 = silu(z2),  out = W3 h2 + b3,
silu(z) = z / (1 + exp(-z)). The loss is the mean squared error over the batch and the three
outputs. Gradients are plain backpropagation in FP64; Adam follows Kingma & Ba (2015), with bias
correction. bf16() rounds to bfloat16 (round to nearest even) so that a forward pass can be
evaluated on the same rounded weights and activations as the tensor-core kernels.

Parameters are one flat FP64 vector in the order W1 (64x5, row-major), b1, W2 (64x64), b2,
W3 (3x64), b3 -- the same packing the C ABI uses.
"""
import numpy as np

N_IN, N_H, N_OUT = 5, 64, 3
SIZES = [("W1", (N_H, N_IN)), ("b1", (N_H,)), ("W2", (N_H, N_H)), ("b2", (N_H,)),
         ("W3", (N_OUT, N_H)), ("b3", (N_OUT,))]
N_PARAMS = sum(int(np.prod(s)) for _, s in SIZES)


def unpack(theta):
    out, o = {}, 0
    for name, shape in SIZES:
        n = int(np.prod(shape))
        out[name] = np.asarray(theta[o:o + n], np.float64).reshape(shape)
        o += n
    return out


def pack(p):
    return np.concatenate([np.asarray(p[name], np.float64).ravel() for name, _ in SIZES])


def init(seed=0):
    """He-style uniform initialisation (fan-in scaled), zero biases."""
    rng = np.random.default_rng(seed)
    p = {}
    for name, shape in SIZES:
        if name.startswith("W"):
            lim = np.sqrt(6.0 / shape[1])
            p[name] = rng.uniform(-lim, lim, shape)
        else:
            p[name] = np.zeros(shape)
    return pack(p)


def silu(z):
    return z / (1.0 + np.exp(-z))


def dsilu(z):
    s = 1.0 / (1.0 + np.exp(-z))
    return s * (1.0 + z * (1.0 - s))


def bf16(a):
    """Round to the nearest bfloat16 (ties to even), returned as float64."""
    a32 = np.asarray(a, np.float32)
    u = a32.view(np.uint32).astype(np.uint64)
    r = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


def forward(theta, X, round_bf16=False):
    """Outputs (B, 3). With round_bf16 the inputs, weights and the hidden activations are
    rounded to bfloat16 before each product (the tensor-core kernels' operand precision);
    accumulation and biases stay in high precision."""
    p = unpack(theta)
    r = bf16 if round_bf16 else (lambda a: a)
    X = np.asarray(X, np.float64)
    h1 = silu(r(X) @ r(p["W1"]).T + p["b1"])
    h2 = silu(r(h1) @ r(p["W2"]).T + p["b2"])
    return r(h2) @ r(p["W3"]).T + p["b3"]


def loss_and_grad(theta, X, T):
    """Mean squared error over batch and outputs, and its gradient (flat, FP64)."""
    p = unpack(theta)
    X = np.asarray(X, np.float64)
    T = np.asarray(T, np.float64)
    B = X.shape[0]
    z1 = X @ p["W1"].T + p["b1"]
    h1 = silu(z1)
    z2 = h1 @ p["W2"].T + p["b2"]
    h2 = silu(z2)
    y = h2 @ p["W3"].T + p["b3"]
    d = y - T
    loss = float(np.mean(d * d))
    dy = 2.0 * d / (B * N_OUT)
    g = {}
    g["W3"] = dy.T @ h2
    g["b3"] = dy.sum(0)
    dz2 = (dy @ p["W3"]) * dsilu(z2)
    g["W2"] = dz2.T @ h1
    g["b2"] = dz2.sum(0)
    dz1 = (dz2 @ p["W2"]) * dsilu(z1)
    g["W1"] = dz1.T @ X
    g["b1"] = dz1.sum(0)
    return loss, pack(g)


def adam(theta, grad, m, v, t, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam step (t counts from 1). Returns (theta, m, v)."""
    m = beta1 * m + (1.0 - beta1) * grad
    v = beta2 * v + (1.0 - beta2) * grad * grad
    mh = m / (1.0 - beta1 ** t)
    vh = v / (1.0 - beta2 ** t)
    return theta - lr * mh / (np.sqrt(vh) + eps), m, v
