"""FP64 reference of the learned proposal network (test infrastructure only).

Mirrors the network of the library: features x (64, bf16) -> 256 -> 256 -> 3, GELU (erf form), BF16
operands with products accumulated exactly (here in FP64), sign-invariant loss 1 - (y_hat . t)^2,
Adam.  The rounding to bf16 happens where the GPU rounds (weights, hidden activations, the output
gradient and the hidden-layer gradients that feed the GEMMs); round=False drops every rounding so
that the gradient can be checked against finite differences.  Random numbers (initialisation,
batch sampling) come from this module's own SplitMix64 (Steele, Lea, Flood 2014).
"""
import numpy as np
from scipy.special import erf

IN, HID = 64, 256
SIZES = [("W1", (HID, IN)), ("b1", (HID,)), ("W2", (HID, HID)), ("b2", (HID,)), ("W3", (3, HID)), ("b3", (3,))]
COUNT = sum(int(np.prod(s)) for _, s in SIZES)
M64 = (1 << 64) - 1


def splitmix64(x):
    x = (x + 0x9E3779B97F4A7C15) & M64
    x = ((x ^ (x >> 30)) * 0xBF58476D1CE4E5B9) & M64
    x = ((x ^ (x >> 27)) * 0x94D049BB133111EB) & M64
    return x ^ (x >> 31)


def unpack(P):
    out, o = {}, 0
    for name, shape in SIZES:
        n = int(np.prod(shape))
        out[name] = np.asarray(P[o:o + n], np.float64).reshape(shape)
        o += n
    return out


def pack(d):
    return np.concatenate([np.asarray(d[name], np.float64).ravel() for name, _ in SIZES])


def bf16(x):
    """Round to bfloat16 (round to nearest, ties to even) via the float32 bit pattern."""
    x32 = np.asarray(x, np.float32)
    b = x32.view(np.uint32).astype(np.uint64)
    r = ((b + 0x7FFF + ((b >> 16) & 1)) & 0xFFFF0000).astype(np.uint32)
    out = r.view(np.float32).astype(np.float64)
    return np.where(np.isfinite(x32), out, x32.astype(np.float64))


def bf16_bits(x):
    return (np.asarray(bf16(x), np.float32).view(np.uint32) >> 16).astype(np.uint16)


def from_bits(u16):
    return (np.asarray(u16, np.uint32) << 16).view(np.float32).astype(np.float64)


def init(seed):
    """Uniform(-1/sqrt(fan_in), 1/sqrt(fan_in)), fan_in 51 for layer 1 (input columns 51..63 zero)."""
    P = np.empty(COUNT)
    o = 0
    for name, shape in SIZES:
        n = int(np.prod(shape))
        fan = 51.0 if name in ("W1", "b1") else 256.0
        for q in range(n):
            e = o + q
            u = (splitmix64(seed ^ splitmix64(e)) >> 11) * (1.0 / 9007199254740992.0)
            P[e] = (2.0 * u - 1.0) / np.sqrt(fan)
        if name == "W1":
            P[o:o + n].reshape(shape)[:, 51:] = 0.0
        o += n
    return np.asarray(np.float32(P), np.float64)


def batch_indices(seed, step, B, n):
    """Sample b of training step `step`: hash(seed, step, b) mod n."""
    return np.array([splitmix64(seed ^ splitmix64(((step << 20) ^ b) & M64)) % n for b in range(B)], np.int64)


def gelu(z):
    return 0.5 * z * (1.0 + erf(z / np.sqrt(2.0)))


def gelu_grad(z):
    return 0.5 * (1.0 + erf(z / np.sqrt(2.0))) + z * np.exp(-0.5 * z * z) / np.sqrt(2.0 * np.pi)


def forward(P, X, round=True):
    """Proposals (n, 3) and the intermediate values for features X (n, 64)."""
    r = bf16 if round else (lambda v: np.asarray(v, np.float64))
    p = unpack(P)
    W1, W2, W3 = r(p["W1"]), r(p["W2"]), r(p["W3"])
    Z1 = X @ W1.T + p["b1"]
    H1 = r(gelu(Z1))
    Z2 = H1 @ W2.T + p["b2"]
    H2 = r(gelu(Z2))
    Y = H2 @ W3.T + p["b3"]
    n = np.linalg.norm(Y, axis=1, keepdims=True)
    D = np.where(n > 0, Y / np.where(n > 0, n, 1.0), np.array([0.0, 0.0, 1.0]))
    return D, dict(W1=W1, W2=W2, W3=W3, Z1=Z1, H1=H1, Z2=Z2, H2=H2, Y=Y)


def loss_and_grads(P, X, T, round=True):
    """Mean loss 1 - (y_hat . t)^2 and its gradient in the parameter-vector layout."""
    r = bf16 if round else (lambda v: np.asarray(v, np.float64))
    B = X.shape[0]
    _, c = forward(P, X, round)
    Y = c["Y"]
    ny = np.linalg.norm(Y, axis=1, keepdims=True)
    yh = Y / ny
    s = np.sum(yh * T, axis=1, keepdims=True)
    loss = float(np.mean(1.0 - s[:, 0] ** 2))
    gY = (-2.0 * s / ny) * (T - s * yh) / B
    dZ3 = r(gY)
    g = {"b3": gY.sum(axis=0), "W3": dZ3.T @ c["H2"]}
    dZ2 = (dZ3 @ c["W3"]) * gelu_grad(c["Z2"])
    g["b2"] = dZ2.sum(axis=0)
    dZ2r = r(dZ2)
    g["W2"] = dZ2r.T @ c["H1"]
    dZ1 = (dZ2r @ c["W2"]) * gelu_grad(c["Z1"])
    g["b1"] = dZ1.sum(axis=0)
    g["W1"] = r(dZ1).T @ X
    return loss, pack(g)


def adam(P, G, M, V, t, lr, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam step at step number t (1-based); returns the new (P, M, V)."""
    M = b1 * M + (1 - b1) * G
    V = b2 * V + (1 - b2) * G * G
    P = P - lr * (M / (1 - b1 ** t)) / (np.sqrt(V / (1 - b2 ** t)) + eps)
    return P, M, V
