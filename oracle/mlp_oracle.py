"""FP64 CPU oracle of the warm-start network (test infrastructure only).

The network: 4 linear layers n_in -> w -> w -> w -> n_out, SiLU after the first three, inputs
standardised (x - in_mean)/in_std, the loss the mean squared error of the standardised outputs
against (y - out_mean)/out_std. Weights enter the products rounded to bf16 (round to nearest
even) when `bf16=True`, and the gradient passes through that rounding unchanged; biases stay
unrounded. Parameters use the flat layout of the library: for each layer W [out][in] then b [out].
"""
import numpy as np


def round_bf16(a):
    """Round float32 values to the nearest bf16 (ties to even), returned as float64."""
    f = np.ascontiguousarray(a, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    r = ((u + 0x7FFF + lsb) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


def unflatten(params, dims):
    out = []
    o = 0
    for l in range(len(dims) - 1):
        w = np.asarray(params[o:o + dims[l + 1] * dims[l]], dtype=np.float64).reshape(dims[l + 1], dims[l])
        o += dims[l + 1] * dims[l]
        b = np.asarray(params[o:o + dims[l + 1]], dtype=np.float64)
        o += dims[l + 1]
        out.append((w, b))
    return out


def _silu(z):
    return z / (1.0 + np.exp(-z))


def _silu_grad(z):
    s = 1.0 / (1.0 + np.exp(-z))
    return s * (1.0 + z * (1.0 - s))


def forward(params, dims, x, norm, bf16=True):
    """Returns the de-standardised outputs and the cache for backward."""
    in_mean, in_std, out_mean, out_std = [np.asarray(v, dtype=np.float64) for v in norm]
    layers = unflatten(params, dims)
    a = (np.asarray(x, dtype=np.float64) - in_mean) / in_std
    cache = []
    for l, (w, b) in enumerate(layers):
        wq = round_bf16(w) if bf16 else w
        z = a @ wq.T + b
        cache.append((a, z, wq))
        a = _silu(z) if l < len(layers) - 1 else z
    return a * out_std + out_mean, cache


def loss_and_grad(params, dims, x, y, norm, bf16=True):
    """Mean squared error of the standardised outputs and its gradient (flat layout)."""
    in_mean, in_std, out_mean, out_std = [np.asarray(v, dtype=np.float64) for v in norm]
    _, cache = forward(params, dims, x, norm, bf16)
    zlast = cache[-1][1]
    t = (np.asarray(y, dtype=np.float64) - out_mean) / out_std
    n = zlast.size
    diff = zlast - t
    loss = float((diff ** 2).sum() / n)
    dz = 2.0 * diff / n
    grads = [None] * len(cache)
    for l in range(len(cache) - 1, -1, -1):
        a, z, wq = cache[l]
        gw = dz.T @ a
        gb = dz.sum(0)
        grads[l] = (gw, gb)
        if l > 0:
            da = dz @ wq
            dz = da * _silu_grad(cache[l - 1][1])
    flat = np.concatenate([np.concatenate([gw.ravel(), gb]) for gw, gb in grads])
    return loss, flat
