"""Seeded initial weights of the per-cell MLP (24 -> 64 -> 64 -> 8).

Flat float64 vector in the order W1 [64, 24], b1 [64], W2 [64, 64], b2 [64],
W3 [8, 64], b3 [8] (row-major). W1, W2 uniform(-1, 1) / sqrt(fan_in) from
PCG64(seed); W3 and the biases zero, so the initial correction is the
identity.
"""
import numpy as np

NF, NH, NO = 24, 64, 8
SIZES = (("W1", (NH, NF)), ("b1", (NH,)), ("W2", (NH, NH)), ("b2", (NH,)),
         ("W3", (NO, NH)), ("b3", (NO,)))
NPARAM = sum(int(np.prod(s)) for _, s in SIZES)


def initial_params(seed):
    rng = np.random.Generator(np.random.PCG64(seed))
    W1 = rng.uniform(-1, 1, (NH, NF)) / np.sqrt(NF)
    W2 = rng.uniform(-1, 1, (NH, NH)) / np.sqrt(NH)
    return dict(W1=W1, b1=np.zeros(NH), W2=W2, b2=np.zeros(NH),
                W3=np.zeros((NO, NH)), b3=np.zeros(NO))


def flatten(params):
    return np.concatenate([np.asarray(params[k], np.float64).reshape(-1) for k, _ in SIZES])


def unflatten(vec):
    out, o = {}, 0
    for k, s in SIZES:
        n = int(np.prod(s))
        out[k] = np.asarray(vec[o:o + n], np.float64).reshape(s)
        o += n
    return out
