"""Seeded inputs shared by the oracle and the GPU tests of the learned slice
move: network parameters and batches.  No arithmetic of the method lives
here.  Parameters are rounded to bfloat16-representable values (round to
nearest even on the float32 bit pattern), so that a path storing its
weights in bfloat16 and the FP64 oracle hold identical numbers."""
import numpy as np


def bf16_exact(x):
    f = np.ascontiguousarray(x, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def random_params(nf, H, seed, out_scale=0.05, mu_bias=0.0, logsig_bias=0.0):
    """Layers W1 (H x 2nf), b1, W2 (H x H), b2, W3 (2nf x H), b3, packed in
    that order; hidden weights ~ N(0, 1/fan_in), output layer scaled by
    out_scale, b3 = [mu_bias] * nf + [logsig_bias] * nf."""
    r = np.random.default_rng(seed)
    parts = [r.standard_normal((H, 2 * nf)) / np.sqrt(2 * nf), 0.1 * r.standard_normal(H),
             r.standard_normal((H, H)) / np.sqrt(H), 0.1 * r.standard_normal(H),
             out_scale * r.standard_normal((2 * nf, H)) / np.sqrt(H),
             np.concatenate([np.full(nf, mu_bias), np.full(nf, logsig_bias)])]
    return bf16_exact(np.concatenate([p.ravel() for p in parts]))


def random_batch(nf, B, seed):
    r = np.random.default_rng(seed)
    return r.standard_normal((B, 2 * nf)), r.standard_normal((B, nf))
