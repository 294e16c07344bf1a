"""A network whose ReLU decisions all have a margin, for well-conditioned gradient checks.

Test infrastructure (used by the register-path parity tests and by the smoke
check). The network of Sec. 2.1 has ReLU units (Eq. relu), so the loss
gradient jumps wherever a unit's pre-activation crosses zero; with Xavier
weights and zero biases some units of a large mesh sit within rounding of zero,
and a float32 and a float64 evaluation then take different sides. The network
built here keeps the Xavier weights and sets the biases from the FP64 oracle's
own pre-activation ranges over every voxel of the given feature fields, so
that no decision is near zero and the float32 path can be held to the
gradient tolerance without the comparison depending on those flips.
"""
import numpy as np

from oracle import nn as onn


def _ranges(u):
    return u.min(axis=1), u.max(axis=1)


def margin_network(w, field_sets, gap=0.5, y_span=8.0):
    """Xavier weights w with biases that keep every ReLU decision away from zero.

    Layer by layer, over every voxel of the given feature fields: the
    pre-activation range [lo, hi] of each unit without bias; even units get a
    bias that puts the range at [gap, 1 + gap] x (hi - lo) (always on), odd
    units at -[1 + gap, gap] x (hi - lo) (always off); the output weights are
    scaled and offset so that y spans [-y_span/2, y_span/2] (a mass range of
    about 300 for the default 8; the unscaled output would span some 10^9 in
    mass, and float32 smoothing errors of the largest masses would then land
    on M0-sized values inside the log). Returns the weight vector and the smallest |pre-activation| /
    range width over all units and voxels (>= gap by construction)."""
    W1, _, W2, _, w3, _ = onn.unpack(w)
    on1 = np.arange(W1.shape[0]) % 2 == 0
    on2 = np.arange(W2.shape[0]) % 2 == 0

    def chunks():
        for f in field_sets:
            n = f.shape[1]
            for idx in np.array_split(np.arange(n ** 3), max(1, n ** 3 // (1 << 17))):
                yield onn.stencil_at(f, np.stack(np.unravel_index(idx, (n, n, n)), axis=1))

    def bias_for(lo, hi, on):
        width = hi - lo
        return np.where(on, -lo + gap * width, -hi - gap * width), width

    lo = np.full(W1.shape[0], np.inf); hi = -lo
    for v in chunks():
        a, b = _ranges(W1 @ v)
        lo, hi = np.minimum(lo, a), np.maximum(hi, b)
    b1, width1 = bias_for(lo, hi, on1)
    lo = np.full(W2.shape[0], np.inf); hi = -lo
    for v in chunks():
        a, b = _ranges(W2 @ onn.relu(W1 @ v + b1[:, None]))
        lo, hi = np.minimum(lo, a), np.maximum(hi, b)
    b2, width2 = bias_for(lo, hi, on2)
    ylo, yhi, margin = np.inf, -np.inf, np.inf
    for v in chunks():
        a1 = W1 @ v + b1[:, None]
        a2 = W2 @ onn.relu(a1) + b2[:, None]
        y = w3 @ onn.relu(a2)
        ylo, yhi = min(ylo, y.min()), max(yhi, y.max())
        margin = min(margin, (np.abs(a1) / width1[:, None]).min(), (np.abs(a2) / width2[:, None]).min())
    scale = y_span / (yhi - ylo)
    b3 = -0.5 * (ylo + yhi) * scale
    out = np.concatenate([W1.ravel(), b1, W2.ravel(), b2, scale * w3, [b3]]).astype(np.float32)
    return out, margin
