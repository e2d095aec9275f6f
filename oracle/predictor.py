"""CPU oracle of the hierarchical-grid bin predictor (interpolation and the
int8 network) and of its training step.  TEST INFRASTRUCTURE ONLY.

The paper keeps quantization bins and leaves prediction to LC's later stages;
this predictor is the project's own extension and has no counterpart in the
paper.  Its definition (fixed here, mirrored independently by the CUDA
kernels):

Grid and levels.  Bins are an N x N x N int32 array, index (i*N + j)*N + k.
Anchors are the points whose three coordinates are multiples of 8; they are
kept as they are.  A point of stride s in {4, 2, 1} has coordinates that are
multiples of s but not all multiples of 2s; its odd axes are those whose
coordinate / s is odd, and its class (1..7) is the bit set of its odd axes
(bit 0 = axis i, bit 1 = axis j, bit 2 = axis k).  Level 1, 2, 3 = stride 4,
2, 1.  A point is predicted from bins of coarser levels only.

Coarse positions.  On an axis, the coarse grid of stride s has spacing 2s;
`last(s)` is the largest multiple of 2s not above N-1; positions past it are
clamped to it (and positions below 0 to 0).

Interpolation.  The corners are the 2^c points p + (+/-s) along each odd axis
(c = number of odd axes), clamped; pred = (sum of corner bins + 2^(c-1)) >> c
(arithmetic shift, in 64-bit).

Network.  base = interpolation.  The stencil is the 3x3x3 set of coarse
points f + 2s*(di, dj, dk), d in {-1, 0, 1}, f = the coordinate rounded down
to a multiple of 2s, clamped; input t = (di+1)*9 + (dj+1)*3 + (dk+1).
  x_t = clamp((bin_t - base) >> s_in, -128, 127)
  h_u = clamp((sum_t W1[u,t] x_t + b1[u] + 2^(s1-1)) >> s1, 0, 127), u < 16
  o   = (sum_u W2[u] h_u + b2 + 2^(s2-1)) >> s2
  pred = base + o
with int8 W1, W2 and int32 b1, b2: one weight set per (level, class).
Residual = bin - pred modulo 2^32 (int32 wrap-around), so that
bin = pred + residual modulo 2^32 inverts it exactly.

Training (quantisation-aware, straight-through).  Shadow parameters are real
numbers in integer units; the forward pass uses rint and clamps them to the
int8 / bias ranges and runs the integer network above exactly; the loss is
the mean of squared residuals; gradients pass through every rounding step as
if it were the identity (and through a clamp only inside its range).
"""
import numpy as np

STRIDES = (4, 2, 1)          # levels 1, 2, 3
ANCHOR = 8
NIN, NHID = 27, 16
B1_LIM = 1 << 22             # |bias| limits (keep every sum exact in float32)


def level_stride(level):
    return STRIDES[level - 1]


def last_coarse(N, s):
    return ((N - 1) // (2 * s)) * (2 * s)


def point_sets(N):
    """For each (level, class): index arrays (i, j, k) of its points, in
    C order of their flat index."""
    out = {}
    for level, s in enumerate(STRIDES, start=1):
        c = np.arange(0, N, s)
        for cls in range(1, 8):
            axes = []
            for ax in range(3):
                odd = (cls >> ax) & 1
                sel = c[(c // s) % 2 == 1] if odd else c[(c // s) % 2 == 0]
                axes.append(sel)
            I, J, K = np.meshgrid(*axes, indexing="ij")
            out[(level, cls)] = (I.ravel(), J.ravel(), K.ravel())
    return out


def anchor_points(N):
    c = np.arange(0, N, ANCHOR)
    I, J, K = np.meshgrid(c, c, c, indexing="ij")
    return I.ravel(), J.ravel(), K.ravel()


def _clamp_coord(v, last):
    return np.clip(v, 0, last)


def interp_pred(b3, N, s, cls, I, J, K):
    """Interpolation of the points (I, J, K) of stride s and class cls."""
    last = last_coarse(N, s)
    coords = [I, J, K]
    odd = [ax for ax in range(3) if (cls >> ax) & 1]
    c = len(odd)
    acc = np.zeros(I.shape, dtype=np.int64)
    for corner in range(1 << c):
        pos = [x.copy() for x in coords]
        for bit, ax in enumerate(odd):
            step = s if (corner >> bit) & 1 else -s
            pos[ax] = _clamp_coord(coords[ax] + step, last)
        acc += b3[pos[0], pos[1], pos[2]].astype(np.int64)
    return (acc + (1 << (c - 1))) >> c


def stencil_inputs(b3, N, s, base, I, J, K, s_in):
    """The 27 network inputs of each point, shape (npoints, 27), int64."""
    last = last_coarse(N, s)
    f = [(x // (2 * s)) * (2 * s) for x in (I, J, K)]
    cols = []
    for di in (-1, 0, 1):
        for dj in (-1, 0, 1):
            for dk in (-1, 0, 1):
                pi = _clamp_coord(f[0] + 2 * s * di, last)
                pj = _clamp_coord(f[1] + 2 * s * dj, last)
                pk = _clamp_coord(f[2] + 2 * s * dk, last)
                cols.append(b3[pi, pj, pk].astype(np.int64))
    c = np.stack(cols, axis=1)
    return np.clip((c - base[:, None]) >> s_in, -128, 127)


def mlp_correction(x, W1, b1, W2, b2, s1, s2):
    """Integer network on inputs x (n, 27); returns o (n,) int64."""
    z = x @ W1.astype(np.int64).T + b1.astype(np.int64)[None, :]   # (n, 16)
    h = np.clip((z + (1 << (s1 - 1))) >> s1, 0, 127)
    return (h @ W2.astype(np.int64) + int(b2) + (1 << (s2 - 1))) >> s2


def wrap32(v):
    return ((np.asarray(v, dtype=np.int64) + (1 << 31)) % (1 << 32) - (1 << 31)).astype(np.int32)


class Params:
    """Integer network parameters per (level, class) plus the shifts."""

    def __init__(self, W1, b1, W2, b2, s_in, s1, s2):
        self.W1 = np.asarray(W1, dtype=np.int8).reshape(3, 7, NHID, NIN)
        self.b1 = np.asarray(b1, dtype=np.int32).reshape(3, 7, NHID)
        self.W2 = np.asarray(W2, dtype=np.int8).reshape(3, 7, NHID)
        self.b2 = np.asarray(b2, dtype=np.int32).reshape(3, 7)
        self.s_in = np.asarray(s_in, dtype=np.int32).reshape(3)
        self.s1 = int(s1)
        self.s2 = int(s2)

    @staticmethod
    def zeros(s_in=(0, 0, 0), s1=8, s2=6):
        return Params(np.zeros((3, 7, NHID, NIN)), np.zeros((3, 7, NHID)), np.zeros((3, 7, NHID)),
                      np.zeros((3, 7)), s_in, s1, s2)


def predict(bins, N, params=None):
    """Predictions of every point (anchors: 0) and the level of each point
    (0 = anchor).  params None: interpolation only."""
    b3 = np.asarray(bins, dtype=np.int32).reshape(N, N, N)
    pred = np.zeros((N, N, N), dtype=np.int64)
    level = np.zeros((N, N, N), dtype=np.int8)
    for (lv, cls), (I, J, K) in point_sets(N).items():
        s = level_stride(lv)
        base = interp_pred(b3, N, s, cls, I, J, K)
        if params is not None:
            x = stencil_inputs(b3, N, s, base, I, J, K, int(params.s_in[lv - 1]))
            o = mlp_correction(x, params.W1[lv - 1, cls - 1], params.b1[lv - 1, cls - 1],
                               params.W2[lv - 1, cls - 1], params.b2[lv - 1, cls - 1], params.s1, params.s2)
            base = base + o
        pred[I, J, K] = base
        level[I, J, K] = lv
    return pred.reshape(-1), level.reshape(-1)


def residuals(bins, N, params=None):
    """int32 residuals: bin - pred (mod 2^32) at predicted points, the bin
    itself at anchors."""
    pred, _ = predict(bins, N, params)
    b = np.asarray(bins, dtype=np.int64).reshape(-1)
    return wrap32(b - pred)


def reconstruct(res, N, params=None):
    """Inverse of residuals(): anchors first, then levels 1..3, each level
    predicted from the bins already reconstructed."""
    r = np.asarray(res, dtype=np.int64).reshape(N, N, N)
    b3 = np.zeros((N, N, N), dtype=np.int32)
    I, J, K = anchor_points(N)
    b3[I, J, K] = r[I, J, K].astype(np.int32)
    sets = point_sets(N)
    for lv in (1, 2, 3):
        s = level_stride(lv)
        for cls in range(1, 8):
            I, J, K = sets[(lv, cls)]
            base = interp_pred(b3, N, s, cls, I, J, K)
            if params is not None:
                x = stencil_inputs(b3, N, s, base, I, J, K, int(params.s_in[lv - 1]))
                base = base + mlp_correction(x, params.W1[lv - 1, cls - 1], params.b1[lv - 1, cls - 1],
                                             params.W2[lv - 1, cls - 1], params.b2[lv - 1, cls - 1],
                                             params.s1, params.s2)
            b3[I, J, K] = wrap32(base + r[I, J, K])
    return b3.reshape(-1)


def entropy_bits(values):
    """Shannon entropy (bits per value) of the empirical distribution."""
    v = np.asarray(values).reshape(-1)
    if v.size == 0:
        return 0.0
    _, counts = np.unique(v, return_counts=True)
    p = counts / v.size
    return float(-(p * np.log2(p)).sum())


def bits_per_value(res, N, outlier_flags=None):
    """Residual entropy of the predicted non-outlier points plus the entropy
    of the anchors' bins, weighted by their counts, over all N^3 values
    (outliers are stored losslessly elsewhere and are not counted here)."""
    _, level = predict(np.zeros(N ** 3, dtype=np.int32), N)
    r = np.asarray(res).reshape(-1)
    keep = np.ones(r.size, dtype=bool) if outlier_flags is None else ~np.asarray(outlier_flags, bool)
    a = (level == 0) & keep
    p = (level > 0) & keep
    return (entropy_bits(r[a]) * a.sum() + entropy_bits(r[p]) * p.sum()) / r.size


# ---------------------------------------------------------------- training --

def fake_quant(w1, b1, w2, b2):
    """Shadow (real, integer units) -> integer parameters used by the forward
    pass, and the straight-through masks (1 where the clamp is inactive)."""
    W1 = np.rint(w1)
    m1 = (W1 >= -128) & (W1 <= 127)
    B1 = np.rint(b1)
    mb1 = np.abs(B1) <= B1_LIM
    W2 = np.rint(w2)
    m2 = (W2 >= -128) & (W2 <= 127)
    B2 = np.rint(b2)
    mb2 = np.abs(B2) <= B1_LIM
    return (np.clip(W1, -128, 127), np.clip(B1, -B1_LIM, B1_LIM), np.clip(W2, -128, 127),
            np.clip(B2, -B1_LIM, B1_LIM), (m1, mb1, m2, mb2))


def train_forward_backward(x, base, target, w1, b1, w2, b2, s1, s2):
    """One network, samples x (n, 27) int, base and target (n,) int.
    Returns (loss_sum, grads dict, abs-term sums dict) in float64: loss_sum is
    the sum of squared residuals; gradients are of loss_sum / n.  The forward
    pass is the exact integer network on the fake-quantised parameters."""
    x = np.asarray(x, dtype=np.float64)
    n = x.shape[0]
    W1, B1, W2, B2, (m1, mb1, m2, mb2) = fake_quant(w1, b1, w2, b2)
    z = x @ W1.T + B1[None, :]                                  # exact integers
    hu = np.floor((z + 2.0 ** (s1 - 1)) / 2.0 ** s1)            # before the clamp
    h = np.clip(hu, 0, 127)
    on = (hu > 0) & (hu < 127)
    o = np.floor((h @ W2 + B2 + 2.0 ** (s2 - 1)) / 2.0 ** s2)
    r = np.asarray(target, np.float64) - (np.asarray(base, np.float64) + o)
    loss = float((r * r).sum())
    go = -2.0 * r / n                                           # d(loss/n)/do
    gz = (go[:, None] * (W2[None, :] / 2.0 ** s2)) * on / 2.0 ** s1
    gW2 = (go[:, None] * h).sum(0) / 2.0 ** s2 * m2
    gB2 = go.sum() / 2.0 ** s2 * mb2
    gW1 = (gz.T @ x) * m1
    gB1 = gz.sum(0) * mb1
    absterms = {
        "w2": (np.abs(go)[:, None] * h).sum(0) / 2.0 ** s2,
        "b2": np.abs(go).sum() / 2.0 ** s2,
        "w1": np.abs(gz).T @ np.abs(x),
        "b1": np.abs(gz).sum(0),
    }
    return loss, {"w1": gW1, "b1": gB1, "w2": gW2, "b2": gB2}, absterms
