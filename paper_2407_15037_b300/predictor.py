"""Binding of the hierarchical-grid bin predictor (include/lcq.h, the
lcq_pred_* and lcq_train_* entry points) and the host side of training.

Every step that touches bins or parameters runs in liblcq.so's kernels:
residuals, reconstruction, histograms, the training forward/backward pass,
the deterministic gradient reduction, Adam and the int8 freeze.  Python only
picks the training samples (seeded), lays them out per network, and turns the
device histograms into entropies.
"""
import ctypes
import math

import numpy as np
import torch

from . import lcq as _L

NETS = 21
NPARAM = 16 * 27 + 16 + 16 + 1
STRIDES = (4, 2, 1)
HIST_HALF = 1 << 20


class PredParams(ctypes.Structure):
    """Mirror of struct lcq_pred_params."""
    _fields_ = [("w1", ctypes.c_int8 * (3 * 7 * 16 * 28)), ("b1", ctypes.c_int32 * (3 * 7 * 16)),
                ("w2", ctypes.c_int8 * (3 * 7 * 16)), ("b2", ctypes.c_int32 * (3 * 7)),
                ("s_in", ctypes.c_int32 * 3), ("s1", ctypes.c_int32), ("s2", ctypes.c_int32),
                ("reserved", ctypes.c_int32)]


PARAMS_BYTES = ctypes.sizeof(PredParams)

_vp, _u32, _i32, _f32 = ctypes.c_void_p, ctypes.c_uint32, ctypes.c_int32, ctypes.c_float
SIGNATURES = {
    "lcq_pred_residuals": ([_vp, _u32, _vp, _vp, _vp], ctypes.c_int),
    "lcq_pred_reconstruct": ([_vp, _u32, _vp, _vp, _vp], ctypes.c_int),
    "lcq_pred_histogram_words": ([], ctypes.c_size_t),
    "lcq_pred_histogram": ([_vp, _u32, _vp, _vp, _vp, _vp], ctypes.c_int),
    "lcq_train_param_count": ([], _u32),
    "lcq_train_gradients": ([_vp, _u32, _vp, _vp, _u32, _vp, _vp, _vp, _vp, _i32, _i32, _vp, _vp, _vp, _vp],
                            ctypes.c_int),
    "lcq_train_adam": ([_vp, _vp, _vp, _vp, _f32, _f32, _f32, _f32, _u32, _vp], ctypes.c_int),
    "lcq_pred_freeze": ([_vp, _vp, _i32, _i32, _vp, _vp], ctypes.c_int),
}
_bound = False


def lib():
    global _bound
    L = _L.lib()
    if not _bound:
        for name, (args, res) in SIGNATURES.items():
            fn = getattr(L, name)
            fn.argtypes = args
            fn.restype = res
        _bound = True
    return L


def _p(t):
    return _L._ptr(t)


def _s(dev):
    return _L._stream_ptr(None, dev)


def params_to_device(params, device):
    """PredParams (host struct) -> uint8 device tensor."""
    raw = bytes(params)
    return torch.frombuffer(bytearray(raw), dtype=torch.uint8).to(device)


def save_params(params, path):
    """Write frozen parameters (a uint8 device tensor from Trainer.freeze or
    params_to_device, or a PredParams) as the raw little-endian bytes of
    struct lcq_pred_params."""
    raw = bytes(params) if isinstance(params, PredParams) else bytes(params.cpu().numpy())
    if len(raw) != PARAMS_BYTES:
        raise ValueError("predictor parameters must be %d bytes" % PARAMS_BYTES)
    with open(path, "wb") as f:
        f.write(raw)


def load_params(path, device):
    """Frozen parameters written by save_params, as a uint8 device tensor."""
    with open(path, "rb") as f:
        raw = f.read()
    if len(raw) != PARAMS_BYTES:
        raise ValueError("%s: %d bytes, expected %d" % (path, len(raw), PARAMS_BYTES))
    return torch.frombuffer(bytearray(raw), dtype=torch.uint8).to(device)


def params_from_device(t):
    p = PredParams()
    ctypes.memmove(ctypes.addressof(p), bytes(t.cpu().numpy()), PARAMS_BYTES)
    return p


def residuals(bins, N, params=None):
    """bins: int32 CUDA tensor of N^3; params: uint8 device tensor or None."""
    res = torch.empty_like(bins)
    code = lib().lcq_pred_residuals(_p(bins), int(N), _p(params) if params is not None else None, _p(res),
                                    _s(bins.device))
    _L._check(code, "lcq_pred_residuals")
    return res


def reconstruct(res, N, params=None):
    bins = torch.empty_like(res)
    code = lib().lcq_pred_reconstruct(_p(res), int(N), _p(params) if params is not None else None, _p(bins),
                                      _s(res.device))
    _L._check(code, "lcq_pred_reconstruct")
    return bins


def histogram(res, N, mask=None):
    """(anchor counts, predicted-point counts, overflow counts) as numpy."""
    words = int(lib().lcq_pred_histogram_words())
    hist = torch.empty(words, dtype=torch.int32, device=res.device)
    over = torch.empty(2, dtype=torch.int64, device=res.device)
    code = lib().lcq_pred_histogram(_p(res), int(N), _p(mask) if mask is not None else None, _p(hist),
                                    _p(over), _s(res.device))
    _L._check(code, "lcq_pred_histogram")
    h = hist.cpu().numpy().view(np.uint32).astype(np.int64)
    return h[:2 * HIST_HALF], h[2 * HIST_HALF:], over.cpu().numpy()


def entropy_from_counts(c):
    c = c[c > 0].astype(np.float64)
    if c.size == 0:
        return 0.0, 0
    n = c.sum()
    p = c / n
    return float(-(p * np.log2(p)).sum()), int(n)


def bits_per_value(res, N, mask=None):
    """Residual entropy of predicted points plus anchor-bin entropy, weighted
    by their counts, per value of the grid (outliers excluded)."""
    ha, hp, over = histogram(res, N, mask)
    if over.any():
        raise ValueError("residuals outside [-2^20, 2^20): entropy needs the exact values")
    ea, na = entropy_from_counts(ha)
    ep, npred = entropy_from_counts(hp)
    return (ea * na + ep * npred) / float(N ** 3), {"anchor_bits": ea, "pred_bits": ep, "anchors": na,
                                                     "predicted": npred}


# ---------------------------------------------------------------- training --

def _class_coords(N, s, cls, rng, m):
    out = []
    for ax in range(3):
        odd = (cls >> ax) & 1
        c = np.arange(0, N, s)
        c = c[(c // s) % 2 == 1] if odd else c[(c // s) % 2 == 0]
        out.append(rng.choice(c, m))
    return out


def choose_s_in(bins_host, N, rng, q=0.99, m=20000):
    """Per level, the smallest right shift that brings the q-quantile of
    |coarse neighbour - interpolation| within 127 (an int8 input)."""
    b3 = bins_host.reshape(N, N, N).astype(np.int64)
    s_in = []
    for s in STRIDES:
        last = ((N - 1) // (2 * s)) * (2 * s)
        i, j, k = _class_coords(N, s, 1, rng, m)
        lo, hi = b3[i - s, j, k], b3[np.minimum(i + s, last), j, k]
        base = (lo + hi + 1) >> 1
        d = np.abs(np.concatenate([lo - base, hi - base]))
        v = float(np.quantile(d, q))
        s_in.append(max(0, int(math.ceil(math.log2(max(v, 1.0) / 127.0)))))
    return s_in


class Trainer:
    """Quantisation-aware training of the 21 int8 networks on bins that the
    quantizer produced.  `fields`: one int32 CUDA tensor with F fields of N^3
    bins back to back.  A fixed, seeded sample set (samples_per_net points of
    every (level, class), drawn uniformly over fields and positions) is used
    for full-batch Adam steps."""

    def __init__(self, fields, N, samples_per_net=65536, seed=0, s_in=(3, 3, 2), s1=8, s2=6,
                 lr=0.5, init_scale=30.0):
        self.dev = fields.device
        self.fields, self.N = fields, int(N)
        F = fields.numel() // self.N ** 3
        rng = np.random.default_rng(seed)
        self.s_in = np.asarray(s_in, dtype=np.int32)
        self.s1, self.s2, self.lr = int(s1), int(s2), float(lr)
        samples, items, item_begin, inv = [], [], [0], []
        for lv, s in enumerate(STRIDES, start=1):
            for cls in range(1, 8):
                net = (lv - 1) * 7 + (cls - 1)
                m = samples_per_net
                i, j, k = _class_coords(self.N, s, cls, rng, m)
                f = rng.integers(0, F, m)
                e = (i.astype(np.int64) * self.N + j) * self.N + k
                start = len(samples) and sum(len(x) for x in samples)
                samples.append((f.astype(np.uint64) << np.uint64(32)) | e.astype(np.uint64))
                for a in range(0, m, 256):
                    items.append((net, start + a, min(256, m - a), 0))
                item_begin.append(len(items))
                inv.append(1.0 / m)
        self.samples = torch.from_numpy(np.concatenate(samples).view(np.int64)).to(self.dev)
        self.items = torch.from_numpy(np.asarray(items, dtype=np.uint32).view(np.int32)).to(self.dev)
        self.num_items = len(items)
        self.item_begin = torch.from_numpy(np.asarray(item_begin, dtype=np.uint32).view(np.int32)).to(self.dev)
        self.inv_count = torch.tensor(inv, dtype=torch.float32, device=self.dev)
        # init: near-linear units (bias puts pre-activations mid-range), output
        # bias cancelling the mid-range offset, small random weights
        w = np.zeros((NETS, NPARAM), dtype=np.float32)
        w[:, :16 * 27] = rng.normal(0.0, init_scale, (NETS, 16 * 27))
        w[:, 16 * 27:16 * 27 + 16] = 64.0 * 2 ** self.s1
        w2 = rng.normal(0.0, 2.0, (NETS, 16))
        w[:, 16 * 27 + 16:16 * 27 + 32] = w2
        w[:, -1] = -64.0 * np.rint(w2).sum(1)
        self.shadow = torch.from_numpy(w.reshape(-1)).to(self.dev)
        self.m = torch.zeros_like(self.shadow)
        self.v = torch.zeros_like(self.shadow)
        self.partial = torch.empty(self.num_items * (NPARAM + 1), dtype=torch.float32, device=self.dev)
        self.grad = torch.empty(NETS * NPARAM, dtype=torch.float32, device=self.dev)
        self.loss = torch.empty(NETS, dtype=torch.float32, device=self.dev)
        self.t = 0

    def gradients(self):
        s_in = (ctypes.c_int32 * 3)(*[int(v) for v in self.s_in])
        code = lib().lcq_train_gradients(
            _p(self.fields), self.N, _p(self.samples), _p(self.items), self.num_items, _p(self.item_begin),
            _p(self.shadow), _p(self.inv_count), s_in, self.s1, self.s2, _p(self.partial), _p(self.grad),
            _p(self.loss), _s(self.dev))
        _L._check(code, "lcq_train_gradients")

    def step(self):
        self.gradients()
        self.t += 1
        code = lib().lcq_train_adam(_p(self.shadow), _p(self.m), _p(self.v), _p(self.grad), self.lr, 0.9, 0.999,
                                    1e-8, self.t, _s(self.dev))
        _L._check(code, "lcq_train_adam")

    def mean_squared_residual(self):
        torch.cuda.synchronize(self.dev)
        return float(self.loss.double().sum().item() / (self.samples.numel()))

    def state_dict(self):
        """Training state for checkpoints: float32 shadow parameters, Adam
        moments, step count and the fixed shifts (host tensors)."""
        return {"shadow": self.shadow.cpu(), "m": self.m.cpu(), "v": self.v.cpu(), "t": self.t,
                "s_in": self.s_in.copy(), "s1": self.s1, "s2": self.s2, "lr": self.lr}

    def load_state_dict(self, st):
        """Resume from state_dict(); the sample set is the constructor's
        (same fields and seed give the same samples)."""
        if st["shadow"].numel() != self.shadow.numel():
            raise ValueError("checkpoint for a different network shape")
        self.shadow.copy_(st["shadow"].to(self.dev))
        self.m.copy_(st["m"].to(self.dev))
        self.v.copy_(st["v"].to(self.dev))
        self.t = int(st["t"])
        self.s_in = np.asarray(st["s_in"], dtype=np.int32)
        self.s1, self.s2, self.lr = int(st["s1"]), int(st["s2"]), float(st["lr"])

    def freeze(self):
        out = torch.zeros(PARAMS_BYTES, dtype=torch.uint8, device=self.dev)
        s_in = (ctypes.c_int32 * 3)(*[int(v) for v in self.s_in])
        code = lib().lcq_pred_freeze(_p(self.shadow), s_in, self.s1, self.s2, _p(out), _s(self.dev))
        _L._check(code, "lcq_pred_freeze")
        return out
