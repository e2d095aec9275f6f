"""Predictor kernels vs the predictor oracle: residuals (interpolation and
int8 network) and reconstruction bit for bit, histogram counts exactly,
training gradients within a bound derived from float32 summation, the int8
freeze exactly; and a small end-to-end run showing the trained network
lowering the residual entropy below interpolation."""
import ctypes

import numpy as np
import pytest
import torch

import oracle.predictor as PR
import paper_2407_15037_b300 as P
from paper_2407_15037_b300 import predictor as PD
import synth

pytestmark = pytest.mark.gpu

DEV = "cuda"


def _params_struct(p):
    """oracle Params -> lcq_pred_params."""
    s = PD.PredParams()
    w1 = np.zeros((3, 7, 16, 28), dtype=np.int8)
    w1[..., :27] = p.W1
    ctypes.memmove(s.w1, w1.tobytes(), w1.nbytes)
    ctypes.memmove(s.b1, p.b1.astype(np.int32).tobytes(), p.b1.nbytes)
    ctypes.memmove(s.w2, p.W2.astype(np.int8).tobytes(), p.W2.nbytes)
    ctypes.memmove(s.b2, p.b2.astype(np.int32).tobytes(), p.b2.nbytes)
    for l in range(3):
        s.s_in[l] = int(p.s_in[l])
    s.s1, s.s2 = p.s1, p.s2
    return s


def _random_params(rng, s_in=(2, 1, 0)):
    return PR.Params(rng.integers(-128, 128, (3, 7, 16, 27)), rng.integers(-5000, 5000, (3, 7, 16)),
                     rng.integers(-128, 128, (3, 7, 16)), rng.integers(-5000, 5000, (3, 7)), s_in, 8, 6)


@pytest.mark.parametrize("N", [9, 16, 33, 64, 100, 130])
def test_residuals_and_reconstruct_match_oracle(N):
    """Grids of one to several boxes of coarse cells per axis (32 cells
    along k, 4 along j, 2 along i), ragged ones included."""
    rng = np.random.default_rng(N)
    bins = rng.integers(-(1 << 30) + 1, 1 << 30, N ** 3).astype(np.int32)
    bins[: N ** 3 // 2] = rng.integers(-3000, 3000, N ** 3 // 2)  # a smooth-ish part and an extreme part
    db = torch.from_numpy(bins).to(DEV)
    for params in (None, _random_params(rng)):
        dp = PD.params_to_device(_params_struct(params), DEV) if params is not None else None
        res = PD.residuals(db, N, dp)
        want = PR.residuals(bins, N, params)
        assert np.array_equal(res.cpu().numpy(), want)
        back = PD.reconstruct(res, N, dp)
        assert np.array_equal(back.cpu().numpy(), bins)


@pytest.mark.parametrize("s1,s2,s_in", [(1, 1, (0, 0, 0)), (24, 24, (30, 30, 30)), (8, 24, (0, 13, 30)),
                                         (24, 1, (30, 1, 0))])
def test_network_extreme_parameters_match_oracle(s1, s2, s_in):
    """Weights at -128 / 127, biases at +-2^22 and the shifts at the ends of
    their supported ranges: the sums of both layers stay exact (binary16
    operands, float32 accumulators) and the clamps (before the shifts) agree
    with the oracle's int64 arithmetic."""
    N = 33
    rng = np.random.default_rng(s1 * 100 + s2)
    bins = rng.integers(-(1 << 30) + 1, 1 << 30, N ** 3).astype(np.int32)
    bins[: N ** 3 // 2] = rng.integers(-600, 600, N ** 3 // 2)
    ext = np.array([-128, 127])
    W1 = ext[rng.integers(0, 2, (3, 7, 16, 27))]
    W1[0, 0] = 127                     # one network with every product at its largest
    W1[0, 1] = -128
    b1 = np.where(rng.integers(0, 2, (3, 7, 16)) == 1, 1 << 22, -(1 << 22))
    b1[1] = rng.integers(-(1 << 22), (1 << 22) + 1, (7, 16))
    W2 = ext[rng.integers(0, 2, (3, 7, 16))]
    b2 = np.where(rng.integers(0, 2, (3, 7)) == 1, 1 << 22, -(1 << 22))
    params = PR.Params(W1, b1, W2, b2, s_in, s1, s2)
    dp = PD.params_to_device(_params_struct(params), DEV)
    db = torch.from_numpy(bins).to(DEV)
    res = PD.residuals(db, N, dp)
    assert np.array_equal(res.cpu().numpy(), PR.residuals(bins, N, params))
    back = PD.reconstruct(res, N, dp)
    assert np.array_equal(back.cpu().numpy(), bins)


def test_histogram_counts_match():
    N = 40
    rng = np.random.default_rng(7)
    res = rng.integers(-5000, 5000, N ** 3).astype(np.int32)
    res[::97] = rng.integers(-(1 << 20), 1 << 20, res[::97].size)
    mask = rng.integers(0, 1 << 32, (N ** 3 + 31) // 32, dtype=np.uint64).astype(np.uint32) & 0x01010101
    ha, hp, over = PD.histogram(torch.from_numpy(res).to(DEV), N,
                                torch.from_numpy(mask.view(np.int32)).to(DEV))
    idx = np.arange(N ** 3)
    keep = ((mask[idx >> 5] >> (idx & 31)) & 1) == 0
    _, level = PR.predict(np.zeros(N ** 3, np.int32), N)
    for h, sel in ((ha, keep & (level == 0)), (hp, keep & (level > 0))):
        want = np.bincount(res[sel].astype(np.int64) + (1 << 20), minlength=1 << 21)
        assert np.array_equal(h, want)
    assert over.sum() == 0


def test_training_gradients_match_oracle():
    N = 32
    F = 3
    fields = torch.cat([torch.from_numpy(
        np.rint(synth.grf(N, seed=s).numpy() / 2e-3).astype(np.int32)) for s in range(F)]).to(DEV)
    tr = PD.Trainer(fields, N, samples_per_net=700, seed=3, s_in=(3, 3, 2), s1=8, s2=6)
    tr.shadow += torch.randn(tr.shadow.shape, generator=torch.Generator(DEV).manual_seed(1), device=DEV) * 3
    tr.gradients()
    torch.cuda.synchronize()
    grad = tr.grad.cpu().numpy().reshape(PD.NETS, PD.NPARAM)
    loss = tr.loss.cpu().numpy()
    shadow = tr.shadow.cpu().numpy().reshape(PD.NETS, PD.NPARAM)
    samples = tr.samples.cpu().numpy().view(np.uint64)
    fb = fields.cpu().numpy().reshape(F, N, N, N)
    ib = tr.item_begin.cpu().numpy()
    items = tr.items.cpu().numpy().view(np.uint32).reshape(-1, 4)
    for net in range(PD.NETS):
        lv, cls = net // 7 + 1, net % 7 + 1
        s = PR.level_stride(lv)
        its = items[ib[net]:ib[net + 1]]
        sm = np.concatenate([samples[a:a + c] for _, a, c, _ in its])
        f = (sm >> np.uint64(32)).astype(np.int64)
        e = (sm & np.uint64(0xFFFFFFFF)).astype(np.int64)
        I, J, K = e // (N * N), (e // N) % N, e % N
        xs, bases, tgts = [], [], []
        for ff in range(F):
            sel = f == ff
            base = PR.interp_pred(fb[ff], N, s, cls, I[sel], J[sel], K[sel])
            xs.append(PR.stencil_inputs(fb[ff], N, s, base, I[sel], J[sel], K[sel], int(tr.s_in[lv - 1])))
            bases.append(base)
            tgts.append(fb[ff][I[sel], J[sel], K[sel]])
        order = np.concatenate([np.flatnonzero(f == ff) for ff in range(F)])
        inv = np.empty_like(order)
        inv[order] = np.arange(order.size)
        x = np.concatenate(xs)[inv]
        base = np.concatenate(bases)[inv]
        tgt = np.concatenate(tgts)[inv]
        w = shadow[net].astype(np.float64)
        L, g, absg = PR.train_forward_backward(x, base, tgt, w[:432].reshape(16, 27), w[432:448], w[448:464],
                                               w[464], tr.s1, tr.s2)
        # float32 sums of n terms: |error| <= ~n * 2^-23 * sum|terms| (+ the 1/n rounding)
        n = x.shape[0]
        tol = lambda a: 4 * n * 2.0 ** -23 * a + 1e-30
        assert abs(loss[net] - L) <= tol(L)
        got = grad[net]
        for name, sl in (("w1", slice(0, 432)), ("b1", slice(432, 448)), ("w2", slice(448, 464)),
                         ("b2", slice(464, 465))):
            ref = np.atleast_1d(g[name]).reshape(-1)
            bound = tol(np.atleast_1d(absg[name]).reshape(-1))
            assert np.all(np.abs(got[sl] - ref) <= bound), (net, name)


def test_freeze_matches_rint_clamp():
    N = 16
    fields = torch.zeros(N ** 3, dtype=torch.int32, device=DEV)
    tr = PD.Trainer(fields, N, samples_per_net=16, seed=0)
    tr.shadow.copy_(torch.randn(tr.shadow.shape, generator=torch.Generator(DEV).manual_seed(2), device=DEV) * 300)
    p = PD.params_from_device(tr.freeze())
    w = tr.shadow.cpu().numpy().astype(np.float64).reshape(PD.NETS, PD.NPARAM)
    W1, B1, W2, B2, _ = PR.fake_quant(w[:, :432], w[:, 432:448], w[:, 448:464], w[:, 464])
    w1 = np.frombuffer(bytes(p.w1), dtype=np.int8).reshape(3, 7, 16, 28)
    assert np.array_equal(w1[..., :27].reshape(PD.NETS, 432), W1.astype(np.int8))
    assert np.all(w1[..., 27] == 0)
    assert np.array_equal(np.frombuffer(bytes(p.b1), dtype=np.int32).reshape(PD.NETS, 16), B1.astype(np.int32))
    assert np.array_equal(np.frombuffer(bytes(p.w2), dtype=np.int8).reshape(PD.NETS, 16), W2.astype(np.int8))
    assert np.array_equal(np.frombuffer(bytes(p.b2), dtype=np.int32), B2.astype(np.int32))


def test_trained_network_beats_interpolation_on_held_out_fields():
    """Quantize small k^-3 fields (ABS 1e-3) with the CUDA quantizer, train
    on 6 fields, evaluate on 3 others: the learned residuals must have lower
    entropy than interpolation, and decode back to the bins exactly."""
    N = 96
    bins = []
    for s in range(9):
        x = synth.grf(N, seed=s, device=DEV)
        q = P.quantize(x, "abs", 1e-3)
        bins.append(q)
    train = torch.cat([q.bins for q in bins[:6]])
    rng = np.random.default_rng(0)
    s_in = PD.choose_s_in(bins[0].bins.cpu().numpy(), N, rng)
    tr = PD.Trainer(train, N, samples_per_net=8192, seed=1, s_in=s_in)
    first = None
    for it in range(150):
        tr.step()
        if it == 0:
            first = tr.mean_squared_residual()
    assert tr.mean_squared_residual() < first
    params = tr.freeze()
    gain = []
    for q in bins[6:]:
        r0 = PD.residuals(q.bins, N)
        r1 = PD.residuals(q.bins, N, params)
        b0, _ = PD.bits_per_value(r0, N, q.mask)
        b1, _ = PD.bits_per_value(r1, N, q.mask)
        gain.append(b0 - b1)
        assert torch.equal(PD.reconstruct(r1, N, params), q.bins)
    assert min(gain) > 0, gain


def test_checkpoint_resume_is_exact(tmp_path):
    """Training resumed from a state_dict continues bit for bit as if it had
    not stopped; frozen parameters survive save_params / load_params."""
    N = 32
    fields = torch.cat([torch.from_numpy(
        np.rint(synth.grf(N, seed=s).numpy() / 2e-3).astype(np.int32)) for s in range(2)]).to(DEV)
    a = PD.Trainer(fields, N, samples_per_net=600, seed=4, s_in=(3, 3, 2))
    for _ in range(5):
        a.step()
    st = a.state_dict()
    torch.save(st, tmp_path / "ckpt.pt")
    for _ in range(5):
        a.step()
    b = PD.Trainer(fields, N, samples_per_net=600, seed=4, s_in=(3, 3, 2))
    b.load_state_dict(torch.load(tmp_path / "ckpt.pt", weights_only=False))
    for _ in range(5):
        b.step()
    torch.cuda.synchronize()
    assert torch.equal(a.shadow, b.shadow) and a.t == b.t
    fa = a.freeze()
    PD.save_params(fa, tmp_path / "params.bin")
    fb = PD.load_params(tmp_path / "params.bin", DEV)
    assert torch.equal(fa, fb)
    assert torch.equal(PD.residuals(fields[:N ** 3], N, fa), PD.residuals(fields[:N ** 3], N, fb))

