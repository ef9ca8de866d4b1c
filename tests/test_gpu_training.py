"""Differentiation: the hand-written selective-scan backward against the
FP64 oracle's reverse-mode gradient, and the whole predictor's gradient
against central finite differences of the oracle's cross-entropy; then a
short training run that lowers the loss and compresses better."""
import math
import os

import numpy as np
import pytest

from oracle import oracle as O
from paper_2511_11337_b300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def tr():
    from paper_2511_11337_b300 import build
    build.build()
    from paper_2511_11337_b300 import train as T
    return T


def test_scan_backward_matches_oracle_gradient(tr):
    import torch
    g = np.random.default_rng(3)
    Bsz, T, E, N = 2, 150, 130, 16            # ragged channel block, 3 chunks of 64 with a tail
    u = g.normal(size=(Bsz, T, E)).astype(np.float32)
    delta = np.log1p(np.exp(g.normal(-1, 0.5, size=(Bsz, T, E)))).astype(np.float32)
    A = (-np.exp(g.normal(size=(E, N)))).astype(np.float32)
    Bm = g.normal(size=(Bsz, T, N)).astype(np.float32)
    Cm = g.normal(size=(Bsz, T, N)).astype(np.float32)
    D = g.normal(size=E).astype(np.float32)
    dy = g.normal(size=(Bsz, T, E)).astype(np.float32)
    ts = [torch.tensor(x, device="cuda", requires_grad=True) for x in (u, delta, A, Bm, Cm, D)]
    y = tr.selective_scan(*ts, chunk=64)
    y.backward(torch.tensor(dy, device="cuda"))
    got = {k: t.grad.cpu().numpy().astype(np.float64) for k, t in zip(["u", "delta", "A", "B", "C", "D"], ts)}
    ref = {k: 0.0 for k in got}
    for b in range(Bsz):
        yo = O.selective_scan(u[b], delta[b], A, Bm[b], Cm[b], D)
        assert np.allclose(y[b].detach().cpu().numpy(), yo, rtol=1e-4, atol=1e-4)
        gr = O.selective_scan_grad(u[b], delta[b], A, Bm[b], Cm[b], D, dy[b])
        for k in ("A", "D"):
            ref[k] = ref[k] + gr[k]
        for k in ("u", "delta", "B", "C"):
            got_b = got[k][b]
            assert np.allclose(got_b, gr[k], rtol=2e-3, atol=2e-3 * np.abs(gr[k]).max()), k
    for k in ("A", "D"):
        assert np.allclose(got[k], ref[k], rtol=2e-3, atol=2e-3 * np.abs(ref[k]).max()), k


def test_model_gradient_matches_oracle_finite_differences(tr, tmp_path):
    """d_model 32, 2 layers, FP32 throughout: autograd through the library's
    scan vs central differences of the FP64 oracle's total cross-entropy."""
    import torch
    shape = synth.ModelShape(d_model=32, n_layer=2)
    g = np.random.default_rng(9)
    w = synth.init_weights(shape, seed=9)
    for k, a in w.items():          # non-trivial values everywhere
        if not k.endswith("A_log"):
            w[k] = (a + g.normal(0, 0.1, a.shape)).astype(np.float32)
    data = bytes(g.integers(0, 256, 40, dtype=np.uint8))
    model = tr.TorchPredictor(shape, w).cuda()
    tok = torch.tensor(np.frombuffer(data, np.uint8)[None].copy(), device="cuda")
    loss = tr.cross_entropy_bytes(model(tok, bf16=False), tok) * (len(data) - 1) * math.log(256.0)
    loss.backward()

    def oracle_nll(weights):
        path = str(tmp_path / "fd.boaw")
        synth.write_model(path, shape, weights)
        lp = O.Model(path).logprobs(data)
        idx = np.frombuffer(data, np.uint8)[1:]
        return -float(lp[np.arange(len(idx)), idx].sum()) * math.log(2.0)

    picks = [("embed", (data[3], 5)), ("layers.0.in_proj.w", (7, 3)), ("layers.0.in_proj.w", (70, 11)),
             ("layers.1.conv.w", (9, 3)), ("layers.0.conv.b", (4,)), ("layers.1.x_proj.w", (2, 17)),
             ("layers.0.x_proj.w", (20, 40)), ("layers.1.dt_proj.w", (30, 1)), ("layers.0.dt_proj.b", (12,)),
             ("layers.1.A_log", (5, 7)), ("layers.0.D", (33,)), ("layers.1.out_proj.w", (3, 50)),
             ("layers.0.ln_a.w", (6,)), ("layers.1.ln_b.b", (8,)), ("head.w", (data[10], 4)), ("head.b", (data[20],))]
    for name, idx in picks:
        h = 1e-3
        wp = {k: v.copy() for k, v in w.items()}
        wm = {k: v.copy() for k, v in w.items()}
        wp[name][idx] += h
        wm[name][idx] -= h
        fd = (oracle_nll(wp) - oracle_nll(wm)) / (float(wp[name][idx]) - float(wm[name][idx]))
        ag = float(model.w(name).grad[idx].item())
        assert abs(ag - fd) <= 2e-2 * abs(fd) + 2e-3, (name, idx, ag, fd)


def test_training_lowers_loss_and_compresses(tr, tmp_path):
    import torch
    from paper_2511_11337_b300 import api
    shape = synth.ModelShape(d_model=64, n_layer=2)
    data = synth.cms_records(2_000_000, seed=5000)
    held = synth.cms_records(200_000, seed=5001)
    model = tr.TorchPredictor(shape, synth.init_weights(shape, seed=1)).cuda()
    hist = tr.train(model, data, steps=120, batch=16, seqlen=1024, lr=3e-3, log_every=20)
    assert hist[-1][1] < 0.5 * hist[0][1], hist
    path = str(tmp_path / "trained.boaw")
    model.save(path)
    m = api.Model(path)
    streams = synth.split_equal(held, 24)
    comp = m.compress(streams)
    assert m.decompress(comp, [len(s) for s in streams]) == streams
    ratio = sum(map(len, streams)) / sum(map(len, comp))
    print(f"trained d64 model: loss {hist[0][1]:.3f} -> {hist[-1][1]:.3f} bytes/byte, held-out ratio {ratio:.2f}")
    assert ratio > 1.3            # random-init weights give about 1.0
    om = O.Model(path)
    ref = om.compress(streams[0][:3000])
    assert abs(len(m.compress([streams[0][:3000]])[0]) - len(ref)) / len(ref) <= 0.005
