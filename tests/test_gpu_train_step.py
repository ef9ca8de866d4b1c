"""The native training step (boa_train_step): its gradient against central
finite differences of the FP64 oracle's cross-entropy and against torch
autograd of the same predictor, the AdamW update, a short training run that
then compresses held-out data, and the weight-file round trip."""
import math
import os

import numpy as np
import pytest

from oracle import oracle as O
from paper_2511_11337_b300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def api():
    from paper_2511_11337_b300 import api as A, build
    build.build()
    return A


def noisy_weights(shape, seed):
    """Random weights with every tensor away from its special init values."""
    g = np.random.default_rng(seed)
    w = synth.init_weights(shape, seed=seed)
    for k, a in w.items():
        if not k.endswith("A_log"):
            w[k] = (a + g.normal(0, 0.1, a.shape)).astype(np.float32)
    return w


def flat_offsets(shape):
    out, o = {}, 0
    for name, dims in synth.tensor_specs(shape):
        out[name] = (o, dims)
        o += int(np.prod(dims))
    return out, o


def test_gradient_matches_oracle_finite_differences(api, tmp_path):
    """d_model 64, 2 layers, two sequences of 33 bytes: boa_debug_train_grad
    against central differences of the FP64 oracle's cross-entropy (mean over
    the 64 predicted positions, in bytes per byte)."""
    shape = synth.ModelShape(d_model=64, n_layer=2)
    w = noisy_weights(shape, 9)
    path = str(tmp_path / "g.boaw")
    synth.write_model(path, shape, w)
    g = np.random.default_rng(4)
    batch = g.integers(0, 256, size=(2, 33), dtype=np.uint8)
    m = api.Model(path)
    loss, grad = m.train_grad(batch)
    offs, total = flat_offsets(shape)
    assert grad.shape == (total,) and m.param_count == total
    rows = batch.shape[0] * (batch.shape[1] - 1)

    def oracle_loss(weights):
        p = str(tmp_path / "fd.boaw")
        synth.write_model(p, shape, weights)
        om = O.Model(p)
        nll = 0.0
        for seq in batch:
            lp = om.logprobs(bytes(seq))
            nll -= float(lp[np.arange(len(seq) - 1), seq[1:]].sum())     # log2 p
        return nll / 8.0 / rows                                           # bytes per byte

    assert abs(loss - oracle_loss(w)) < 1e-4 * max(1.0, loss)
    picks = [("embed", (int(batch[0, 3]), 5)), ("layers.0.in_proj.w", (7, 3)), ("layers.0.in_proj.w", (200, 11)),
             ("layers.1.conv.w", (9, 3)), ("layers.1.conv.w", (40, 0)), ("layers.0.conv.b", (4,)),
             ("layers.1.x_proj.w", (2, 17)), ("layers.0.x_proj.w", (10, 40)), ("layers.0.x_proj.w", (30, 100)),
             ("layers.1.dt_proj.w", (30, 1)), ("layers.0.dt_proj.b", (12,)), ("layers.1.A_log", (5, 7)),
             ("layers.0.D", (33,)), ("layers.1.out_proj.w", (3, 50)), ("layers.0.ln_a.w", (6,)),
             ("layers.0.ln_a.b", (60,)), ("layers.1.ln_b.w", (8,)), ("layers.1.ln_b.b", (8,)),
             ("head.w", (int(batch[1, 10]), 4)), ("head.b", (int(batch[0, 20]),))]
    for name, idx in picks:
        h = 2e-3
        wp = {k: v.copy() for k, v in w.items()}
        wm = {k: v.copy() for k, v in w.items()}
        wp[name][idx] += h
        wm[name][idx] -= h
        fd = (oracle_loss(wp) - oracle_loss(wm)) / (float(wp[name][idx]) - float(wm[name][idx]))
        o, dims = offs[name]
        ag = float(grad[o + int(np.ravel_multi_index(idx, dims))])
        assert abs(ag - fd) <= 2e-2 * abs(fd) + 2e-4, (name, idx, ag, fd)


def test_gradient_matches_torch_autograd(api, tmp_path):
    """Every entry of the gradient against torch autograd of the same FP32
    predictor (train.TorchPredictor, FP32 projections)."""
    import torch
    from paper_2511_11337_b300 import train as T
    torch.backends.cudnn.allow_tf32 = False
    torch.backends.cuda.matmul.allow_tf32 = False
    shape = synth.ModelShape(d_model=64, n_layer=2)
    w = noisy_weights(shape, 3)
    path = str(tmp_path / "t.boaw")
    synth.write_model(path, shape, w)
    batch = np.random.default_rng(5).integers(0, 256, size=(3, 300), dtype=np.uint8)
    loss, grad = api.Model(path).train_grad(batch)
    model = T.TorchPredictor(shape, w).cuda()
    tok = torch.tensor(batch, device="cuda")
    ref = T.cross_entropy_bytes(model(tok, bf16=False), tok)
    ref.backward()
    assert abs(loss - float(ref)) < 1e-4
    offs, _ = flat_offsets(shape)
    for name, (o, dims) in offs.items():
        got = grad[o:o + int(np.prod(dims))].reshape(dims)
        exp = model.w(name).grad.detach().cpu().numpy()
        scale = max(float(np.abs(exp).max()), 1e-6)
        assert np.abs(got - exp).max() <= 2e-3 * scale + 1e-7, (name, float(np.abs(got - exp).max()), scale)


def test_step_is_adamw_and_deterministic(api, tmp_path):
    """Two models given the same batches take bit-identical steps; the first
    step moves every weight by lr * (sign of its gradient + decay) as AdamW's
    first bias-corrected step does."""
    shape = synth.ModelShape(d_model=64, n_layer=2)
    w = noisy_weights(shape, 7)
    path = str(tmp_path / "s.boaw")
    synth.write_model(path, shape, w)
    batch = np.random.default_rng(8).integers(0, 256, size=(4, 129), dtype=np.uint8)
    a, b = api.Model(path), api.Model(path)
    _, g = a.train_grad(batch)
    lr = 1e-3
    la = a.train_step(batch, lr)
    lb = b.train_step(batch, lr)
    assert la == lb
    pa, pb = str(tmp_path / "a.boaw"), str(tmp_path / "b.boaw")
    a.save(pa)
    b.save(pb)
    assert open(pa, "rb").read() == open(pb, "rb").read()
    assert a.fingerprint == b.fingerprint != api.Model(path).fingerprint
    _, wa = synth.read_model(pa)
    offs, _ = flat_offsets(shape)
    for name, (o, dims) in offs.items():
        p0 = w[name].astype(np.float64)
        gn = g[o:o + int(np.prod(dims))].reshape(dims).astype(np.float64)
        # first AdamW step: mhat / (sqrt(vhat) + eps) = g / (|g| + eps)
        exp = p0 * (1 - lr * 0.01) - lr * gn / (np.abs(gn) + 1e-8)
        assert np.allclose(wa[name], exp, rtol=1e-5, atol=2e-6), name


def test_training_lowers_loss_and_compresses(api, tmp_path):
    """120 steps of boa_train_step on CMS-like records (d_model 64, 2 layers,
    16 x 1024 bytes per batch) halve the loss; the saved weights reload with
    the same fingerprint and compress the held-out tail of the same record
    stream losslessly and better than random-init weights.  (Another
    generator seed has other run numbers and constant columns, which a model
    trained this long predicts confidently and wrongly.)"""
    shape = synth.ModelShape(d_model=64, n_layer=2)
    path = synth.make_model_file(str(tmp_path / "init.boaw"), shape, seed=1)
    stream = synth.cms_records(2_200_000, seed=5000)
    data = np.frombuffer(stream[:2_000_000], np.uint8)
    held = stream[2_000_000:]
    m = api.Model(path)
    g = np.random.default_rng(0)
    losses = []
    for step in range(120):
        starts = g.integers(0, len(data) - 1024, 16)
        batch = np.stack([data[s:s + 1024] for s in starts])
        losses.append(m.train_step(batch, 3e-3))
    assert all(math.isfinite(x) for x in losses)
    assert np.mean(losses[-10:]) < 0.5 * np.mean(losses[:3]), (losses[:3], losses[-10:])
    out = str(tmp_path / "trained.boaw")
    m.save(out)
    m2 = api.Model(out)
    assert m2.fingerprint == m.fingerprint
    streams = synth.split_equal(held, 24)
    comp = m2.compress(streams)
    assert m2.decompress(comp, [len(s) for s in streams]) == streams
    assert m.compress(streams) == comp
    ratio = sum(map(len, streams)) / sum(map(len, comp))
    print(f"native training: loss {np.mean(losses[:3]):.3f} -> {np.mean(losses[-10:]):.3f} bytes/byte, "
          f"held-out ratio {ratio:.2f}")
    assert ratio > 1.3


def test_save_untrained_model_is_the_file(api, tmp_path, tiny_model_path):
    m = api.Model(tiny_model_path)
    out = str(tmp_path / "copy.boaw")
    m.save(out)
    assert open(out, "rb").read() == open(tiny_model_path, "rb").read()
    assert api.Model(out).fingerprint == m.fingerprint


def test_train_step_rejects_bad_batches(api, tiny_model_path):
    m = api.Model(tiny_model_path)
    with pytest.raises(api.BoaError):
        m.train_step(np.zeros((2, 1), np.uint8), 1e-3)
    with pytest.raises(api.BoaError):
        m.train_step(np.zeros((0, 16), np.uint8), 1e-3)


def test_bf16_training_step(api, tmp_path):
    """A BF16 model trains with its projections, input gradients and weight
    gradients on the tensor cores (BF16 operands, FP32 accumulation, FP32
    master weights).  Its loss and gradient against the FP32 step's on the
    same weights and batch (d_model 128, 2 layers, 6000 predicted positions:
    two 4096-row parts of the weight gradients, the second one ragged); two
    BF16 models take bit-identical steps; 60 steps on CMS-like records halve
    the loss and the result compresses held-out data losslessly."""
    shape = synth.ModelShape(d_model=128, n_layer=2)
    w = noisy_weights(shape, 21)
    path = str(tmp_path / "b.boaw")
    synth.write_model(path, shape, w)
    batch = np.random.default_rng(22).integers(0, 256, size=(24, 251), dtype=np.uint8)
    l32, g32 = api.Model(path).train_grad(batch)
    mb = api.Model(path, precision=api.PREC_BF16)
    l16, g16 = mb.train_grad(batch)
    assert abs(l16 - l32) <= 1e-2 * abs(l32), (l16, l32)
    offs, _ = flat_offsets(shape)
    worst = 0.0
    for name, (o, dims) in offs.items():
        n = int(np.prod(dims))
        a, b = g32[o:o + n].astype(np.float64), g16[o:o + n].astype(np.float64)
        if np.linalg.norm(a) == 0:
            continue
        rel = np.linalg.norm(b - a) / np.linalg.norm(a)
        worst = max(worst, rel)
        # BF16 rounds every GEMM operand to 8 significant bits (relative 2^-9);
        # errors of that size, propagated through two layers, stay within 5 %
        assert rel <= 0.05, (name, rel)
    print(f"BF16 training gradient: worst per-tensor relative L2 error {worst:.3e}")
    a2 = api.Model(path, precision=api.PREC_BF16)
    assert a2.train_grad(batch)[1].tobytes() == g16.tobytes()
    # a short run
    stream = synth.cms_records(1_300_000, seed=5000)
    data = np.frombuffer(stream[:1_200_000], np.uint8)
    held = stream[1_200_000:]
    m = api.Model(synth.make_model_file(str(tmp_path / "i.boaw"), shape, seed=1), precision=api.PREC_BF16)
    g = np.random.default_rng(0)
    losses = []
    for step in range(60):
        starts = g.integers(0, len(data) - 1024, 16)
        losses.append(m.train_step(np.stack([data[s:s + 1024] for s in starts]), 3e-3))
    assert all(math.isfinite(x) for x in losses)
    assert np.mean(losses[-5:]) < 0.5 * np.mean(losses[:3]), (losses[:3], losses[-5:])
    streams = synth.split_equal(held, 16)
    comp = m.compress(streams)
    assert m.decompress(comp, [len(s) for s in streams]) == streams
