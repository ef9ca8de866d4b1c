"""Training the BOA predictor on byte streams (paper, "Entropy-Based
Compression and Cross-Entropy Loss": minimising the base-256 cross-entropy
minimises the code length).

Two routes.  train_native drives the library's own training step
(boa_train_step: forward, backward and AdamW in its kernels; FP32 on the
CUDA cores, or for a model loaded in the BF16 form the projections and
their gradients on the tensor cores with FP32 master weights).  The
autograd route (TorchPredictor, train) runs the selective scan, forward and
backward, in the library's hand-written kernels (boa_scan_train_fwd /
boa_scan_train_bwd) behind a torch.autograd.Function, with states recomputed
per chunk of 256 steps instead of stored, and the rest of the block
(norms, projections, depthwise conv, activations) as torch operations, the
projections in BF16 under autocast with FP32 master weights.  Parameters
mirror the weight-file layout, so either route's model exports to a file
that boa_load_model reads.
"""
from __future__ import annotations

import ctypes as C
import math

import numpy as np
import torch
import torch.nn.functional as F

from . import synth
from ._lib import check, load

SCAN_CHUNK = 256


class SelectiveScanFn(torch.autograd.Function):
    """y = scan(u, delta, A, B, C, D) over [Bsz, T, E] with h_0 = 0."""

    @staticmethod
    def forward(ctx, u, delta, A, Bm, Cm, D, chunk: int = SCAN_CHUNK):
        u, delta, Bm, Cm = (t.float().contiguous() for t in (u, delta, Bm, Cm))
        A, D = A.float().contiguous(), D.float().contiguous()
        Bsz, T, E = u.shape
        N = A.shape[1]
        nck = (T + chunk - 1) // chunk
        y = torch.empty_like(u)
        hin = torch.empty((Bsz, nck, N, E), device=u.device, dtype=torch.float32)
        stream = torch.cuda.current_stream(u.device).cuda_stream
        check(load().boa_scan_train_fwd(Bsz, T, E, N, chunk, *(C.c_void_p(t.data_ptr()) for t in
                                                              (u, delta, A, Bm, Cm, D, y, hin)), C.c_void_p(stream)))
        ctx.save_for_backward(u, delta, A, Bm, Cm, D, hin)
        ctx.chunk = chunk
        return y

    @staticmethod
    def backward(ctx, dy):
        u, delta, A, Bm, Cm, D, hin = ctx.saved_tensors
        chunk = ctx.chunk
        dy = dy.float().contiguous()
        Bsz, T, E = u.shape
        N = A.shape[1]
        nblk = (E + 127) // 128
        dev = u.device
        scratch = torch.empty((Bsz, chunk, N, E), device=dev, dtype=torch.float32)
        du, ddelta = torch.empty_like(u), torch.empty_like(u)
        dA_p = torch.empty((Bsz, E, N), device=dev, dtype=torch.float32)
        dD_p = torch.empty((Bsz, E), device=dev, dtype=torch.float32)
        dB_p = torch.empty((Bsz, T, nblk, N), device=dev, dtype=torch.float32)
        dC_p = torch.empty((Bsz, T, nblk, N), device=dev, dtype=torch.float32)
        stream = torch.cuda.current_stream(dev).cuda_stream
        check(load().boa_scan_train_bwd(Bsz, T, E, N, chunk, *(C.c_void_p(t.data_ptr()) for t in
                                                              (u, delta, A, Bm, Cm, D, dy, hin, scratch, du, ddelta,
                                                               dA_p, dD_p, dB_p, dC_p)), C.c_void_p(stream)))
        return du, ddelta, dA_p.sum(0), dB_p.sum(2), dC_p.sum(2), dD_p.sum(0), None


def selective_scan(u, delta, A, Bm, Cm, D, chunk: int = SCAN_CHUNK):
    return SelectiveScanFn.apply(u, delta, A, Bm, Cm, D, chunk)


class TorchPredictor(torch.nn.Module):
    """The predictor Q (Alg. 1) as torch parameters named like the weight file."""

    def __init__(self, shape: synth.ModelShape, weights: dict[str, np.ndarray]):
        super().__init__()
        self.shape = shape
        self.params = torch.nn.ParameterDict(
            {k.replace(".", "__"): torch.nn.Parameter(torch.from_numpy(np.array(v, np.float32))) for k, v in
             weights.items()})

    def w(self, name):
        return self.params[name.replace(".", "__")]

    def forward(self, tokens: torch.Tensor, bf16: bool = True) -> torch.Tensor:
        sh = self.shape
        d, E, N, K, r = sh.d_model, sh.d_inner, sh.d_state, sh.d_conv, sh.dt_rank
        x = self.w("embed")[tokens.long()]
        for l in range(sh.n_layer):
            p = f"layers.{l}."
            xn = F.layer_norm(x, (d,), self.w(p + "ln_a.w"), self.w(p + "ln_a.b"), eps=1e-5)
            with torch.autocast("cuda", dtype=torch.bfloat16, enabled=bf16):
                xz = xn @ self.w(p + "in_proj.w").t()
            xz = xz.float()
            xi, z = xz[..., :E], xz[..., E:]
            xc = F.conv1d(F.pad(xi.transpose(1, 2), (K - 1, 0)), self.w(p + "conv.w").unsqueeze(1),
                          self.w(p + "conv.b"), groups=E).transpose(1, 2)
            u = F.silu(xc)
            with torch.autocast("cuda", dtype=torch.bfloat16, enabled=bf16):
                dbc = u @ self.w(p + "x_proj.w").t()
            dbc = dbc.float()
            dlt, Bm, Cm = dbc[..., :r], dbc[..., r:r + N], dbc[..., r + N:]
            delta = F.softplus(dlt @ self.w(p + "dt_proj.w").t() + self.w(p + "dt_proj.b"), threshold=20.0)
            A = -torch.exp(self.w(p + "A_log"))
            y = selective_scan(u, delta, A, Bm, Cm, self.w(p + "D"))
            y = y * F.silu(z)
            with torch.autocast("cuda", dtype=torch.bfloat16, enabled=bf16):
                o = y @ self.w(p + "out_proj.w").t()
            x = x + o.float()
            if sh.ffn_mult:
                with torch.autocast("cuda", dtype=torch.bfloat16, enabled=bf16):
                    hdn = F.gelu(x @ self.w(p + "ffn.w1").t() + self.w(p + "ffn.b1"))
                    o2 = hdn @ self.w(p + "ffn.w2").t() + self.w(p + "ffn.b2")
                x = x + o2.float()
            x = F.layer_norm(x, (d,), self.w(p + "ln_b.w"), self.w(p + "ln_b.b"), eps=1e-5)
        with torch.autocast("cuda", dtype=torch.bfloat16, enabled=bf16):
            logits = x @ self.w("head.w").t() + self.w("head.b")
        return logits.float()

    def export(self) -> dict[str, np.ndarray]:
        return {k.replace("__", "."): v.detach().float().cpu().numpy() for k, v in self.params.items()}

    def save(self, path: str) -> None:
        synth.write_model(path, self.shape, self.export())


def cross_entropy_bytes(logits: torch.Tensor, tokens: torch.Tensor) -> torch.Tensor:
    """Mean -log_256 Q(y_t | y_<t) over the predicted positions: bytes per byte."""
    lp = F.log_softmax(logits[:, :-1].float(), dim=-1)
    nll = -lp.gather(-1, tokens[:, 1:].long().unsqueeze(-1)).squeeze(-1)
    return nll.mean() / math.log(256.0)


def batches(data: bytes, batch: int, seqlen: int, seed: int, device):
    """Random windows of seqlen bytes (as a [batch, seqlen] uint8 tensor)."""
    buf = torch.from_numpy(np.frombuffer(data, np.uint8).copy()).to(device)
    g = np.random.Generator(np.random.PCG64(seed))
    n = len(data) - seqlen
    while True:
        starts = torch.from_numpy(g.integers(0, n, batch)).to(device)
        idx = starts[:, None] + torch.arange(seqlen, device=device)[None, :]
        yield buf[idx]


def train(model: TorchPredictor, data: bytes, steps: int, batch: int = 64, seqlen: int = 4096, lr: float = 1e-3,
          weight_decay: float = 0.01, seed: int = 0, log_every: int = 10, bf16: bool = True):
    """AdamW on the base-256 cross-entropy; returns [(step, loss), ...]."""
    dev = next(model.parameters()).device
    opt = torch.optim.AdamW(model.parameters(), lr=lr, weight_decay=weight_decay)
    it = batches(data, batch, seqlen, seed, dev)
    hist = []
    for step in range(steps):
        tok = next(it)
        loss = cross_entropy_bytes(model(tok, bf16=bf16), tok)
        opt.zero_grad(set_to_none=True)
        loss.backward()
        opt.step()
        if step % log_every == 0 or step == steps - 1:
            hist.append((step, float(loss.item())))
    return hist


def train_native(path: str, data: bytes, steps: int, batch: int, seqlen: int, lr: float, seed: int = 0,
                 log_every: int = 10, precision: int = 0, epochs: int = 0):
    """The same loop through the library's own training step (boa_train_step:
    forward, backward and AdamW all in its kernels); returns the model and
    [(step, loss), ...].  With epochs > 0 the batches walk a shuffled order of
    the non-overlapping seqlen-byte windows of data, every window once per
    epoch (steps is then epochs x windows / batch); otherwise each batch
    draws window starts at random."""
    from . import api
    m = api.Model(path, precision=precision)
    buf = np.frombuffer(data, np.uint8)
    g = np.random.Generator(np.random.PCG64(seed))
    order = []
    if epochs > 0:
        n_win = len(buf) // seqlen
        for _ in range(epochs):
            order.extend((g.permutation(n_win) * seqlen).tolist())
        steps = len(order) // batch
    hist = []
    for step in range(steps):
        starts = order[step * batch:(step + 1) * batch] if epochs > 0 else g.integers(0, len(buf) - seqlen, batch)
        loss = m.train_step(np.stack([buf[s:s + seqlen] for s in starts]), lr)
        if step % log_every == 0 or step == steps - 1:
            hist.append((step, loss))
    return m, hist


def main():
    import argparse
    import json
    import os
    import tempfile
    import time

    from . import api
    ap = argparse.ArgumentParser(description="Train the predictor on CMS-like records, then compress held-out data.")
    ap.add_argument("--route", choices=["native", "torch"], default="native",
                    help="native: boa_train_step; torch: autograd with the library's scan kernels")
    ap.add_argument("--train-mb", type=float, default=256.0)
    ap.add_argument("--heldout-mb", type=float, default=64.0)
    ap.add_argument("--steps", type=int, default=300)
    ap.add_argument("--batch", type=int, default=64)
    ap.add_argument("--seqlen", type=int, default=4096)
    ap.add_argument("--lr", type=float, default=1e-3)
    ap.add_argument("--epochs", type=int, default=0,
                    help="native route: passes over every window of the training set (overrides --steps)")
    ap.add_argument("--precision", choices=["fp32", "bf16"], default="fp32",
                    help="native route: the training step's arithmetic (bf16: tensor-core projections)")
    ap.add_argument("--eval-precision", choices=["fp32", "tf32x3", "bf16", "fp8"], default="tf32x3",
                    help="the form that compresses the held-out data with the trained weights")
    ap.add_argument("--out", default="")
    args = ap.parse_args()
    prec = {"fp32": api.PREC_FP32, "tf32x3": api.PREC_TF32X3, "bf16": api.PREC_BF16, "fp8": api.PREC_FP8}
    shape = synth.PAPER_SCALE
    n_train = int(args.train_mb * 1e6)
    stream = synth.cms_records(n_train + int(args.heldout_mb * 1e6), seed=5000)
    train_data, held = stream[:n_train], stream[n_train:]
    path = args.out or os.path.join(tempfile.mkdtemp(), "trained.boaw")
    init = os.path.join(tempfile.mkdtemp(), "init.boaw")
    synth.make_model_file(init, shape, seed=2)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    if args.route == "native":
        nm, hist = train_native(init, train_data, args.steps, args.batch, args.seqlen, args.lr,
                                precision=prec[args.precision], epochs=args.epochs)
        args.steps = hist[-1][0] + 1
        nm.save(path)
    else:
        model = TorchPredictor(shape, synth.init_weights(shape, seed=2)).cuda()
        hist = train(model, train_data, args.steps, args.batch, args.seqlen, args.lr)
        model.save(path)
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t0
    m = api.Model(path, precision=prec[args.eval_precision])
    streams = synth.split_equal(held, max(1, len(held) // 16384))
    flat, in_off = api.pack(streams)
    lens = np.diff(in_off)
    out_off = api.compressed_slot_offsets(lens)
    d_in = torch.from_numpy(flat.copy()).cuda()
    d_out = torch.zeros(int(out_off[-1]), dtype=torch.uint8, device="cuda")
    d_dec = torch.zeros(len(flat), dtype=torch.uint8, device="cuda")
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    sizes = m.compress_device(d_in.data_ptr(), in_off, d_out.data_ptr(), out_off)
    t_c = time.perf_counter() - t0
    t0 = time.perf_counter()
    m.decompress_device(d_out.data_ptr(), out_off, lens, d_dec.data_ptr(), in_off, in_sizes=sizes)
    t_d = time.perf_counter() - t0
    ok = bool(torch.equal(d_dec, d_in))
    total = int(len(flat))
    tokens = args.steps * args.batch * (args.seqlen - 1)
    print(json.dumps({"route": args.route, "precision": args.precision, "epochs": args.epochs,
                      "train_bytes": n_train, "eval_precision": args.eval_precision,
                      "train_steps": args.steps, "train_s": t_train,
                      "train_tokens_per_s": tokens / t_train, "loss_bytes_per_byte": hist,
                      "heldout_bytes": total, "compressed_bytes": int(sizes.sum()),
                      "compression_ratio": total / int(sizes.sum()), "compress_MBps": total / 1e6 / t_c,
                      "decompress_MBps": total / 1e6 / t_d, "lossless": ok}))


if __name__ == "__main__":
    main()
