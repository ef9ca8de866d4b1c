"""The allocation-free decoder (boa_decode_cdfs_static) against the
allocating one (boa_debug_decode_cdfs).

Some callers of this library cannot allocate device memory once running (a
data-acquisition process with a GPU memory budget fixed at start-up, or a host
framework whose own pool owns all device memory); for them the decoder keeps
its scratch in a static device array.  This file is collected last so that a
run stopping at the first failure has already run every other test.
"""
import numpy as np
import pytest

from paper_2511_11337_b300 import synth

pytestmark = pytest.mark.gpu


def _case(seed, adversarial):
    g = np.random.default_rng(seed)
    lens = [int(x) for x in g.integers(0, 900, 7)] + [1, 0]
    hist, syms = synth.random_histograms(sum(lens), seed=seed, adversarial=adversarial)
    cdf = np.zeros((hist.shape[0], 257), np.uint32)
    cdf[:, 1:] = np.cumsum(hist, axis=1)
    cdf_list, sym_list, o = [], [], 0
    for n in lens:
        cdf_list.append(cdf[o:o + n]); sym_list.append(syms[o:o + n]); o += n
    return lens, cdf_list, sym_list


def test_static_decoder_matches_allocating_decoder():
    import torch
    from paper_2511_11337_b300 import api, build
    build.build()
    for call, adversarial in enumerate([False, True]):          # two calls in a row
        lens, cdf_list, sym_list = _case(800 + call, adversarial)
        coded = api.encode_cdfs(cdf_list, sym_list)
        ref = api.decode_cdfs(cdf_list, coded)                 # existing (allocating) entry point
        stride = max(len(c) for c in coded)
        inb = np.zeros(len(coded) * stride, np.uint8)
        for i, c in enumerate(coded):
            inb[i * stride:i * stride + len(c)] = np.frombuffer(c, np.uint8)
        d_cdf = torch.from_numpy(np.concatenate(cdf_list).astype(np.uint32).view(np.int32)).cuda()
        d_in = torch.from_numpy(inb).cuda()
        d_syms = torch.full((max(sum(lens), 1),), 0xAB, dtype=torch.uint8, device="cuda")
        torch.cuda.synchronize()
        api.decode_cdfs_static(lens, d_cdf.data_ptr(), d_in.data_ptr(), stride, [len(c) for c in coded],
                               d_syms.data_ptr())
        got = d_syms.cpu().numpy()
        o = 0
        for n, r, s in zip(lens, ref, sym_list):
            assert np.array_equal(got[o:o + n], r) and np.array_equal(r, s)
            o += n


def _static_decode(lens, cdf_list, coded):
    """Sequences through boa_decode_cdfs_static (device buffers in and out)."""
    import torch
    from paper_2511_11337_b300 import api
    stride = max(max(len(c) for c in coded), 1)
    inb = np.zeros(len(coded) * stride, np.uint8)
    for i, c in enumerate(coded):
        inb[i * stride:i * stride + len(c)] = np.frombuffer(c, np.uint8)
    d_cdf = torch.from_numpy(np.concatenate(cdf_list).astype(np.uint32).view(np.int32)).cuda()
    d_in = torch.from_numpy(inb).cuda()
    d_syms = torch.full((max(sum(lens), 1),), 0xAB, dtype=torch.uint8, device="cuda")
    torch.cuda.synchronize()
    api.decode_cdfs_static(lens, d_cdf.data_ptr(), d_in.data_ptr(), stride, [len(c) for c in coded],
                           d_syms.data_ptr())
    got = d_syms.cpu().numpy()
    out, o = [], 0
    for n in lens:
        out.append(got[o:o + n])
        o += n
    return out


@pytest.mark.parametrize("n_seq", [3000, 65536])
def test_static_decoder_many_sequences(n_seq):
    """More sequences than the prefix-sum block has threads (several counts
    per thread), up to the stated limit of 65536, each with a few symbols or
    none; two calls in a row, against the allocating decoder."""
    from paper_2511_11337_b300 import api
    for call in range(2):
        g = np.random.default_rng(1000 * n_seq + call)
        if n_seq <= 4096:
            lens = [int(x) for x in g.integers(0, 5, n_seq)]
            hist, syms = synth.random_histograms(sum(lens), seed=n_seq + call, adversarial=call == 1)
            cdf = np.zeros((hist.shape[0], 257), np.uint32)
            cdf[:, 1:] = np.cumsum(hist, axis=1)
        else:
            # at the limit: zero or one symbol each, uniform CDF C(s) = 256 s
            lens = [int(x) for x in g.integers(0, 2, n_seq)]
            syms = g.integers(0, 256, sum(lens)).astype(np.uint8)
            cdf = np.tile((np.arange(257, dtype=np.uint32) * 256)[None, :], (len(syms), 1))
        cdf_list, sym_list, o = [], [], 0
        for n in lens:
            cdf_list.append(cdf[o:o + n]); sym_list.append(syms[o:o + n]); o += n
        coded = api.encode_cdfs(cdf_list, sym_list)
        ref = api.decode_cdfs(cdf_list, coded)
        got = _static_decode(lens, cdf_list, coded)
        for r, s, x in zip(ref, sym_list, got):
            assert np.array_equal(x, r) and np.array_equal(r, s)


def test_static_decoder_limits_and_corruption():
    import torch
    from paper_2511_11337_b300 import api
    with pytest.raises(api.BoaError) as e:
        api.decode_cdfs_static([1] * 65537, 0, 0, 1, [1] * 65537, 0)
    assert e.value.code == 1
    lens, cdf_list, sym_list = _case(900, False)
    coded = api.encode_cdfs(cdf_list, sym_list)
    stride = max(len(c) for c in coded)
    inb = np.zeros(len(coded) * stride, np.uint8)
    for i, c in enumerate(coded):
        inb[i * stride:i * stride + len(c)] = np.frombuffer(c, np.uint8)
    d_cdf = torch.from_numpy(np.concatenate(cdf_list).astype(np.uint32).view(np.int32)).cuda()
    d_in = torch.from_numpy(inb).cuda()
    d_syms = torch.zeros(max(sum(lens), 1), dtype=torch.uint8, device="cuda")
    sizes = [len(c) for c in coded]
    k = int(np.argmax(lens))
    sizes[k] -= 3                                             # truncate one sequence
    torch.cuda.synchronize()
    with pytest.raises(api.BoaError) as e:
        api.decode_cdfs_static(lens, d_cdf.data_ptr(), d_in.data_ptr(), stride, sizes, d_syms.data_ptr())
    assert e.value.code == 7
