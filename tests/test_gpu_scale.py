"""The uneven ATLAS-like / CMS-like mix at scale, on the benchmark model.

2000 streams of log-uniform length 1 KB .. 362 KB (several of them longer
than 256 KB), each cut into 16 KB chunks as the .boa container stores them,
compressed and decompressed as one batch through fewer slots than chunks, so
slots take queued chunks as they finish (paper, section "Coders &
Parallelisation": all active streams stepped together).  Checked: a
lossless round trip of every chunk; the code length of sampled chunks (taken
from the big batch) within 0.5 % of the FP64 oracle's; a chunk compressed
alone gives the same bytes as inside the batch.
"""
import os

import numpy as np
import pytest

from oracle import oracle as O
from paper_2511_11337_b300 import api, synth

pytestmark = pytest.mark.gpu

CHUNK = 16384


@pytest.fixture(scope="module")
def paper_model(model_dir):
    return synth.make_model_file(os.path.join(model_dir, "paper_scale.boaw"), synth.PAPER_SCALE, seed=2)


def test_uneven_mix_2000_streams(paper_model):
    src = synth.mixed_workload(2000, seed=3100, lo_log2=10.0, hi_log2=18.5)
    lens = np.array([len(s) for s in src])
    assert (lens >= 262144).sum() >= 5 and lens.min() >= 1024
    chunks = [s[i:i + CHUNK] for s in src for i in range(0, len(s), CHUNK)]
    m = api.Model(paper_model, precision=api.PREC_TF32X3, max_slots=2048)
    assert len(chunks) > 2 * 2048                         # queued chunks refill slots
    comp = m.compress(chunks)
    assert m.decompress(comp, [len(c) for c in chunks]) == chunks
    # 16 chunks of 1-4 KB (a stream's tail, or a whole short stream),
    # spread evenly over the batch, against the oracle
    cand = [i for i, c in enumerate(chunks) if 1024 <= len(c) <= 4096]
    order = [cand[k] for k in np.linspace(0, len(cand) - 1, 16).astype(int)]
    sample = [chunks[i] for i in order]
    om = O.Model(paper_model)
    ref = om.compress_batch(sample, n_threads=min(16, os.cpu_count() or 1))
    got = sum(len(comp[i]) for i in order)
    want = sum(map(len, ref))
    assert abs(got - want) <= 0.005 * want, (got, want)
    # batch invariance at this scale: a sampled chunk alone
    for i in order[:2]:
        assert m.compress([chunks[i]])[0] == comp[i]
    m.close()
