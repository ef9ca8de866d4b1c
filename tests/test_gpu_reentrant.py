"""Several host threads calling into one model at once.

Every call on a model holds that model's lock for its whole duration, so
concurrent compress / decompress / container calls from several threads run
one after another and must give exactly the bytes of the same calls made in
sequence (include/boa.h, calling conventions).  ctypes releases the GIL
during each library call, so the threads really enter the library together.
"""
import threading

import numpy as np
import pytest

from paper_2511_11337_b300 import api, synth

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("precision", [api.PREC_FP32, api.PREC_TF32X3])
def test_threads_share_one_model(tiny_model_path, precision):
    m = api.Model(tiny_model_path, device=0, precision=precision)
    batches = [[synth.records_stream(7000 + 10 * b + i, 700 + 97 * i + 31 * b) for i in range(5)] for b in range(4)]
    serial = [m.compress(b) for b in batches]
    blob = b"".join(batches[0])
    serial_pack = m.pack(blob, chunk_len=1024)
    results, errors = {}, []

    def work(k):
        try:
            b = batches[k % 4]
            for rep in range(3):
                c = m.compress(b)
                d = m.decompress(c, [len(s) for s in b])
                results[(k, rep)] = (c, d)
            if k % 4 == 0:
                results[("pack", k)] = m.unpack(m.pack(blob, chunk_len=1024))
        except Exception as e:            # re-raised on the main thread below
            errors.append(e)

    threads = [threading.Thread(target=work, args=(k,)) for k in range(8)]
    for t in threads:
        t.start()
    for t in threads:
        t.join()
    assert not errors, errors
    for key, val in results.items():
        if key[0] == "pack":
            assert val == blob
            continue
        k = key[0]
        c, d = val
        assert c == serial[k % 4]
        assert d == batches[k % 4]
    assert m.pack(blob, chunk_len=1024) == serial_pack
    m.close()
