"""The unit microbenchmarks behind the rooflines (boa_microbench) run and
report rates in a physically possible range for one GPU."""
import ctypes as C

import pytest

from paper_2511_11337_b300._lib import check, load

pytestmark = pytest.mark.gpu

EX2, FFMA, FFMA2, L2, MMA = 0, 1, 2, 3, 4


def _mb(test, kind=0, M=128, N=128, flags=0):
    rate, aux = C.c_double(), C.c_double()
    check(load().boa_microbench(0, test, kind, M, N, flags, C.byref(rate), C.byref(aux)))
    return rate.value, aux.value


def test_unit_rates():
    ex2, _ = _mb(EX2)
    ffma, _ = _mb(FFMA)
    l2, _ = _mb(L2)
    assert 1e12 < ex2 < 1e14
    assert 1e13 < ffma < 3e14
    assert 1e12 < l2 < 1e14


def test_mma_rates_and_cycles():
    tf32, c_tf32 = _mb(MMA, kind=0, N=256)
    bf16, c_bf16 = _mb(MMA, kind=1, N=256)
    fp8, _ = _mb(MMA, kind=2, N=256)
    assert 1e14 < tf32 < 5e15 and 1e14 < bf16 < 5e15 and 1e14 < fp8 < 1e16
    assert bf16 > tf32 and fp8 > bf16
    assert 16 < c_tf32 < 4096 and 16 < c_bf16 < 4096
    ta, _ = _mb(MMA, kind=0, N=64, flags=1)
    assert ta > 0
    with pytest.raises(Exception):
        _mb(MMA, kind=1, N=64, flags=1)          # A from TMEM is offered for TF32 only
