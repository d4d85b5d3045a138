"""The allocation-free product (bmm_product_noalloc) against the CPU oracle
and against bmm_gf2 / bmm_bool.

It serves callers that cannot allocate device memory while they run; its
only scratch is a fixed device array shared by every call. Two calls in a row
with different inputs must each match the oracle's product and the
allocating entry point's bit for bit (so nothing left in the array from the
first call leaks into the second), and sizes beyond the array are refused.
This file is named to be collected last, and passes both alone in a fresh
process and after the other tests."""
import ctypes

import pytest

import oracle as O
from gpu_util import first_mismatch, from_dev, gen, to_dev

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover - CPU machine
    pytest.skip("no GPU", allow_module_level=True)

import paper_1909_01554_gb300 as bmm  # noqa: E402


def noalloc(op, dA, dB, dC, m, k, n):
    L = bmm.lib()
    stream = torch.cuda.current_stream().cuda_stream
    return L.bmm_product_noalloc(op, dA.data_ptr(), dB.data_ptr(), dC.data_ptr(), m, k, n,
                                 ctypes.c_void_p(stream))


@pytest.mark.parametrize("op", [bmm.GF2, bmm.BOOL])
def test_noalloc_matches_oracle_and_allocating_entry_point_twice(op):
    shapes = [(1024, 2048, 1536, 31), (448, 1344, 960, 32)]  # second call: ragged, smaller
    for m, k, n, seed in shapes:
        p = None if op == bmm.GF2 else "1/32"
        Ah, Bh = gen(m, k, seed, 0, p), gen(k, n, seed, 1, p)
        want = O.cubic(O.GF2 if op == bmm.GF2 else O.BOOL, Ah, Bh, m, k, n)
        dA, dB = to_dev(Ah), to_dev(Bh)
        ref, got = bmm.empty(m, n), bmm.empty(m, n)
        got.fill_(-1)
        bmm.product(op, dA, dB, ref, m, k, n)
        assert noalloc(op, dA, dB, got, m, k, n) == bmm.OK
        bmm.stream_status()
        mm = first_mismatch(from_dev(got, m, n), want)
        assert mm is None, f"op={op} shape={(m, k, n)} against the oracle: {mm}"
        mm = first_mismatch(from_dev(got, m, n), from_dev(ref, m, n))
        assert mm is None, f"op={op} shape={(m, k, n)} against bmm_gf2/bmm_bool: {mm}"


def test_noalloc_refuses_sizes_beyond_its_scratch():
    limit_bits = 8 * (8 << 20)
    k, n = 8192, limit_bits // 8192 + 64  # k*n just over the array
    d = bmm.empty(64, 64)
    dA = bmm.empty(64, k)
    dB = bmm.empty(k, n)
    dC = bmm.empty(64, n)
    assert noalloc(bmm.GF2, dA, dB, dC, 64, k, n) == bmm.ERR_NOMEM
    assert noalloc(bmm.GF2, d, d, d, 100, 64, 64) == bmm.ERR_INVALID
    assert noalloc(bmm.BOOL, d, d, d, 64, 64, 64) == bmm.ERR_INVALID  # C overlaps A and B
