"""Products with operands in host memory (the host layer: Strassen levels
expanded and aggregated on the host, or C in blocks), against the CPU oracle.

The plan checks need no GPU (an explicit device budget); the products run on
the GPU and are compared bit for bit with the oracle's cubic product."""
import numpy as np
import pytest

import oracle as O
from gpu_util import gen

import paper_1909_01554_gb300 as bmm

MiB = 1 << 20


def built():
    import os

    if not os.path.exists(bmm.LIB_PATH):
        from paper_1909_01554_gb300 import build

        build.build()


# ------------------------------------------------------------ plans (no GPU)
def test_plan_whole_product_when_it_fits():
    built()
    p = bmm.host_plan(bmm.GF2, 2048, 2048, 2048, device_bytes=1 << 34)
    assert (p["host_depth"], p["count"]) == (0, 1)
    assert (p["sub_m"], p["sub_k"], p["sub_n"]) == (2048, 2048, 2048)
    assert p["upload_bytes"] == 2 * 2048 * 2048 // 8 and p["download_bytes"] == 2048 * 2048 // 8
    assert p["staging_bytes"] == 0


def test_plan_host_levels_halve_every_side():
    built()
    m, k, n = 4096, 2048, 3072
    for d in (1, 2, 3):
        p = bmm.host_plan(bmm.GF2, m, k, n, device_bytes=1 << 34, host_depth=d)
        assert p["host_depth"] == d and p["count"] == 7 ** d
        assert (p["sub_m"], p["sub_k"], p["sub_n"]) == (m >> d, k >> d, n >> d)
        t, s, q = (m >> d) * (k >> d) // 8, (k >> d) * (n >> d) // 8, (m >> d) * (n >> d) // 8
        assert p["upload_bytes"] == 7 ** d * (t + s)
        assert p["download_bytes"] == 7 ** d * q
        assert p["staging_bytes"] == 2 * (t + s + q)


def test_plan_auto_takes_the_fewest_levels_that_fit():
    built()
    m = k = n = 8192
    whole = bmm.host_plan(bmm.GF2, m, k, n, device_bytes=1 << 34)["device_bytes"]
    one = bmm.host_plan(bmm.GF2, m, k, n, device_bytes=1 << 34, host_depth=1)["device_bytes"]
    two = bmm.host_plan(bmm.GF2, m, k, n, device_bytes=1 << 34, host_depth=2)["device_bytes"]
    assert whole > one > two
    assert bmm.host_plan(bmm.GF2, m, k, n, device_bytes=whole)["host_depth"] == 0
    assert bmm.host_plan(bmm.GF2, m, k, n, device_bytes=whole - 1)["host_depth"] == 1
    assert bmm.host_plan(bmm.GF2, m, k, n, device_bytes=one - 1)["host_depth"] == 2
    assert bmm.host_plan(bmm.GF2, m, k, n, device_bytes=two)["host_depth"] == 2


def test_plan_device_bytes_follow_the_device_plan():
    """The device estimate is the sub-instance buffers plus the scratch of
    the device product's own plan, whatever its options: with the innermost
    level inside the CUDA-core kernel it is the scratch of one level fewer."""
    built()
    m = k = n = 16384
    for d in (1, 2, 3):
        for kl in (0, 1):
            kw = dict(path=bmm.PATH_POPC, depth=d, kernel_level=kl)
            hp = bmm.host_plan(bmm.GF2, m, k, n, device_bytes=1 << 36, host_depth=1, **kw)
            sm, sk, sn = hp["sub_m"], hp["sub_k"], hp["sub_n"]
            dev = bmm.plan(bmm.GF2, sm, sk, sn, serial=max(0, d - kl - 2), **kw)
            bufs = 2 * (sm * sk + sk * sn + sm * sn) // 8
            assert hp["device_bytes"] == bufs + dev["workspace_bytes"] + (8 << 20)
            if not bmm.device_supported():
                # AUTO resolves to the CUDA cores here: the same estimate
                auto = dict(kw, path=bmm.PATH_AUTO)
                ha = bmm.host_plan(bmm.GF2, m, k, n, device_bytes=1 << 36, host_depth=1, **auto)
                assert ha["device_bytes"] == hp["device_bytes"]


def test_plan_boolean_blocks_c_and_rereads_b_per_block_row():
    built()
    m, k, n = 8192, 4096, 8192
    whole = bmm.host_plan(bmm.BOOL, m, k, n, device_bytes=1 << 34)["device_bytes"]
    p = bmm.host_plan(bmm.BOOL, m, k, n, device_bytes=whole // 3)
    assert p["host_depth"] == 0 and p["count"] > 1 and p["device_bytes"] <= whole // 3
    rows = -(-m // p["sub_m"])
    cols = -(-n // p["sub_n"])
    assert p["count"] == rows * cols and p["sub_k"] == k
    assert p["upload_bytes"] == m * k // 8 + rows * k * n // 8
    assert p["download_bytes"] == m * n // 8


def test_plan_errors():
    built()
    with pytest.raises(bmm.BmmError) as e:  # no additive inverse
        bmm.host_plan(bmm.BOOL, 4096, 4096, 4096, device_bytes=1 << 34, host_depth=1)
    assert e.value.status == bmm.ERR_INVALID
    with pytest.raises(bmm.BmmError) as e:  # 64 * 2^2 does not divide 320
        bmm.host_plan(bmm.GF2, 320, 4096, 4096, device_bytes=1 << 34, host_depth=2)
    assert e.value.status == bmm.ERR_UNSUPPORTED
    with pytest.raises(bmm.BmmError) as e:  # nothing fits 1 KiB
        bmm.host_plan(bmm.BOOL, 4096, 4096, 4096, device_bytes=1024)
    assert e.value.status == bmm.ERR_NOMEM
    with pytest.raises(bmm.BmmError) as e:
        bmm.host_plan(bmm.GF2, 100, 64, 64, device_bytes=1 << 34)
    assert e.value.status == bmm.ERR_INVALID


# ------------------------------------------------------------ products (GPU)
torch = pytest.importorskip("torch")
OPS = {bmm.GF2: O.GF2, bmm.BOOL: O.BOOL}


def host_product(op, Ah, Bh, m, k, n, pinned=False, **kw):
    C = np.full((m, n // 64), np.uint64(0x5A5A5A5A5A5A5A5A))
    if pinned:
        tA = torch.from_numpy(Ah.view(np.int64).ravel().copy()).pin_memory()
        tB = torch.from_numpy(Bh.view(np.int64).ravel().copy()).pin_memory()
        tC = torch.from_numpy(C.view(np.int64).ravel().copy()).pin_memory()
        bmm.product_host(op, tA, tB, tC, m, k, n, **kw)
        return tC.numpy().view(np.uint64).reshape(m, n // 64)
    bmm.product_host(op, np.ascontiguousarray(Ah), np.ascontiguousarray(Bh), C, m, k, n, **kw)
    return C


def gpu_ok():
    return torch.cuda.is_available()


@pytest.mark.gpu
@pytest.mark.parametrize("variant", [bmm.SELF_INVERSE, bmm.CHAINING, bmm.WINOGRAD])
@pytest.mark.parametrize("host_depth", [1, 2])
def test_gf2_host_levels_match_oracle(variant, host_depth):
    if not gpu_ok():
        pytest.skip("no GPU")
    m, k, n = 1024, 1536, 768
    Ah, Bh = gen(m, k, 61, 0), gen(k, n, 61, 1)
    got = host_product(bmm.GF2, Ah, Bh, m, k, n, pinned=True, host_depth=host_depth,
                       variant=variant, device_bytes=1 << 30)
    assert (got == O.cubic(O.GF2, Ah, Bh, m, k, n)).all()


@pytest.mark.gpu
@pytest.mark.parametrize("op", [bmm.GF2, bmm.BOOL])
@pytest.mark.parametrize("pinned", [True, False])
def test_blocked_with_ragged_blocks_matches_oracle(op, pinned):
    """A budget that forces blocks of C whose last row and column are short."""
    if not gpu_ok():
        pytest.skip("no GPU")
    m, k, n = 1344, 640, 1472
    p = None if op == bmm.GF2 else "1/16"
    Ah, Bh = gen(m, k, 67, 0, p), gen(k, n, 67, 1, p)
    whole = bmm.host_plan(op, m, k, n, device_bytes=1 << 34, host_depth=0)["device_bytes"]
    budget = whole
    while True:
        budget = budget * 9 // 10
        plan = bmm.host_plan(op, m, k, n, device_bytes=budget, host_depth=0)
        if plan["count"] >= 4:
            break
    assert m % plan["sub_m"] or n % plan["sub_n"], plan  # a ragged edge is exercised
    got = host_product(op, Ah, Bh, m, k, n, pinned=pinned, host_depth=0, device_bytes=budget)
    assert (got == O.cubic(OPS[op], Ah, Bh, m, k, n)).all(), plan


@pytest.mark.gpu
@pytest.mark.parametrize("op", [bmm.GF2, bmm.BOOL])
def test_whole_product_and_auto_plan_match_oracle(op):
    if not gpu_ok():
        pytest.skip("no GPU")
    m, k, n = 512, 2048, 1024
    p = None if op == bmm.GF2 else "1/32"
    Ah, Bh = gen(m, k, 71, 0, p), gen(k, n, 71, 1, p)
    want = O.cubic(OPS[op], Ah, Bh, m, k, n)
    assert (host_product(op, Ah, Bh, m, k, n) == want).all()
    assert (host_product(op, Ah, Bh, m, k, n, pinned=True, path=bmm.PATH_POPC) == want).all()


@pytest.mark.gpu
def test_gf2_host_levels_over_device_strassen():
    """Host levels above device Strassen levels: 2 on the host, 2 on the GPU."""
    if not gpu_ok():
        pytest.skip("no GPU")
    n = 4096
    Ah, Bh = gen(n, n, 73, 0), gen(n, n, 73, 1)
    got = host_product(bmm.GF2, Ah, Bh, n, n, n, pinned=True, host_depth=2, depth=2,
                       device_bytes=1 << 30)
    assert (got == O.cubic(O.GF2, Ah, Bh, n, n, n)).all()


@pytest.mark.gpu
def test_cached_buffers_across_calls_and_release():
    """Consecutive host-memory products reuse (and grow) the kept buffers:
    small, large, small again, then after a release; every result exact."""
    if not gpu_ok():
        pytest.skip("no GPU")
    cases = [(512, 1024, 512, 1), (1024, 2048, 1536, 1), (512, 1024, 512, 1), (768, 640, 960, 0)]
    for i, (m, k, n, hd) in enumerate(cases):
        if i == 3:
            bmm.host_release()
        op = bmm.GF2
        Ah, Bh = gen(m, k, 79 + i, 0), gen(k, n, 79 + i, 1)
        got = host_product(op, Ah, Bh, m, k, n, pinned=True, host_depth=hd, device_bytes=1 << 30)
        assert (got == O.cubic(O.GF2, Ah, Bh, m, k, n)).all(), (m, k, n, hd)
    bmm.host_release()


@pytest.mark.gpu
@pytest.mark.parametrize("path", [bmm.PATH_POPC, bmm.PATH_TC_FP4_PAIR])
def test_gf2_host_level_over_in_kernel_level(path):
    """A host level above device products whose innermost Strassen level runs
    inside the base-case kernel, on both paths that have that form; the
    device estimate follows the padded k of the tensor form."""
    if not gpu_ok():
        pytest.skip("no GPU")
    if path == bmm.PATH_TC_FP4_PAIR and not bmm.device_supported():
        pytest.skip("tensor-core paths need sm_103")
    m, k, n = 2048, 2048, 1536
    kw = dict(path=path, depth=2, kernel_level=1, device_bytes=1 << 30)
    hp = bmm.host_plan(bmm.GF2, m, k, n, host_depth=1, **kw)
    dev = bmm.plan(bmm.GF2, hp["sub_m"], hp["sub_k"], hp["sub_n"], path=path, depth=2,
                   kernel_level=1)
    assert dev["kernel_level"] == 1
    bufs = 2 * (hp["sub_m"] * hp["sub_k"] + hp["sub_k"] * hp["sub_n"] + hp["sub_m"] * hp["sub_n"]) // 8
    assert hp["device_bytes"] == bufs + dev["workspace_bytes"] + (8 << 20)
    Ah, Bh = gen(m, k, 83, 0), gen(k, n, 83, 1)
    got = host_product(bmm.GF2, Ah, Bh, m, k, n, pinned=True, host_depth=1, **kw)
    assert (got == O.cubic(O.GF2, Ah, Bh, m, k, n)).all()
