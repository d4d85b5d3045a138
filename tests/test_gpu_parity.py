"""GPU path against the CPU oracle, bit for bit, through the C ABI.

Sizes span several tiles with ragged tails (multiples of 64 that are not
multiples of the 128/256 tile sizes), degenerate inputs (zero, identity,
all ones), every base-case path, every Strassen variant and depth split."""
import numpy as np
import pytest

import oracle as O
from gpu_util import first_mismatch, from_dev, gen, to_dev

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover - CPU machine
    pytest.skip("no GPU", allow_module_level=True)

import paper_1909_01554_gb300 as bmm  # noqa: E402

OPS = {bmm.GF2: O.GF2, bmm.BOOL: O.BOOL}


def paths():
    ps = [bmm.PATH_POPC]
    if bmm.device_supported():
        ps += list(bmm.TENSOR_PATHS)
    return ps


def run(op, Ah, Bh, m, k, n, **kw):
    dA, dB = to_dev(Ah), to_dev(Bh)
    dC = bmm.empty(m, n)
    dC.fill_(-1)
    bmm.product(op, dA, dB, dC, m, k, n, **kw)
    bmm.stream_status()
    return from_dev(dC, m, n)


def check(got, want, what):
    mm = first_mismatch(got, want)
    assert mm is None, f"{what}: first mismatch (row, word, got, want, count) = {mm}"


# ------------------------------------------------------------ transpose
# The last three shapes take the TMA form (both pitches even, at least one
# 512 x 512 tile), with tiles ragged in both directions; the first five the
# load/store form (odd pitches or less than a tile a side).
@pytest.mark.parametrize("rows,cols", [(64, 64), (256, 512), (320, 192), (4096, 128), (64, 1344),
                                       (512, 512), (1664, 640), (1152, 2048)])
def test_transpose(rows, cols):
    X = gen(rows, cols, 3, 0)
    dX = to_dev(X)
    dT = bmm.empty(cols, rows)
    bmm.transpose(dX, dT, rows, cols)
    bmm.stream_status()
    check(from_dev(dT, cols, rows), O.transpose(X, rows, cols), "transpose")


# ------------------------------------------------------------ base case
@pytest.mark.parametrize("path", paths())
@pytest.mark.parametrize("op", [bmm.GF2, bmm.BOOL])
@pytest.mark.parametrize("m,k,n", [(64, 64, 64), (128, 256, 256), (192, 320, 448),
                                   (384, 1152, 320), (1024, 2048, 1024)])
def test_base_product(path, op, m, k, n):
    if path != bmm.PATH_POPC and k % 128:
        pytest.skip("tensor paths need k % 128 == 0 (TMA row pitch)")
    p = None if op == bmm.GF2 else "1/16"
    Ah, Bh = gen(m, k, 5, 0, p), gen(k, n, 5, 1, p)
    Bt = O.transpose(Bh, k, n)
    dC = bmm.empty(m, n)
    dC.fill_(-1)
    bmm.base_product(op, path, to_dev(Ah), to_dev(Bt), dC, m, k, n)
    bmm.stream_status()
    check(from_dev(dC, m, n), O.cubic(OPS[op], Ah, Bh, m, k, n), f"base op={op} path={path}")


@pytest.mark.parametrize("path", paths())
def test_base_product_counts_cover_every_parity(path):
    """Row i of A has its first c_i bits set and B is all ones: entry (i, j) of the
    integer product is c_i for every j, so c_i = 0..k exercises every count."""
    m, k, n = 256, 1024, 256
    c = np.array([(37 * i) % (k + 1) for i in range(m)])
    Ab = (np.arange(k)[None, :] < c[:, None]).astype(np.uint8)
    Ah = O.pack(Ab)
    Bt = O.pack(np.ones((n, k), dtype=np.uint8))
    for op in (bmm.GF2, bmm.BOOL):
        dC = bmm.empty(m, n)
        bmm.base_product(op, path, to_dev(Ah), to_dev(Bt), dC, m, k, n)
        bmm.stream_status()
        want = O.cubic(OPS[op], Ah, O.transpose(Bt, n, k), m, k, n)
        check(from_dev(dC, m, n), want, f"counts op={op} path={path}")


@pytest.mark.parametrize("path", paths())
def test_base_product_all_ones_large_k(path):
    """All-ones operands: every count equals k (the largest count a run reaches)."""
    m, n = 128, 256
    for k in (8192, 65536 + 128):
        if path != bmm.PATH_POPC and k % 128:
            continue
        Ah = np.full((m, k // 64), np.uint64(0xFFFFFFFFFFFFFFFF))
        Bt = np.full((n, k // 64), np.uint64(0xFFFFFFFFFFFFFFFF))
        for op in (bmm.GF2, bmm.BOOL):
            dC = bmm.empty(m, n)
            bmm.base_product(op, path, to_dev(Ah), to_dev(Bt), dC, m, k, n)
            bmm.stream_status()
            want = (k % 2) if op == bmm.GF2 else 1
            got = O.unpack(from_dev(dC, m, n), m, n)
            assert (got == want).all(), f"k={k} op={op} path={path}"


def prefix_rows(counts, k):
    """Packed rows whose row r has exactly its first counts[r] bits set."""
    kw = k // 64
    c = torch.tensor(counts, dtype=torch.int64, device="cuda")[:, None]
    idx = torch.arange(kw, dtype=torch.int64, device="cuda")[None, :]
    rem = c % 64
    part = torch.bitwise_left_shift(torch.ones_like(rem), rem) - 1  # rem = 0 gives 0
    out = torch.where(idx < c // 64, torch.full_like(idx, -1),
                      torch.where(idx == c // 64, part, torch.zeros_like(idx)))
    return out.reshape(-1).contiguous()


@pytest.mark.parametrize("path", paths())
def test_base_product_exact_counts_past_2pow23(path):
    """Prefix rows: entry (i, j) of the integer product is min(c_i, d_j), a closed
    form. k = 2^23 + 2^21 bits takes the counts past 2^23, where the tensor
    paths must flush their FP32 accumulator (they read parity off
    count * 2^-12, exact below 2^23: every 65534 stages of 128 k for e4m3,
    32766 of 256 k for e2m1), and puts every parity next to 2^22, 2^23, both
    flush points and k."""
    m, n, k = 128, 256, (1 << 23) + (1 << 21)
    rng = np.random.default_rng(31)
    edge = [0, 1, 2, 63, 64, 65, (1 << 22) - 1, 1 << 22, (1 << 22) + 1,
            65534 * 128 - 1, 65534 * 128, 65534 * 128 + 1, 32766 * 256 - 1, 32766 * 256,
            32766 * 256 + 1, (1 << 23) - 1, 1 << 23,
            (1 << 23) + 1, k - 1, k]
    c = edge + rng.integers(0, k + 1, m - len(edge)).tolist()
    d = [k] * (n // 2) + edge + rng.integers(0, k + 1, n // 2 - len(edge)).tolist()
    A, Bt = prefix_rows(c, k), prefix_rows(d, k)
    cnt = np.minimum(np.array(c)[:, None], np.array(d)[None, :])
    for op in (bmm.GF2, bmm.BOOL):
        dC = bmm.empty(m, n)
        dC.fill_(-1)
        bmm.base_product(op, path, A, Bt, dC, m, k, n)
        bmm.stream_status()
        want = O.pack(((cnt & 1) if op == bmm.GF2 else (cnt > 0)).astype(np.uint8))
        check(from_dev(dC, m, n), want, f"large-count op={op} path={path}")


# ------------------------------------------------------------ full products
@pytest.mark.parametrize("op", [bmm.GF2, bmm.BOOL])
@pytest.mark.parametrize("m,k,n", [(64, 128, 64), (448, 320, 576), (1024, 1024, 1024)])
def test_cubic_product(op, m, k, n):
    p = None if op == bmm.GF2 else "1/32"
    Ah, Bh = gen(m, k, 7, 0, p), gen(k, n, 7, 1, p)
    for path in paths():  # the product calls pad k for the tensor paths
        got = run(op, Ah, Bh, m, k, n, path=path, depth=0)
        check(got, O.cubic(OPS[op], Ah, Bh, m, k, n), f"cubic op={op} path={path}")


@pytest.mark.parametrize("m,k,n,depth", [(512, 320, 448, 0), (256, 64, 192, 0),
                                         (1024, 384, 768, 1), (1024, 768, 512, 2)])
def test_tensor_paths_pad_k(m, k, n, depth):
    """k that is not a multiple of 128 bits per leaf: the tensor paths run on
    a copy of A and a B^T padded with zero columns, which leaves the product
    unchanged."""
    if not bmm.device_supported():
        pytest.skip("tensor-core paths need sm_103")
    for op in (bmm.GF2, bmm.BOOL):
        if op == bmm.BOOL and depth:
            continue
        p = None if op == bmm.GF2 else "1/16"
        Ah, Bh = gen(m, k, 37, 0, p), gen(k, n, 37, 1, p)
        want = O.cubic(OPS[op], Ah, Bh, m, k, n)
        for path in bmm.TENSOR_PATHS:
            info = bmm.plan(op, m, k, n, path=path, depth=depth)
            assert info["path"] == path
            check(run(op, Ah, Bh, m, k, n, path=path, depth=depth), want,
                  f"padded k op={op} path={path} depth={depth}")
        if depth == 0:  # the automatic choice takes a tensor path too
            assert bmm.plan(op, m, k, n)["path"] in bmm.TENSOR_PATHS
            check(run(op, Ah, Bh, m, k, n), want, f"padded k auto op={op}")


def test_identity_and_zero():
    n = 512
    I = O.pack(np.eye(n, dtype=np.uint8))
    A = gen(n, n, 9, 0)
    Z = np.zeros_like(A)
    for op in (bmm.GF2, bmm.BOOL):
        check(run(op, A, I, n, n, n), A, "A I")
        check(run(op, I, A, n, n, n), A, "I A")
        check(run(op, A, Z, n, n, n), Z, "A 0")


def test_config1_4096_full_compare():
    """m = k = n = 4096: GF(2) with p = 1/2, Boolean with p = 1/64, seed 1."""
    n = 4096
    A, B = gen(n, n, 1, 0), gen(n, n, 1, 1)
    Ab, Bb = gen(n, n, 1, 0, "1/64"), gen(n, n, 1, 1, "1/64")
    want_g = O.cubic(O.GF2, A, B, n, n, n)
    want_b = O.cubic(O.BOOL, Ab, Bb, n, n, n)
    for path in paths():
        check(run(bmm.GF2, A, B, n, n, n, path=path, depth=0), want_g, f"gf2 path={path}")
        check(run(bmm.BOOL, Ab, Bb, n, n, n, path=path), want_b, f"bool path={path}")
    density = O.unpack(want_b, n, n).mean()
    assert abs(density - (1 - np.exp(-1))) < 0.01


# ------------------------------------------------------------ Strassen
@pytest.mark.parametrize("variant", [bmm.WINOGRAD, bmm.SELF_INVERSE, bmm.CHAINING])
@pytest.mark.parametrize("depth,serial", [(1, 0), (2, 0), (1, 1), (2, 1), (3, 1), (3, 2)])
def test_strassen_variants(variant, depth, serial):
    m, k, n = 1024, 2048, 1536
    if depth == 3:
        m, k, n = 2048, 2048, 1024
    Ah, Bh = gen(m, k, 13, 0), gen(k, n, 13, 1)
    want = O.cubic(O.GF2, Ah, Bh, m, k, n)
    got = run(bmm.GF2, Ah, Bh, m, k, n, depth=depth, serial=serial, variant=variant,
              path=bmm.PATH_POPC)
    check(got, want, f"strassen v={variant} d={depth} s={serial}")


# The Strassen passes over the tensor-core base cases. Shapes (mq, kq, nq) <<
# depth give leaves of mq x kq x nq bits: 320 and 384 leaf rows are not
# multiples of the 256-row SM-pair tile, and kq = 192 is not a multiple of the
# 128 bits a tensor leaf needs, so the plan pads k (zero columns of A, zero
# rows of B) below every level.
@pytest.mark.parametrize("path,shape", [(bmm.PATH_TC_FP4_PAIR, (320, 192, 448)),
                                        (bmm.PATH_TC_FP4_PAIR, (384, 256, 320)),
                                        (bmm.PATH_TC_FP8_PAIR, (320, 192, 448))])
@pytest.mark.parametrize("variant", [bmm.WINOGRAD, bmm.SELF_INVERSE, bmm.CHAINING])
@pytest.mark.parametrize("depth,serial", [(1, 0), (2, 0), (1, 1), (2, 1), (3, 1), (3, 2)])
def test_strassen_variants_tensor(path, shape, variant, depth, serial):
    if not bmm.device_supported():
        pytest.skip("tensor-core paths need sm_103")
    m, k, n = (x << depth for x in shape)
    info = bmm.plan(bmm.GF2, m, k, n, depth=depth, serial=serial, variant=variant, path=path)
    assert info["path"] == path and info["serial_depth"] == serial
    Ah, Bh = gen(m, k, 41, 0), gen(k, n, 41, 1)
    want = O.cubic(O.GF2, Ah, Bh, m, k, n)
    got = run(bmm.GF2, Ah, Bh, m, k, n, depth=depth, serial=serial, variant=variant, path=path)
    check(got, want, f"strassen path={path} {shape} v={variant} d={depth} s={serial}")


# The innermost level inside the CUDA-core kernel. m, k, n = (320, kq, 448)
# << depth: the in-kernel quadrants are 2.5 x 3.5 tiles of 128 rows and
# kq = 576 bits (9 words of k: two full stages of 4 and a ragged one; 8-byte
# copies) or kq = 512 bits (8 words; every pitch and stride the launcher sees
# is then a multiple of 8 words too, so it takes the 16-byte copy form, here
# on the same ragged row tiles).
@pytest.mark.parametrize("kq", [576, 512])
@pytest.mark.parametrize("variant", [bmm.WINOGRAD, bmm.SELF_INVERSE, bmm.CHAINING])
@pytest.mark.parametrize("depth,serial", [(1, 0), (2, 0), (2, 1), (3, 1), (3, 2)])
def test_kernel_level(variant, depth, serial, kq):
    m, k, n = 320 << depth, kq << depth, 448 << depth
    Ah, Bh = gen(m, k, 29, 0), gen(k, n, 29, 1)
    want = O.cubic(O.GF2, Ah, Bh, m, k, n)
    info = bmm.plan(bmm.GF2, m, k, n, depth=depth, serial=serial, variant=variant,
                    path=bmm.PATH_POPC, kernel_level=1)
    assert info["kernel_level"] == 1 and info["serial_depth"] == serial
    got = run(bmm.GF2, Ah, Bh, m, k, n, depth=depth, serial=serial, variant=variant,
              path=bmm.PATH_POPC, kernel_level=1)
    check(got, want, f"kernel level v={variant} d={depth} s={serial}")


@pytest.mark.parametrize("m,k,n", [(384, 2688, 640), (256, 4096, 256)])
def test_kernel_level_long_k(m, k, n):
    """Quadrants of 21 and 32 words of k: the staging ring wraps several times."""
    Ah, Bh = gen(m, k, 37, 0), gen(k, n, 37, 1)
    want = O.cubic(O.GF2, Ah, Bh, m, k, n)
    got = run(bmm.GF2, Ah, Bh, m, k, n, depth=1, path=bmm.PATH_POPC, kernel_level=1)
    check(got, want, f"kernel level {m}x{k}x{n}")


def test_kernel_level_degenerate_and_unsupported():
    """All-ones operands (every product's operand combination is all ones or
    zero), the identity, and the tensor paths' refusal."""
    m = k = n = 1024
    ones = np.full((m, k // 64), np.uint64(0xFFFFFFFFFFFFFFFF), dtype=np.uint64)
    want = O.cubic(O.GF2, ones, ones, m, k, n)
    got = run(bmm.GF2, ones, ones, m, k, n, depth=2, path=bmm.PATH_POPC, kernel_level=1)
    check(got, want, "kernel level, all ones")
    eye = O.pack(np.eye(n, dtype=np.uint8))
    A = gen(m, k, 31, 0)
    check(run(bmm.GF2, A, eye, m, k, n, depth=1, path=bmm.PATH_POPC, kernel_level=1), A,
          "kernel level, A I")
    if bmm.device_supported():
        for path in (bmm.PATH_TC_FP8, bmm.PATH_TC_FP8_PAIR):
            with pytest.raises(bmm.BmmError):
                run(bmm.GF2, ones, ones, m, k, n, depth=2, path=path, kernel_level=1)
        got = run(bmm.GF2, ones, ones, m, k, n, depth=2, path=bmm.PATH_TC_FP4_PAIR,
                  kernel_level=1)
        check(got, want, "tensor kernel level, all ones")
        check(run(bmm.GF2, A, eye, m, k, n, depth=1, path=bmm.PATH_TC_FP4_PAIR,
                  kernel_level=1), A, "tensor kernel level, A I")


# The innermost level inside the e2m1 tensor kernel: quadrants of (320, kq,
# 448) bits, ragged in the 256-row and 256-column tiles; kq = 576 is padded to
# 1024 (two 512-bit packed stages, the second partly zero), kq = 1024 needs
# no padding; the depth-first and breadth-first splits above it as for the
# CUDA-core form.
@pytest.mark.parametrize("kq", [576, 1024])
@pytest.mark.parametrize("variant", [bmm.WINOGRAD, bmm.SELF_INVERSE, bmm.CHAINING])
@pytest.mark.parametrize("depth,serial", [(1, 0), (2, 0), (2, 1), (3, 1), (3, 2)])
def test_kernel_level_tensor(variant, depth, serial, kq):
    if not bmm.device_supported():
        pytest.skip("tensor-core paths need sm_103")
    m, k, n = 320 << depth, kq << depth, 448 << depth
    Ah, Bh = gen(m, k, 61, 0), gen(k, n, 61, 1)
    want = O.cubic(O.GF2, Ah, Bh, m, k, n)
    info = bmm.plan(bmm.GF2, m, k, n, depth=depth, serial=serial, variant=variant,
                    path=bmm.PATH_TC_FP4_PAIR, kernel_level=1)
    assert info["kernel_level"] == 1 and info["serial_depth"] == serial
    got = run(bmm.GF2, Ah, Bh, m, k, n, depth=depth, serial=serial, variant=variant,
              path=bmm.PATH_TC_FP4_PAIR, kernel_level=1)
    check(got, want, f"tensor kernel level v={variant} d={depth} s={serial} kq={kq}")


def test_kernel_level_tensor_long_k():
    """Quadrants of 4096 bits of k (eight packed stages per product)."""
    m, k, n = 512, 8192, 768
    if not bmm.device_supported():
        pytest.skip("tensor-core paths need sm_103")
    Ah, Bh = gen(m, k, 67, 0), gen(k, n, 67, 1)
    want = O.cubic(O.GF2, Ah, Bh, m, k, n)
    got = run(bmm.GF2, Ah, Bh, m, k, n, depth=1, path=bmm.PATH_TC_FP4_PAIR, kernel_level=1)
    check(got, want, "tensor kernel level, long k")


@pytest.mark.parametrize("path", paths())
def test_strassen_over_each_base_case(path):
    n = 2048
    Ah, Bh = gen(n, n, 17, 0), gen(n, n, 17, 1)
    want = O.cubic(O.GF2, Ah, Bh, n, n, n)
    check(run(bmm.GF2, Ah, Bh, n, n, n, depth=2, path=path), want, f"strassen path={path}")


@pytest.mark.parametrize("variant", [bmm.SELF_INVERSE, bmm.CHAINING])
@pytest.mark.parametrize("inverse", [False, True])
def test_basis_change_matches_oracle(variant, inverse):
    rows, cols, d = 1024, 2048, 3
    X = gen(rows, cols, 19, 0)
    dX = to_dev(X)
    bmm.basis_change(variant, inverse, dX, rows, cols, d)
    bmm.stream_status()
    want, _ = O.basis_change(variant, inverse, X, rows, cols, d)
    check(from_dev(dX, rows, cols), want, "basis change")


def test_errors_are_reported():
    dA = bmm.empty(128, 128)
    dC = bmm.empty(128, 128)
    with pytest.raises(bmm.BmmError) as e:
        bmm.boolean(dA, dA, dC, 128, 128, 128, depth=1)
    assert e.value.status == bmm.ERR_INVALID
    with pytest.raises(bmm.BmmError) as e:
        bmm.gf2(dA, dA, dC, 128, 128, 128, depth=3)
    assert e.value.status == bmm.ERR_UNSUPPORTED
    with pytest.raises(bmm.BmmError) as e:
        bmm.gf2(dA.data_ptr() + 8, dA, dC, 64, 64, 64)
    assert e.value.status == bmm.ERR_ALIGN
    with pytest.raises(bmm.BmmError) as e:
        bmm.gf2(dA, dA, dA, 128, 128, 128)
    assert e.value.status == bmm.ERR_INVALID


def test_bounded_wait_times_out_and_context_survives():
    """A device-side wait that nothing satisfies gives up after its limit; the
    host reads BMM_ERR_TIMEOUT and the context keeps working."""
    stream = torch.cuda.current_stream().cuda_stream
    assert bmm.lib().bmm_selftest_wait_timeout(20_000_000, stream) == bmm.OK  # 20 ms
    with pytest.raises(bmm.BmmError) as e:
        bmm.stream_status()
    assert e.value.status == bmm.ERR_TIMEOUT
    bmm.stream_status()  # cleared
    n = 256
    A, B = gen(n, n, 29, 0), gen(n, n, 29, 1)
    check(run(bmm.GF2, A, B, n, n, n), O.cubic(O.GF2, A, B, n, n, n), "after timeout")


def test_int8_tensor_path_is_unsupported_on_sm103():
    """sm_103a has no 8-bit integer tensor-core MMA: the path reports UNSUPPORTED."""
    d = bmm.empty(128, 128)
    c = bmm.empty(128, 128)
    with pytest.raises(bmm.BmmError) as e:
        bmm.base_product(bmm.GF2, bmm.PATH_TC_I8, d, d, c, 128, 128, 128)
    assert e.value.status == bmm.ERR_UNSUPPORTED


def test_device_generator_matches_cpu_generator():
    import bitgen

    for p in (None, "2^-7.5", "1/64"):
        t = bmm.empty(192, 640)
        bitgen.fill_device(t, 640, 23, 1, p=p, stream=torch.cuda.current_stream().cuda_stream)
        torch.cuda.synchronize()
        assert (from_dev(t, 192, 640) == gen(192, 640, 23, 1, p)).all()


def test_plan_pass_bytes_with_padded_k():
    """On the tensor paths a k that is not a multiple of 128 * 2^d bits is
    padded: the plan's streaming bytes then add the padded copy of A (A read,
    the copy written) and write Bt at the padded width, and every pass below
    works on kp (the closed form of a breadth-first plan, Secs. 3.9 and 3.11)."""
    if not bmm.device_supported():
        pytest.skip("tensor-core paths need sm_103")
    m, k, n, d = 2048, 2048 + 256, 1024, 2  # k: a multiple of 64 * 2^d, not of 128 * 2^d
    pl = bmm.plan(bmm.GF2, m, k, n, path=bmm.PATH_TC_FP4_PAIR, depth=d, serial=0)
    kp = pl["kp"]
    assert kp % (128 << d) == 0 and k < kp < k + (128 << d)
    grow = 7 ** d / 4 ** d
    want = (k * n + kp * n + m * k + m * kp + m * kp * (1 + grow) + kp * n * (1 + grow)
            + m * n * (1 + grow)) / 8
    assert pl["pass_bytes"] == want
