"""Full-size products (the benchmark's configurations) checked on outputs the
oracle computes one by one: sampled rows (oracle rows against the whole B),
sampled columns (oracle column against the whole A), and for GF(2) Freivalds
checks C x == A (B x) with seeded random vectors (a wrong C passes one vector
with probability <= 1/2).

Inputs on the GPU come from the device generator; the oracle's inputs come
from the CPU generator (the two are checked equal in test_gpu_parity)."""
import numpy as np
import pytest

import bitgen
import oracle as O
from gpu_util import from_dev

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover - CPU machine
    pytest.skip("no GPU", allow_module_level=True)

import paper_1909_01554_gb300 as bmm  # noqa: E402

IDS_GF2 = (0, 1)
IDS_BOOL = (4, 5)


def dev_gen(rows, cols, seed, mid, p):
    t = bmm.empty(rows, cols)
    bitgen.fill_device(t, cols, seed, mid, p=p, stream=torch.cuda.current_stream().cuda_stream)
    return t


def sampled_check(op, n, seed, ids, p, C, nrows=8, ncols=8, freivalds=8):
    """C (host, n x n/64 words) against oracle rows, columns and Freivalds."""
    rng = np.random.default_rng(seed * 7919 + op)
    o = O.GF2 if op == bmm.GF2 else O.BOOL
    B = bitgen.fill_cpu(n, n, seed, ids[1], p=p)
    rows = sorted(rng.choice(n, nrows, replace=False).tolist())
    Ar = np.concatenate([bitgen.fill_cpu(n, n, seed, ids[0], p=p, row0=r, nrows=1) for r in rows])
    want_rows = O.rows(o, Ar, B, n, n)
    for i, r in enumerate(rows):
        assert (C[r] == want_rows[i]).all(), f"row {r}"
    A = bitgen.fill_cpu(n, n, seed, ids[0], p=p)
    for j in sorted(rng.choice(n, ncols, replace=False).tolist()):
        want = O.column(o, A, B, j, n, n, n)
        got = ((C[:, j // 64] >> np.uint64(j % 64)) & np.uint64(1)).astype(np.uint8)
        assert (got == want).all(), f"column {j}"
    if op == bmm.GF2:
        for _ in range(freivalds):
            x = rng.integers(0, np.iinfo(np.uint64).max, size=n // 64, dtype=np.uint64,
                             endpoint=True)
            assert (O.matvec_gf2(C, x, n, n) ==
                    O.matvec_gf2(A, O.matvec_gf2(B, x, n, n), n, n)).all(), "Freivalds"
    # Output density: k p^2 = 1 in every Boolean workload -> 1 - 1/e; a GF(2)
    # product of uniform random bits is uniform -> 1/2
    dens = np.unpackbits(C[:: max(1, n // 512)].view(np.uint8)).mean()
    if op == bmm.BOOL:
        assert abs(dens - (1 - np.exp(-1))) < 0.02
    else:
        assert abs(dens - 0.5) < 0.01


def run_product(op, n, seed, ids, p, **kw):
    A = dev_gen(n, n, seed, ids[0], p)
    B = dev_gen(n, n, seed, ids[1], p)
    C = bmm.empty(n, n)
    C.fill_(-1)
    bmm.product(op, A, B, C, n, n, n, **kw)
    bmm.stream_status()
    out = from_dev(C, n, n)
    del A, B, C
    torch.cuda.empty_cache()
    return out


def test_config2_square32768_bench_launch_configuration():
    """m = k = n = 32768, seed 2: GF(2) p = 1/2 and Boolean p = 2^-7.5 in the
    configuration bench.py times (autotuned first, as the bench does: for
    GF(2) a self-inverse Strassen depth on the tensor base case), and GF(2)
    also at the planner's untuned rule (depth 2)."""
    n, seed = 32768, 2
    bmm.autotune_clear()
    assert bmm.plan(bmm.GF2, n, n, n)["strassen_depth"] == 2  # the untuned rule
    Cg = run_product(bmm.GF2, n, seed, IDS_GF2, None)
    sampled_check(bmm.GF2, n, seed, IDS_GF2, None, Cg)
    del Cg
    tg = bmm.autotune(bmm.GF2, n, n, n)
    tb = bmm.autotune(bmm.BOOL, n, n, n)
    info = bmm.plan(bmm.GF2, n, n, n)
    assert (info["path"], info["strassen_depth"]) == (tg["path"], tg["strassen_depth"])
    Cg = run_product(bmm.GF2, n, seed, IDS_GF2, None)
    sampled_check(bmm.GF2, n, seed, IDS_GF2, None, Cg)
    del Cg
    assert bmm.plan(bmm.BOOL, n, n, n)["path"] == tb["path"]
    Cb = run_product(bmm.BOOL, n, seed, IDS_BOOL, "2^-7.5")
    sampled_check(bmm.BOOL, n, seed, IDS_BOOL, "2^-7.5", Cb)
    bmm.autotune_clear()


def test_config3_square65536_paths_agree():
    """m = k = n = 65536, seed 3: the tensor-core base cases (one SM or an SM
    pair per tile, e4m3 or e2m1 operands) and the CUDA-core base case give
    bit-identical products
    (cubic), and match the oracle's samples; the planner's Strassen product
    matches too. GF(2) p = 1/2, Boolean p = 2^-8."""
    n, seed = 65536, 3
    if not bmm.device_supported():
        pytest.skip("tensor-core path needs sm_103")
    for op, ids, p in ((bmm.GF2, IDS_GF2, None), (bmm.BOOL, IDS_BOOL, "2^-8")):
        tc = run_product(op, n, seed, ids, p, path=bmm.PATH_TC_FP8, depth=0)
        pc = run_product(op, n, seed, ids, p, path=bmm.PATH_POPC, depth=0)
        assert (tc == pc).all(), f"tensor vs CUDA-core disagree (op={op})"
        tp = run_product(op, n, seed, ids, p, path=bmm.PATH_TC_FP8_PAIR, depth=0)
        assert (tp == tc).all(), f"SM-pair vs single-SM tensor paths disagree (op={op})"
        del tp
        t4 = run_product(op, n, seed, ids, p, path=bmm.PATH_TC_FP4_PAIR, depth=0)
        assert (t4 == tc).all(), f"e2m1 vs e4m3 tensor paths disagree (op={op})"
        del t4
        if op == bmm.GF2:
            st = run_product(op, n, seed, ids, p)
            assert (st == tc).all(), "Strassen (planner rule) vs cubic disagree"
            del st
            bmm.autotune(op, n, n, n)  # the configuration bench.py times
            st = run_product(op, n, seed, ids, p)
            bmm.autotune_clear()
            assert (st == tc).all(), "Strassen (autotuned) vs cubic disagree"
            del st
        sampled_check(op, n, seed, ids, p, tc, nrows=4, ncols=4, freivalds=4)


def test_config4_square524288():
    """m = k = n = 2^19 (32 GiB per operand, minutes), seed 4: GF(2) p = 1/2
    through the planner's Strassen (depth-first top levels so that it fits
    HBM), Boolean p = 2^-9.5 cubic; sampled rows and columns plus GF(2)
    Freivalds."""
    n, seed = 1 << 19, 4
    Cg = run_product(bmm.GF2, n, seed, IDS_GF2, None)
    sampled_check(bmm.GF2, n, seed, IDS_GF2, None, Cg, nrows=4, ncols=4, freivalds=4)
    del Cg
    Cb = run_product(bmm.BOOL, n, seed, IDS_BOOL, "2^-9.5")
    sampled_check(bmm.BOOL, n, seed, IDS_BOOL, "2^-9.5", Cb, nrows=4, ncols=4, freivalds=0)
