"""Batched uneven products (one persistent launch) against the CPU oracle.

Problem i of a batch draws its inputs from the generator with seed
base * 2^16 + i (A: matrix id 0, B: matrix id 1)."""
import numpy as np
import pytest

import bitgen
import oracle as O
from gpu_util import first_mismatch, from_dev, to_dev

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover - CPU machine
    pytest.skip("no GPU", allow_module_level=True)

import paper_1909_01554_gb300 as bmm  # noqa: E402


def density(op, k):
    return None if op == bmm.GF2 else f"1/sqrt({k})"


def make_batch(shapes, base_seed):
    host, dev = [], []
    for i, (m, k, n, op) in enumerate(shapes):
        seed = (base_seed << 16) + i
        A = bitgen.fill_cpu(m, k, seed, 0, p=density(op, k))
        B = bitgen.fill_cpu(k, n, seed, 1, p=density(op, k))
        host.append((A, B))
        C = bmm.empty(m, n)
        C.fill_(-1)
        dev.append((to_dev(A), to_dev(B), C))
    return host, dev


def check_all(shapes, host, dev, which=None):
    for i, ((m, k, n, op), (A, B), (_, _, C)) in enumerate(zip(shapes, host, dev)):
        if which is not None and i not in which:
            continue
        want = O.cubic(O.GF2 if op == bmm.GF2 else O.BOOL, A, B, m, k, n)
        mm = first_mismatch(from_dev(C, m, n), want)
        assert mm is None, f"problem {i} {(m, k, n, op)}: {mm}"


SMALL = [(64, 64, 64, 0), (192, 320, 448, 1), (384, 1152, 320, 0), (128, 256, 256, 1),
         (576, 704, 832, 0), (256, 128, 64, 1), (1024, 960, 1088, 0), (64, 2048, 192, 1)]


def test_batched_mixed_small():
    host, dev = make_batch(SMALL, 41)
    ops = [s[3] for s in SMALL]
    bmm.batched(ops, [d[0] for d in dev], [d[1] for d in dev], [d[2] for d in dev],
                [s[0] for s in SMALL], [s[1] for s in SMALL], [s[2] for s in SMALL])
    bmm.stream_status()
    check_all(SMALL, host, dev)


@pytest.mark.parametrize("path", [bmm.PATH_POPC, *bmm.TENSOR_PATHS])
def test_batched_plan_on_each_path(path):
    """The same uneven batch through a plan on every base case (the automatic
    choice takes the fastest; the others stay reachable and exact)."""
    if path != bmm.PATH_POPC and not bmm.device_supported():
        pytest.skip("tensor-core paths need sm_103")
    host, dev = make_batch(SMALL, 43)
    ops = [s[3] for s in SMALL]
    plan = bmm.BatchedPlan(ops, [d[0] for d in dev], [d[1] for d in dev], [d[2] for d in dev],
                           [s[0] for s in SMALL], [s[1] for s in SMALL], [s[2] for s in SMALL],
                           path=path)
    assert plan.path() == path
    plan.run()
    bmm.stream_status()
    plan.destroy()
    check_all(SMALL, host, dev)


def test_batched_plan_auto_path_is_fastest_tensor_path():
    if not bmm.device_supported():
        pytest.skip("tensor-core paths need sm_103")
    host, dev = make_batch(SMALL[:2], 47)
    plan = bmm.BatchedPlan([s[3] for s in SMALL[:2]], [d[0] for d in dev], [d[1] for d in dev],
                           [d[2] for d in dev], [s[0] for s in SMALL[:2]],
                           [s[1] for s in SMALL[:2]], [s[2] for s in SMALL[:2]])
    st = plan.stats()
    assert st["tensor_path"] == bmm.plan(bmm.GF2, 4096, 4096, 4096, depth=0)["path"]
    assert st["tensor_path"] == bmm.PATH_TC_FP4_PAIR
    plan.destroy()


def run_plan(shapes, seed, **kw):
    host, dev = make_batch(shapes, seed)
    plan = bmm.BatchedPlan([s[3] for s in shapes], [d[0] for d in dev], [d[1] for d in dev],
                           [d[2] for d in dev], [s[0] for s in shapes], [s[1] for s in shapes],
                           [s[2] for s in shapes], **kw)
    plan.run()
    bmm.stream_status()
    return host, dev, plan


def test_batched_model_is_measured():
    """The cost model the plans decide with is measured on this device, per
    stage of k and per tile of each kernel."""
    m = bmm.batched_model(bmm.PATH_POPC)
    assert m["measured"] == 1 and m["popc_units"] > 0
    assert m["popc_stage_ns"] > 0 and m["popc_tile_ns"] >= 0
    if bmm.device_supported():
        for path in bmm.TENSOR_PATHS:
            t = bmm.batched_model(path)
            assert t["measured"] == 1 and t["path"] == path and t["tensor_units"] > 0
            assert t["tensor_stage_ns"] > 0 and t["tensor_stage_n128_ns"] > 0
            assert t["tensor_tile_ns"] >= 0


def test_batched_per_problem_paths():
    """Base cases named per problem (CUDA cores, the tensor path, or left to
    the model) in one plan: each problem runs where it was sent, all exact."""
    if not bmm.device_supported():
        pytest.skip("tensor-core paths need sm_103")
    req = [bmm.PATH_POPC, bmm.PATH_TC_FP4_PAIR, bmm.PATH_AUTO, bmm.PATH_POPC,
           bmm.PATH_TC_FP4_PAIR, bmm.PATH_AUTO, bmm.PATH_POPC, bmm.PATH_TC_FP4_PAIR]
    host, dev, plan = run_plan(SMALL, 53, paths=req)
    st = plan.stats()
    for i, r in enumerate(req):
        c = plan.choice(i)
        if r != bmm.PATH_AUTO:
            assert c["path"] == r, (i, c)
        assert c["path"] in (bmm.PATH_POPC, bmm.PATH_TC_FP4_PAIR)
        assert c["strassen_depth"] == 0
    assert st["popc_problems"] >= 3 and st["tensor_problems"] >= 3
    assert st["popc_problems"] + st["tensor_problems"] == len(SMALL)
    check_all(SMALL, host, dev)
    plan.destroy()
    with pytest.raises(bmm.BmmError) as e:  # two tensor paths in one plan
        bmm.BatchedPlan([s[3] for s in SMALL[:2]], [d[0] for d in dev[:2]],
                        [d[1] for d in dev[:2]], [d[2] for d in dev[:2]],
                        [s[0] for s in SMALL[:2]], [s[1] for s in SMALL[:2]],
                        [s[2] for s in SMALL[:2]],
                        paths=[bmm.PATH_TC_FP4_PAIR, bmm.PATH_TC_FP8_PAIR])
    assert e.value.status == bmm.ERR_INVALID


# Tail tiles and half k stages: n = 256 j + 64 or + 128 leaves at most 128
# columns in the last column tile (N = 128 where the model measured that form
# cheaper); k = 768 and 1280 are 3 and 5 stages of 256 bits (the last packed
# stage of 512 is half padding, not multiplied), k = 320 and 448 pad to 384
# and 512; m = 320 and 704 leave part of the last 256-row tile empty.
TAILS = [(320, 768, 320, 0), (704, 1280, 384, 1), (256, 256, 128, 0), (448, 320, 64, 1),
         (320, 448, 576, 0), (1024, 1792, 1152, 1), (64, 768, 192, 0), (512, 256, 640, 1)]


@pytest.mark.parametrize("path", list(bmm.TENSOR_PATHS))
def test_batched_tail_tiles_and_half_stages(path):
    if not bmm.device_supported():
        pytest.skip("tensor-core paths need sm_103")
    model = bmm.batched_model(path)
    host, dev, plan = run_plan(TAILS, 59, path=path)
    kstep = 256 if path == bmm.PATH_TC_FP4_PAIR else 128
    narrow = model["tensor_stage_n128_ns"] < model["tensor_stage_ns"]
    for i, (m, k, n, op) in enumerate(TAILS):
        c = plan.choice(i)
        assert c["path"] == path and c["k_step"] == kstep
        kpad = (k // 64 + 1) // 2 * 2 * 64
        assert c["k_steps"] == -(-kpad // kstep)
        tail = n - (-(-n // 256) - 1) * 256
        assert c["tail_n"] == (128 if narrow and tail <= 128 else 256), (i, c)
    st = plan.stats()
    if narrow:
        assert st["tensor_tiles_n128"] > 0
    assert st["macs_issued"] >= st["macs_needed"]
    check_all(TAILS, host, dev)
    plan.destroy()


def test_uniform_op_batched_entry_points():
    shapes = [(s[0], s[1], s[2], 0) for s in SMALL[:4]]
    host, dev = make_batch(shapes, 42)
    L = bmm.lib()
    import ctypes

    arr = bmm._batch_arrays([0] * 4, [d[0] for d in dev], [d[1] for d in dev],
                            [d[2] for d in dev], [s[0] for s in shapes], [s[1] for s in shapes],
                            [s[2] for s in shapes])
    st = L.bmm_gf2_batched(arr[0], *arr[2:], ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == bmm.OK
    check_all(shapes, host, dev)


def test_plan_reuse_and_graph_replay():
    shapes = bitgen.batched_shapes(48, 7, lo=256, hi=1536)
    host, dev = make_batch(shapes, 43)
    plan = bmm.BatchedPlan([s[3] for s in shapes], [d[0] for d in dev], [d[1] for d in dev],
                           [d[2] for d in dev], [s[0] for s in shapes], [s[1] for s in shapes],
                           [s[2] for s in shapes])
    plan.run()
    bmm.stream_status()
    check_all(shapes, host, dev)
    # new data in the same buffers, replayed through a captured CUDA graph
    host2 = []
    for i, ((m, k, n, op), (dA, dB, dC)) in enumerate(zip(shapes, dev)):
        seed = (44 << 16) + i
        A = bitgen.fill_cpu(m, k, seed, 0, p=density(op, k))
        B = bitgen.fill_cpu(k, n, seed, 1, p=density(op, k))
        dA.copy_(to_dev(A))
        dB.copy_(to_dev(B))
        dC.fill_(-1)
        host2.append((A, B))
    torch.cuda.synchronize()
    s = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        plan.run(stream=s)
    g.replay()
    torch.cuda.synchronize()
    bmm.stream_status()
    check_all(shapes, host2, dev)
    plan.destroy()


def test_batched_config5_shapes_sampled():
    """2048 problems, m, k, n log-uniform in [256, 8192] (multiples of 64), 50/50
    GF(2)/Boolean, seed 5: every problem checked on two oracle rows, 12 in full."""
    shapes = bitgen.batched_shapes(2048, 5)
    dev, rows = [], []
    rng = np.random.default_rng(5)
    for i, (m, k, n, op) in enumerate(shapes):
        seed = (5 << 16) + i
        A = bmm.empty(m, k)
        B = bmm.empty(k, n)
        bitgen.fill_device(A, k, seed, 0, p=density(op, k))
        bitgen.fill_device(B, k, seed, 1, p=density(op, k))
        C = bmm.empty(m, n)
        C.fill_(-1)
        dev.append((A, B, C))
        rows.append(sorted(rng.choice(m, 2, replace=False).tolist()))
    torch.cuda.synchronize()
    plan = bmm.BatchedPlan([s[3] for s in shapes], [d[0] for d in dev], [d[1] for d in dev],
                           [d[2] for d in dev], [s[0] for s in shapes], [s[1] for s in shapes],
                           [s[2] for s in shapes])
    st = plan.stats()
    assert st["problems"] == 2048
    assert st["macs_needed"] == float(sum(m * k * n for m, k, n, _ in shapes))
    assert st["macs_issued"] >= st["macs_needed"]
    plan.run()
    bmm.stream_status()
    plan.destroy()
    full = set(rng.choice(2048, 12, replace=False).tolist())
    for i, (m, k, n, op) in enumerate(shapes):
        seed = (5 << 16) + i
        p = density(op, k)
        B = bitgen.fill_cpu(k, n, seed, 1, p=p)
        got = from_dev(dev[i][2], m, n)
        o = O.GF2 if op == bmm.GF2 else O.BOOL
        if i in full:
            A = bitgen.fill_cpu(m, k, seed, 0, p=p)
            mm = first_mismatch(got, O.cubic(o, A, B, m, k, n))
            assert mm is None, f"problem {i} {(m, k, n, op)}: {mm}"
        else:
            for r in rows[i]:
                Ar = bitgen.fill_cpu(m, k, seed, 0, p=p, row0=r, nrows=1)
                want = O.rows(o, Ar, B, k, n)
                assert (got[r] == want[0]).all(), f"problem {i} row {r}"


def test_plan_first_run_captured_in_a_graph():
    """A plan whose very first run is captured in a CUDA graph (everything a
    run needs is set up when the plan is made), with problems on both base
    cases, then replayed: exact."""
    if not bmm.device_supported():
        pytest.skip("tensor-core paths need sm_103")
    shapes = SMALL + [(1024, 1024, 1024, 0), (512, 2048, 768, 1)]
    req = [bmm.PATH_POPC if i % 3 == 0 else bmm.PATH_AUTO for i in range(len(shapes))]
    host, dev = make_batch(shapes, 71)
    plan = bmm.BatchedPlan([s[3] for s in shapes], [d[0] for d in dev], [d[1] for d in dev],
                           [d[2] for d in dev], [s[0] for s in shapes], [s[1] for s in shapes],
                           [s[2] for s in shapes], paths=req)
    torch.cuda.synchronize()
    s = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        plan.run(stream=s)
    g.replay()
    torch.cuda.synchronize()
    bmm.stream_status()
    check_all(shapes, host, dev)
    plan.destroy()


def test_empty_batch_plan():
    """A plan over no problems builds, runs (launching nothing) and frees."""
    L = bmm.lib()
    import ctypes

    h = ctypes.c_void_p(0)
    assert L.bmm_batched_plan_create(0, None, None, None, None, None, None, None,
                                     ctypes.byref(h)) == bmm.OK
    l0 = bmm.launch_count()
    assert L.bmm_batched_plan_run(h, None) == bmm.OK
    assert bmm.launch_count() == l0
    st = bmm.BatchedStats()
    assert L.bmm_batched_plan_stats(h, ctypes.byref(st)) == bmm.OK and st.problems == 0
    assert L.bmm_batched_plan_destroy(h) == bmm.OK


def test_batched_strassen_problems():
    """Binary problems of 16384^3 get the single-product planner's depth
    (one level: leaves of 8192) and run as their own Strassen products after
    the batched launches, on the tensor path or, when sent there, the CUDA
    cores; a Boolean problem of the same size stays cubic. Every product
    equals the cubic single product bit for bit and the oracle's sampled
    rows; a second run replayed from a captured graph is exact too."""
    if not bmm.device_supported():
        pytest.skip("tensor-core paths need sm_103")
    bmm.autotune_clear()
    big = 16384
    # the last binary problem's k (16512) pads to 16640 on the tensor path
    # (leaf k a multiple of 128 bits), so its plan holds a padded copy of A
    shapes = [(big, big, big, 0), (512, 768, 1024, 0), (big, big, big, 0),
              (big, 8192, big, 1), (1024, 1024, 1088, 1), (big + 128, big + 128, big, 0)]
    req = [bmm.PATH_AUTO, bmm.PATH_AUTO, bmm.PATH_POPC, bmm.PATH_AUTO, bmm.PATH_AUTO,
           bmm.PATH_AUTO]
    sh = torch.cuda.current_stream().cuda_stream
    dev = []
    for i, (m, k, n, op) in enumerate(shapes):
        seed = (73 << 16) + i
        A, B, C = bmm.empty(m, k), bmm.empty(k, n), bmm.empty(m, n)
        bitgen.fill_device(A, k, seed, 0, p=density(op, k), stream=sh)
        bitgen.fill_device(B, n, seed, 1, p=density(op, k), stream=sh)
        C.fill_(-1)
        dev.append((A, B, C))
    plan = bmm.BatchedPlan([s[3] for s in shapes], [d[0] for d in dev], [d[1] for d in dev],
                           [d[2] for d in dev], [s[0] for s in shapes], [s[1] for s in shapes],
                           [s[2] for s in shapes], paths=req)
    want_depth = [1, 0, 1, 0, 0, 1]
    for i, d in enumerate(want_depth):
        c = plan.choice(i)
        assert c["strassen_depth"] == d, (i, c)
    assert plan.choice(2)["path"] == bmm.PATH_POPC
    assert plan.choice(0)["path"] in bmm.TENSOR_PATHS
    st = plan.stats()
    assert st["strassen_problems"] == 3
    assert st["tensor_problems"] + st["popc_problems"] == len(shapes)
    plan.run()
    bmm.stream_status()
    rng = np.random.default_rng(73)

    def check():
        for i, (m, k, n, op) in enumerate(shapes):
            seed = (73 << 16) + i
            got = from_dev(dev[i][2], m, n)
            ref = bmm.empty(m, n)
            bmm.product(op, dev[i][0], dev[i][1], ref, m, k, n, path=bmm.PATH_TC_FP4_PAIR,
                        depth=0)
            bmm.stream_status()
            assert (got == from_dev(ref, m, n)).all(), f"problem {i} vs cubic"
            del ref
            p = density(op, k)
            B = bitgen.fill_cpu(k, n, seed, 1, p=p)
            o = O.GF2 if op == bmm.GF2 else O.BOOL
            for r in sorted(rng.choice(m, 2, replace=False).tolist()):
                Ar = bitgen.fill_cpu(m, k, seed, 0, p=p, row0=r, nrows=1)
                assert (got[r] == O.rows(o, Ar, B, k, n)[0]).all(), f"problem {i} row {r}"

    check()
    for d in dev:
        d[2].fill_(-1)
    torch.cuda.synchronize()
    s = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        plan.run(stream=s)
    g.replay()
    torch.cuda.synchronize()
    bmm.stream_status()
    check()
    plan.destroy()
    del g, dev
    torch.cuda.empty_cache()


def test_batched_strassen_problem_follows_the_plan_path():
    """A plan made on the e4m3 SM-pair path (every entry names it) runs its
    Strassen problem on that path too: depth 1, bit-identical to the cubic
    e2m1 product."""
    if not bmm.device_supported():
        pytest.skip("tensor-core paths need sm_103")
    bmm.autotune_clear()
    big = 16384
    shapes = [(big, big, big, 0), (512, 640, 768, 1)]
    sh = torch.cuda.current_stream().cuda_stream
    dev = []
    for i, (m, k, n, op) in enumerate(shapes):
        A, B, C = bmm.empty(m, k), bmm.empty(k, n), bmm.empty(m, n)
        bitgen.fill_device(A, k, (79 << 16) + i, 0, p=density(op, k), stream=sh)
        bitgen.fill_device(B, n, (79 << 16) + i, 1, p=density(op, k), stream=sh)
        C.fill_(-1)
        dev.append((A, B, C))
    plan = bmm.BatchedPlan([s[3] for s in shapes], [d[0] for d in dev], [d[1] for d in dev],
                           [d[2] for d in dev], [s[0] for s in shapes], [s[1] for s in shapes],
                           [s[2] for s in shapes], path=bmm.PATH_TC_FP8_PAIR)
    c = plan.choice(0)
    assert (c["path"], c["strassen_depth"], c["k_step"]) == (bmm.PATH_TC_FP8_PAIR, 1, 128)
    assert plan.choice(1)["strassen_depth"] == 0
    plan.run()
    bmm.stream_status()
    for i, (m, k, n, op) in enumerate(shapes):
        ref = bmm.empty(m, n)
        bmm.product(op, dev[i][0], dev[i][1], ref, m, k, n, path=bmm.PATH_TC_FP4_PAIR, depth=0)
        bmm.stream_status()
        assert (from_dev(dev[i][2], m, n) == from_dev(ref, m, n)).all(), f"problem {i}"
    plan.destroy()


def test_batched_problem_follows_a_tuned_record():
    """A binary shape the autotuner has recorded gets, inside a batch, the
    depth (and, with depth > 0, the path) a single product of that shape
    gets; the product is exact either way."""
    if not bmm.device_supported():
        pytest.skip("tensor-core paths need sm_103")
    n = 8192
    bmm.autotune_clear()
    try:
        bmm.autotune(bmm.GF2, n, n, n)
        single = bmm.plan(bmm.GF2, n, n, n)
        shapes = [(n, n, n, 0), (320, 448, 576, 1)]
        host, dev = make_batch(shapes, 83)
        plan = bmm.BatchedPlan([s[3] for s in shapes], [d[0] for d in dev],
                               [d[1] for d in dev], [d[2] for d in dev],
                               [s[0] for s in shapes], [s[1] for s in shapes],
                               [s[2] for s in shapes])
        c = plan.choice(0)
        assert c["strassen_depth"] == single["strassen_depth"]
        if single["strassen_depth"] > 0:
            assert c["path"] == single["path"]
        plan.run()
        bmm.stream_status()
        check_all(shapes, host, dev, which={1})
        ref = bmm.empty(n, n)
        bmm.product(bmm.GF2, dev[0][0], dev[0][1], ref, n, n, n, path=bmm.PATH_TC_FP4_PAIR,
                    depth=0)
        bmm.stream_status()
        assert (from_dev(dev[0][2], n, n) == from_dev(ref, n, n)).all()
        plan.destroy()
    finally:
        bmm.autotune_clear()
