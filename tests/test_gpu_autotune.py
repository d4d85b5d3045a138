"""The autotuner: its recorded choice drives the planner's automatic mode and
the products it chooses stay bit-exact against the oracle."""
import pytest

import oracle as O
from gpu_util import first_mismatch, from_dev, gen, to_dev

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover - CPU machine
    pytest.skip("no GPU", allow_module_level=True)

import paper_1909_01554_gb300 as bmm  # noqa: E402

VALID_PATHS = {*bmm.TENSOR_PATHS, bmm.PATH_POPC}


def product_matches(op, m, k, n, seed):
    p = None if op == bmm.GF2 else "1/32"
    Ah, Bh = gen(m, k, seed, 0, p), gen(k, n, seed, 1, p)
    dC = bmm.empty(m, n)
    dC.fill_(-1)
    bmm.product(op, to_dev(Ah), to_dev(Bh), dC, m, k, n)
    bmm.stream_status()
    want = O.cubic(O.GF2 if op == bmm.GF2 else O.BOOL, Ah, Bh, m, k, n)
    return first_mismatch(from_dev(dC, m, n), want)


@pytest.mark.parametrize("model", [False, True])
def test_tuned_choice_drives_the_planner(model):
    bmm.autotune_clear()
    m, k, n = 2048, 2048, 1536
    r = bmm.autotune(bmm.GF2, m, k, n, model=model)
    assert r["measured"] == (not model)
    assert r["path"] in VALID_PATHS and 0 <= r["strassen_depth"] <= 2
    assert r["est_ms"] > 0 and r["candidates"] >= 3
    info = bmm.plan(bmm.GF2, m, k, n)
    assert (info["path"], info["strassen_depth"]) == (r["path"], r["strassen_depth"])
    assert product_matches(bmm.GF2, m, k, n, 51) is None
    bmm.autotune_clear()


def test_boolean_tunes_the_path_only():
    bmm.autotune_clear()
    r = bmm.autotune(bmm.BOOL, 1024, 2048, 1024)
    assert r["strassen_depth"] == 0 and r["path"] in VALID_PATHS
    assert bmm.plan(bmm.BOOL, 1024, 2048, 1024)["path"] == r["path"]
    assert product_matches(bmm.BOOL, 1024, 2048, 1024, 52) is None
    bmm.autotune_clear()


def test_tensor_cores_beat_cuda_cores_on_a_large_cubic_shape():
    """At 16384^3 both ways of timing pick a tensor-core path over the
    CUDA-core one for the cubic product (Boolean: depth fixed at 0)."""
    if not bmm.device_supported():
        pytest.skip("tensor-core paths need sm_103")
    bmm.autotune_clear()
    for model in (False, True):
        r = bmm.autotune(bmm.BOOL, 16384, 16384, 16384, model=model)
        assert r["path"] in bmm.TENSOR_PATHS
    bmm.autotune_clear()
