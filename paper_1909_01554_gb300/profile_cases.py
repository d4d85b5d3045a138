"""Small cases of the library's kernels for a profiler: each case prepares its
operands, runs its call once untimed, then once more inside an NVTX range
named "bmm_case", so that a profiler can capture exactly the launches of that
second call, e.g.

  ncu --set full --clock-control none --nvtx --nvtx-include "bmm_case/" \\
      -k regex:tc_nt_kernel -c 1 -o prof python -m paper_1909_01554_gb300.profile_cases batched256

Cases (operands from the seeded generator, each a few hundred MB to ~1.5 GB):
  batched256     the first 256 problems of the 2048-problem batch (seed 5)
  leaves_d2      GF(2) 32768^3 on e2m1 SM pairs, Strassen depth 2 breadth-first:
                 one launch over 49 leaves of 8192^3
  level_d2       the same product with the innermost level inside the tensor
                 kernel: one launch over 7 blocks of 16384^3
  popc_level_d1  GF(2) 8192^3 on the CUDA cores, depth 1 inside the kernel
  popc_d1        the same product with the level in XOR passes
"""
from __future__ import annotations

import os
import sys


def _setup():
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    if root not in sys.path:
        sys.path.insert(0, root)
    import torch

    torch.cuda.set_device(0)
    return torch


def _square(torch, bmm, n, seed=2):
    import bitgen

    sh = torch.cuda.current_stream().cuda_stream
    A, B, C = bmm.empty(n, n), bmm.empty(n, n), bmm.empty(n, n)
    bitgen.fill_device(A, n, seed, 0, stream=sh)
    bitgen.fill_device(B, n, seed, 1, stream=sh)
    return A, B, C, sh


def run(case: str) -> None:
    torch = _setup()
    import bitgen
    import paper_1909_01554_gb300 as bmm

    nv = torch.cuda.nvtx
    if case == "batched256":
        sh = torch.cuda.current_stream().cuda_stream
        shapes = bitgen.batched_shapes(2048, 5)[:256]
        As, Bs, Cs = [], [], []
        for i, (m, k, n, op) in enumerate(shapes):
            A, B, C = bmm.empty(m, k), bmm.empty(k, n), bmm.empty(m, n)
            p = None if op == 0 else f"1/sqrt({k})"
            bitgen.fill_device(A, k, (5 << 16) + i, 0, p=p, stream=sh)
            bitgen.fill_device(B, n, (5 << 16) + i, 1, p=p, stream=sh)
            As.append(A)
            Bs.append(B)
            Cs.append(C)
        plan = bmm.BatchedPlan([s[3] for s in shapes], As, Bs, Cs, [s[0] for s in shapes],
                               [s[1] for s in shapes], [s[2] for s in shapes])
        call = lambda: plan.run(stream=sh)  # noqa: E731
    elif case in ("leaves_d2", "level_d2"):
        A, B, C, sh = _square(torch, bmm, 32768)
        kw = dict(path=bmm.PATH_TC_FP4_PAIR, depth=2, serial=0,
                  kernel_level=1 if case == "level_d2" else 0)
        call = lambda: bmm.gf2(A, B, C, 32768, 32768, 32768, stream=sh, **kw)  # noqa: E731
    elif case in ("popc_level_d1", "popc_d1"):
        A, B, C, sh = _square(torch, bmm, 8192)
        kw = dict(path=bmm.PATH_POPC, depth=1, kernel_level=1 if case == "popc_level_d1" else 0)
        call = lambda: bmm.gf2(A, B, C, 8192, 8192, 8192, stream=sh, **kw)  # noqa: E731
    else:
        raise SystemExit(f"unknown case {case!r}")
    call()
    torch.cuda.synchronize()
    nv.range_push("bmm_case")
    call()
    torch.cuda.synchronize()
    nv.range_pop()
    bmm.stream_status(sh)


if __name__ == "__main__":
    for c in sys.argv[1:] or ["batched256"]:
        run(c)
