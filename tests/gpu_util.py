"""Helpers for the GPU tests: move packed words between numpy and the device."""
import numpy as np

import bitgen


def to_dev(words: np.ndarray):
    import torch

    return torch.from_numpy(np.ascontiguousarray(words).view(np.int64).ravel()).to("cuda")


def from_dev(t, rows: int, cols: int) -> np.ndarray:
    return t.cpu().numpy().view(np.uint64).reshape(rows, cols // 64)


def gen(rows: int, cols: int, seed: int, matrix_id: int, p=None) -> np.ndarray:
    return bitgen.fill_cpu(rows, cols, seed, matrix_id, p=p)


def first_mismatch(got: np.ndarray, want: np.ndarray):
    bad = np.argwhere(got != want)
    if len(bad) == 0:
        return None
    r, w = bad[0]
    return (int(r), int(w), hex(int(got[r, w])), hex(int(want[r, w])), len(bad))
