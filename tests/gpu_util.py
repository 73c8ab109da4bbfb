"""Helpers for the GPU parity tests: device buffers in the library's layout."""
import os
import re

import numpy as np
import torch

from conftest import ROOT


def shapes(elem_bytes):
    """(warps, chunks, mode) construct shapes compiled into the library."""
    text = open(os.path.join(ROOT, "paper_2404_04895_gb300", "csrc", "shapes.h")).read()
    name = "ACO_SHAPES_4B" if elem_bytes == 4 else "ACO_SHAPES_2B"
    body = text.split(f"#define {name}(X)")[1].split("\n\n")[0]
    return [(int(a), int(b), int(c)) for a, b, c in re.findall(r"X\((\d+),\s*(\d+),\s*(\d+)\)", body)]


def covers(shape, n, elem_bytes):
    return 32 * shape[0] * shape[1] * (16 // elem_bytes) >= n


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def padded_dev(mat, ld, np_dtype):
    """n x n host matrix -> n x ld device tensor, zero padding columns."""
    n = mat.shape[0]
    assert mat.shape == (n, n) and ld >= n
    out = np.zeros((n, ld), dtype=np_dtype)
    out[:, :n] = mat
    return dev(out)


def P_device(P_val, P_bits, prec, ld):
    if prec == 0:
        return padded_dev(P_val.astype(np.float32), ld, np.float32)
    return padded_dev(P_bits.view(np.int16), ld, np.int16)


def host(t, n=None):
    a = t.cpu().numpy()
    if n is not None:
        a = a[:, :n]
    return np.ascontiguousarray(a)
