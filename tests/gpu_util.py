"""Helpers shared by the GPU parity tests (test infrastructure)."""
import numpy as np
import torch

DEV = torch.device("cuda:0")


def np_of(t):
    return t.detach().cpu().numpy()


def assert_pairs_equal(got, exp):
    got = np_of(got)
    assert got.shape == exp.shape, (got.shape, exp.shape)
    if not np.array_equal(got, exp):
        bad = np.nonzero(np.any(got != exp, axis=1))[0]
        i = int(bad[0])
        raise AssertionError(f"{len(bad)} pairs differ; first at {i}: got {got[i]} exp {exp[i]}")
