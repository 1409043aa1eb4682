"""Helpers for the GPU parity tests: device round trips and result checks."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")


def need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def to_dev_keys(keys: np.ndarray):
    return torch.from_numpy(np.ascontiguousarray(keys)).cuda()


def to_dev_payload(p: np.ndarray):
    return torch.from_numpy(np.ascontiguousarray(p).view(np.int32)).cuda()


def from_dev(keys_t, pay_t):
    k = keys_t.cpu().numpy()
    p = None if pay_t is None else pay_t.cpu().numpy().view(np.uint32)
    return k, p


def assert_bitexact(got_k, got_p, want_k, want_p):
    gk = got_k.view(np.uint64)
    wk = want_k.view(np.uint64)
    if not np.array_equal(gk, wk):
        bad = np.flatnonzero(gk != wk)
        raise AssertionError(f"keys differ at {bad.size} positions, first {bad[:8].tolist()}")
    if want_p is not None:
        if not np.array_equal(got_p, want_p):
            bad = np.flatnonzero(got_p != want_p)
            raise AssertionError(f"payload differs at {bad.size} positions, first {bad[:8].tolist()}")
