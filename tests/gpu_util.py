"""Helpers of the GPU parity tests: device transfer, guard-banded output
buffers and the error metric max |C - C_ref| / (|alpha| |A| |B|)_ij."""
import numpy as np
import torch

SENTINEL = 12345.678


def dev(x, dtype=None):
    t = torch.from_numpy(np.ascontiguousarray(x)).cuda()
    return t if dtype is None else t.to(dtype)


def guarded(m, n, init=None, pad_rows=2, pad_cols=5, dtype=torch.float32):
    """An m x n view inside a larger buffer filled with a sentinel, so that any
    write outside the m x n window (including the columns between n and the
    leading dimension) is detected by check_guard()."""
    full = torch.full((m + 2 * pad_rows, n + 2 * pad_cols), SENTINEL if dtype == torch.float32 else 77,
                      dtype=dtype, device="cuda")
    view = full[pad_rows:pad_rows + m, pad_cols:pad_cols + n]
    if init is not None:
        view.copy_(torch.from_numpy(np.ascontiguousarray(init)).to(dtype))
    return full, view


def check_guard(full, m, n, pad_rows=2, pad_cols=5):
    f = full.cpu().numpy()
    mask = np.ones(f.shape, bool)
    mask[pad_rows:pad_rows + m, pad_cols:pad_cols + n] = False
    want = SENTINEL if full.dtype == torch.float32 else 77
    bad = np.argwhere(f[mask] != np.float32(want) if full.dtype == torch.float32 else f[mask] != want)
    assert bad.size == 0, f"{bad.size} guard elements overwritten"


def rel_err(got, ref, D, beta_c=None):
    """max |got - ref| / D over D > 0; where D == 0 the difference is measured
    against max(|beta*C|, FLT_MIN) instead."""
    got = np.asarray(got, np.float64)
    diff = np.abs(got - ref)
    pos = D > 0
    e = float(np.max(diff[pos] / D[pos])) if pos.any() else 0.0
    if (~pos).any():
        base = np.full(diff.shape, np.finfo(np.float32).tiny)
        if beta_c is not None:
            base = np.maximum(base, np.abs(beta_c))
        e = max(e, float(np.max(diff[~pos] / base[~pos])))
    return e
