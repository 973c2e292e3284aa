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
    """max |got - ref| / (D + |beta*C|), D = |alpha| |A| |B| from the oracle.

    With beta == 0 this is exactly max |C - C_ref| / (|alpha||A||B|)_ij.  With
    beta != 0 the |beta*C| term joins the denominator: the result is stored in
    float32, so rounding it alone costs up to 2^-24 |beta*C|, which no kernel
    can avoid when |beta*C| >> |alpha||A||B| (small k).  Entries whose
    denominator is 0 are compared against FLT_MIN."""
    got = np.asarray(got, np.float64)
    diff = np.abs(got - ref)
    den = np.array(D, np.float64, copy=True)
    if beta_c is not None:
        den = den + np.abs(beta_c)
    den = np.maximum(den, np.finfo(np.float32).tiny)
    return float(np.max(diff / den)) if diff.size else 0.0
