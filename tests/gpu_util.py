"""Helpers of the GPU parity tests: device transfer, guard-banded output
buffers and the error metric max |C - C_ref| / (|alpha| |A| |B|)_ij, both as
stated (strict) and with |beta C| added to the denominator."""
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


def rel_errs(got, ref, D, beta_c=None):
    """(strict, with_beta): the error over |alpha||A||B| alone, as the targets
    state it, and over |alpha||A||B| + |beta C| (rel_err).  Identical when
    beta == 0.  Entries whose denominator is 0 are compared against FLT_MIN."""
    strict = rel_err(got, ref, D, None)
    return strict, (strict if beta_c is None else rel_err(got, ref, D, beta_c))


# From this depth on the stated metric is met with beta != 0 as well: the
# float32 rounding of |beta C| (at most 2^-24 |beta C|) is then far below
# 2e-6 of |alpha||A||B|, which grows with k.
STRICT_MIN_K = 256


def gate(got, ref, D, beta_c, k, tol):
    """Assert the tolerance on the metric with |beta C| in the denominator
    and, for k >= STRICT_MIN_K, on the strict metric too; returns both."""
    strict, with_beta = rel_errs(got, ref, D, beta_c)
    assert with_beta <= tol, ("gate", with_beta)
    if k >= STRICT_MIN_K:
        assert strict <= tol, ("strict gate", strict)
    return strict, with_beta
