"""Seeded synthetic inputs shared by the tests, the smoke check and the benchmark.

This module draws random numbers and nothing else: it holds none of the GEMM's
arithmetic (no rounding, quantisation, scaling of results or products), so the
oracle and the GPU path can both be fed from it without sharing any code.

Every generator uses ``numpy.random.default_rng(seed)`` and draws A, then B,
then C, as float32 (or int8 / int32), so that one seed fixes one problem.
The shapes follow the paper's two workload families: large squares and the
im2col GEMMs of the ResNet50 v1.5 convolution layers (Table 1).
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

# Table 1: GEMM dimensions of the ResNet50 v1.5 convolution layers after the
# im2col transform, batch 128, as (layer type, m = batch*Hout*Wout, n = Cout,
# k = Cin*kh*kw).  The library computes C (Cout x pixels) = W (Cout x k) * X
# (k x pixels), i.e. the transposed problem, so a layer at batch b becomes
# m = Cout, n = (m_table / 128) * b, k.
RESNET50_TABLE1 = (
    (1, 1605632, 64, 147), (2, 401408, 64, 64), (3, 401408, 64, 576),
    (4, 401408, 256, 64), (5, 401408, 64, 256), (6, 401408, 128, 256),
    (7, 100352, 128, 1152), (8, 100352, 512, 128), (9, 100352, 512, 256),
    (10, 100352, 128, 512), (11, 100352, 256, 512), (12, 25088, 256, 2304),
    (13, 25088, 1024, 256), (14, 25088, 1024, 512), (15, 25088, 256, 1024),
    (16, 25088, 512, 1024), (17, 6272, 512, 4608), (18, 6272, 2048, 512),
    (19, 6272, 2048, 1024), (20, 6272, 512, 2048),
)

# The convolution behind each Table 1 layer (ResNet-50 v1.5, square inputs):
# input size H (= W), input channels C, output channels K, filter R x R,
# stride, padding.  Table 1 fixes m / 128 = Hout^2, n = K and k = C R^2; the
# input size and stride follow from where the layer sits in the network (the
# stride-2 3x3 convolutions and 1x1 downsampling projections halve the size).
RESNET50_CONV = tuple(dict(layer=l, H=h, C=c, K=kk, R=r, stride=st, pad=pd) for (l, h, c, kk, r, st, pd) in (
    (1, 224, 3, 64, 7, 2, 3), (2, 56, 64, 64, 1, 1, 0), (3, 56, 64, 64, 3, 1, 1),
    (4, 56, 64, 256, 1, 1, 0), (5, 56, 256, 64, 1, 1, 0), (6, 56, 256, 128, 1, 1, 0),
    (7, 56, 128, 128, 3, 2, 1), (8, 28, 128, 512, 1, 1, 0), (9, 56, 256, 512, 1, 2, 0),
    (10, 28, 512, 128, 1, 1, 0), (11, 28, 512, 256, 1, 1, 0), (12, 28, 256, 256, 3, 2, 1),
    (13, 14, 256, 1024, 1, 1, 0), (14, 28, 512, 1024, 1, 2, 0), (15, 14, 1024, 256, 1, 1, 0),
    (16, 14, 1024, 512, 1, 1, 0), (17, 14, 512, 512, 3, 2, 1), (18, 7, 512, 2048, 1, 1, 0),
    (19, 14, 1024, 2048, 1, 2, 0), (20, 7, 2048, 512, 1, 1, 0)))

# Three batch-1 layers used as named examples of the convolution workload.
IM2COL_BATCH1_EXAMPLES = ((64, 12544, 147), (256, 3136, 576), (2048, 49, 1024))

SQUARE_SWEEP = (1024, 2048, 4096, 8192, 16384)


def im2col_shapes(batch: int = 16):
    """(layer, m=Cout, n=batch*Hout*Wout, k) for the 20 layer types."""
    out = []
    for layer, m_t, n_t, k_t in RESNET50_TABLE1:
        out.append((layer, n_t, (m_t // 128) * batch, k_t))
    return out


@dataclass
class Problem:
    m: int
    n: int
    k: int
    alpha: float
    beta: float
    A: np.ndarray
    B: np.ndarray
    C: np.ndarray | None


def uniform_problem(m, n, k, seed=0, alpha=1.0, beta=0.0, with_c=None):
    """A, B (and C when beta != 0) i.i.d. uniform in [-1, 1], float32."""
    rng = np.random.default_rng(seed)
    A = rng.uniform(-1.0, 1.0, size=(m, k)).astype(np.float32)
    B = rng.uniform(-1.0, 1.0, size=(k, n)).astype(np.float32)
    need_c = (beta != 0.0) if with_c is None else with_c
    C = rng.uniform(-1.0, 1.0, size=(m, n)).astype(np.float32) if need_c else None
    return Problem(m, n, k, alpha, beta, A, B, C)


def normal_problem(m, n, k, seed=0, alpha=1.0, beta=0.0):
    """Convolution-like inputs: weights A ~ N(0,1)/sqrt(k), activations B ~ N(0,1)."""
    rng = np.random.default_rng(seed)
    A = (rng.standard_normal(size=(m, k)) / math.sqrt(max(k, 1))).astype(np.float32)
    B = rng.standard_normal(size=(k, n)).astype(np.float32)
    C = rng.standard_normal(size=(m, n)).astype(np.float32) if beta != 0.0 else None
    return Problem(m, n, k, alpha, beta, A, B, C)


def int8_problem(m, n, k, seed=0, beta=0):
    """A, B uniform integers in [-128, 127]; C int32 when beta != 0."""
    rng = np.random.default_rng(seed)
    A = rng.integers(-128, 128, size=(m, k), dtype=np.int64).astype(np.int8)
    B = rng.integers(-128, 128, size=(k, n), dtype=np.int64).astype(np.int8)
    C = (rng.integers(-(1 << 20), 1 << 20, size=(m, n), dtype=np.int64).astype(np.int32)
         if beta != 0 else None)
    return Problem(m, n, k, 1.0, float(beta), A, B, C)


def small_int_problem(m, n, k, seed=0, lo=-8, hi=8, alpha=1.0, beta=0.0):
    """Integer-valued float32 inputs in [lo, hi]: exact in bfloat16, and every
    partial sum exact in float32 while k*hi*hi < 2^24."""
    rng = np.random.default_rng(seed)
    A = rng.integers(lo, hi + 1, size=(m, k)).astype(np.float32)
    B = rng.integers(lo, hi + 1, size=(k, n)).astype(np.float32)
    C = rng.integers(lo, hi + 1, size=(m, n)).astype(np.float32) if beta != 0.0 else None
    return Problem(m, n, k, alpha, beta, A, B, C)


def grouped_shapes(count=1000, seed=0, lo=16, hi=1024):
    """(m, n, k) per group, each log-uniform in [lo, hi], drawn m, n, k in turn."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(count):
        dims = []
        for _d in range(3):
            dims.append(int(round(math.exp(rng.uniform(math.log(lo), math.log(hi))))))
        out.append(tuple(dims))
    return out
