"""Work partitioning of the blocked GEMM over several GPUs (host logic only).

Every output tile of C := beta*C + alpha*A*B is independent (the blocked
algorithms of the paper's Section 3 parallelise over the ic/jc loops; only
the pc loop carries a reduction), so the path shards with no exchange step:

* one large problem: a 2-D block partition of C over a pr x pc grid of ranks;
  rank (r, c) computes rows R_r and columns C_c of C from rows R_r of A and
  columns C_c of B.  Block edges are multiples of the 128-wide tile so that no
  tile straddles two ranks.
* many problems (grouped): whole problems go to ranks, largest first, each to
  the least-loaded rank (longest-processing-time order on 2mnk).

A split of k across ranks would need a reduction (a collective); it is never
chosen here.
"""
from __future__ import annotations

from dataclasses import dataclass

TILE = 128


@dataclass(frozen=True)
class Block:
    rank: int
    row0: int
    row1: int   # exclusive
    col0: int
    col1: int   # exclusive

    @property
    def empty(self) -> bool:
        return self.row1 <= self.row0 or self.col1 <= self.col0


def grid_shape(m: int, n: int, world: int):
    """(pr, pc) with pr * pc == world whose blocks are closest to square."""
    best = None
    for pr in range(1, world + 1):
        if world % pr:
            continue
        pc = world // pr
        rows, cols = -(-m // pr), -(-n // pc)
        score = max(rows, cols) / max(1, min(rows, cols))
        if best is None or score < best[0]:
            best = (score, pr, pc)
    return best[1], best[2]


def _cuts(extent: int, parts: int, align: int = TILE):
    """parts + 1 cut points over [0, extent], interior cuts on multiples of align."""
    units = -(-extent // align)
    cuts = [0]
    for p in range(1, parts):
        cuts.append(min(extent, ((units * p) // parts) * align))
    cuts.append(extent)
    return cuts


def partition_2d(m: int, n: int, world: int):
    """One Block per rank covering C exactly once (some may be empty)."""
    if world < 1:
        raise ValueError("world must be >= 1")
    pr, pc = grid_shape(m, n, world)
    rc, cc = _cuts(m, pr), _cuts(n, pc)
    out = []
    for r in range(pr):
        for c in range(pc):
            out.append(Block(r * pc + c, rc[r], rc[r + 1], cc[c], cc[c + 1]))
    return out


def assign_problems(shapes, world: int):
    """Indices of the problems each rank runs: LPT on 2mnk, deterministic ties."""
    load = [0.0] * world
    owned = [[] for _ in range(world)]
    order = sorted(range(len(shapes)), key=lambda i: (-2.0 * shapes[i][0] * shapes[i][1] * shapes[i][2], i))
    for i in order:
        r = min(range(world), key=lambda q: (load[q], q))
        owned[r].append(i)
        m, n, k = shapes[i]
        load[r] += 2.0 * m * n * k
    return [sorted(o) for o in owned]
