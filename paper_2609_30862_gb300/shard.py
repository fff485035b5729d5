"""Host side of one instance sharded over ranks by chromosome rows.

Each rank owns a contiguous block of rows; a generation's QIP and Evaluation are local
(every draw is keyed by the global chromosome index, so a row's alleles do not depend on
where it lives), and the only exchange per generation is DetermineElite (paper Sec. III-B:
the elite is the generation's best chromosome, lowest index on ties) followed by CIP toward
the elite's alleles, which every rank needs:

  1. an all-reduce MAX of a 64-bit key that orders (fitness, -global index)
     lexicographically: f * 2^32 + (2^32 - 1 - c) for fitness in [-2^31, 2^31); wider
     fitness takes two reductions (MAX of f, then MIN of c among the ranks holding it).
     Which form is used is decided once, from the problem's bounds, identically on every
     rank (key_is_wide), so no rank can meet a fitness its form cannot carry;
  2. a broadcast of the elite's alleles (ng bytes) from the rank that owns the row.

The per-rank compute is passed in (a callable per step), so this module holds no QIEO
arithmetic and works with any backend of torch.distributed.
"""
from __future__ import annotations

import numpy as np

KEY_F_MIN = -(1 << 31)
KEY_F_MAX = (1 << 31) - 1


def row_range(np_: int, world: int, rank: int) -> tuple[int, int]:
    """Rows [r0, r1) of `rank`: contiguous blocks, the first np % world ranks one row more."""
    base, extra = divmod(np_, world)
    r0 = rank * base + min(rank, extra)
    return r0, r0 + base + (1 if rank < extra else 0)


def owner_of(c: int, np_: int, world: int) -> int:
    """Rank whose block holds global row c."""
    for r in range(world):
        r0, r1 = row_range(np_, world, r)
        if r0 <= c < r1:
            return r
    raise ValueError("row %d outside [0, %d)" % (c, np_))


def pack_key(f: int, c: int) -> int:
    """(fitness, -index) as one signed 64-bit integer; larger key = better elite."""
    if not (KEY_F_MIN <= f <= KEY_F_MAX) or not (0 <= c <= 0xFFFFFFFF):
        raise ValueError("fitness or index out of the packed key's range")
    return f * (1 << 32) + (0xFFFFFFFF - c)


def unpack_key(key: int) -> tuple[int, int]:
    f, low = divmod(key, 1 << 32)
    return f, 0xFFFFFFFF - low


def key_is_wide(weights, values, lam: int = 1) -> bool:
    """True when a fitness of this problem can leave the packed key's range: eq. (1) gives
    f = sum(v x) <= sum(|v|) for a feasible chromosome and f = -lam (sum(w x) - W) >=
    -lam sum(w) for an infeasible one (W >= 0)."""
    sw = int(np.sum(np.asarray(weights, dtype=np.int64)))
    sv = int(np.sum(np.abs(np.asarray(values, dtype=np.int64))))
    return int(lam) * sw > -KEY_F_MIN or sv > KEY_F_MAX


def local_elite(f_local: np.ndarray, r0: int) -> tuple[int, int]:
    """Lowest-index maximum of this rank's fitness values, as (fitness, global index);
    (None, None) for an empty block."""
    if f_local.size == 0:
        return None, None
    i = int(np.argmax(f_local))            # numpy returns the first maximum
    return int(f_local[i]), r0 + i


class EliteExchange:
    """DetermineElite across ranks: one collective for the key, one broadcast for the row.

    The key form follows from the problem (key_is_wide), the same on every rank; `wide`
    overrides it (True always works; False only for problems whose fitness fits)."""

    def __init__(self, np_: int, ng: int, problem=None, lam: int = 1, group=None, wide=None):
        import torch
        import torch.distributed as dist
        if wide is None:
            if problem is None:
                raise ValueError("EliteExchange needs the problem (or an explicit key form)")
            wide = key_is_wide(problem.weights, problem.values, lam)
        elif not wide and problem is not None and key_is_wide(problem.weights, problem.values, lam):
            raise ValueError("this problem's fitness does not fit the packed key: use wide=True")
        self.torch, self.dist = torch, dist
        self.np, self.ng, self.group, self.wide = np_, ng, group, bool(wide)
        self.world = dist.get_world_size(group)
        self.rank = dist.get_rank(group)

    def __call__(self, f_best, c_best, rows: dict) -> tuple[int, int, np.ndarray]:
        """f_best, c_best: this rank's local elite (None when it has no rows); rows maps a
        global row index to its alleles (only the local elite's row is read). Returns
        (elite fitness, elite global index, elite alleles) on every rank."""
        torch, dist = self.torch, self.dist
        if not self.wide:
            lo = torch.iinfo(torch.int64).min
            key = torch.tensor([lo if f_best is None else pack_key(f_best, c_best)], dtype=torch.int64)
            dist.all_reduce(key, op=dist.ReduceOp.MAX, group=self.group)
            f_e, c_e = unpack_key(int(key[0]))
        else:
            lo = torch.iinfo(torch.int64).min
            fv = torch.tensor([lo if f_best is None else int(f_best)], dtype=torch.int64)
            dist.all_reduce(fv, op=dist.ReduceOp.MAX, group=self.group)
            f_e = int(fv[0])
            cv = torch.tensor([c_best if (f_best is not None and f_best == f_e) else self.np],
                              dtype=torch.int64)
            dist.all_reduce(cv, op=dist.ReduceOp.MIN, group=self.group)
            c_e = int(cv[0])
        src = owner_of(c_e, self.np, self.world)
        buf = torch.zeros(self.ng, dtype=torch.uint8)
        if self.rank == src:
            buf.copy_(torch.from_numpy(np.ascontiguousarray(rows[c_e], dtype=np.uint8)))
        dist.broadcast(buf, src=dist.get_global_rank(self.group, src) if self.group is not None else src,
                       group=self.group)
        return f_e, c_e, buf.numpy().copy()


class _RowOnDemand(dict):
    """The local best row, fetched only if the exchange reads it (on the owning rank)."""

    def __init__(self, c, fetch):
        super().__init__()
        self.c, self.fetch = c, fetch

    def __getitem__(self, c):
        if c != self.c:
            raise KeyError(c)
        return self.fetch(c)


def run_sharded_blocks(gens: int, observe_best, row_of, rotate_rows, exchange, t0: int = 0):
    """Runs `gens` generations of one sharded instance from generation t0, with the local
    DetermineElite done by the rank's own compute.

    observe_best(t) -> (f_best, c_best): QIP + Evaluation of this rank's rows and their
        lowest-index best (c_best a global index), or (None, None) for an empty block.
    row_of(c) -> alleles (ng) of this rank's row c; called only on the rank that holds the
        population's elite.
    rotate_rows(x_elite): CIP of this rank's rows toward the elite's alleles.
    exchange: an EliteExchange (or any callable with its signature).
    Returns (hist_e, hist_f, best) where best = (fitness, generation, chromosome, alleles),
    the best-so-far record replaced only by a strictly larger fitness (ties keep the
    earliest generation)."""
    hist_e = np.zeros(gens, dtype=np.int32)
    hist_f = np.zeros(gens, dtype=np.int64)
    best = (None, -1, -1, None)
    for g in range(gens):
        t = t0 + g
        f_b, c_b = observe_best(t)
        rows = {} if c_b is None else _RowOnDemand(c_b, row_of)
        f_e, c_e, x_e = exchange(f_b, c_b, rows)
        hist_e[g], hist_f[g] = c_e, f_e
        if best[1] < 0 or f_e > best[0]:
            best = (f_e, t, c_e, x_e)
        rotate_rows(x_e)
    return hist_e, hist_f, best


def run_sharded(np_: int, ng: int, gens: int, observe_rows, rotate_rows, exchange,
                r0: int, t0: int = 0):
    """run_sharded_blocks for a rank whose compute returns all its rows:
    observe_rows(t) -> (f_local[nr], x_local[nr, ng]); the local DetermineElite is done here."""
    last = {}

    def observe_best(t):
        f_loc, x_loc = observe_rows(t)
        last["x"] = x_loc
        return local_elite(f_loc, r0)

    return run_sharded_blocks(gens, observe_best, lambda c: last["x"][c - r0], rotate_rows,
                              exchange, t0)
