"""One solve split over devices by island (Section IV-B, the island model).

The solution pools are the islands: search s breeds its target from island
s mod P (and, for Xrossover, from island (s mod P) + 1 mod P).  A solve of
P islands on R ranks gives rank r the searches of islands
[r P / R, (r + 1) P / R); every generation each rank

  1. breeds all S targets from its copy of the pools (stage 0: cheap, and
     identical on every rank),
  2. runs the batch searches of its own islands only (stage 1),
  3. exchanges the results: every rank contributes its searches' (BEST,
     E(BEST), flips) and receives everyone else's (one all-gather),
  4. merges all S results in search order into its copy of the pools and
     finalises (stages 2 and 3: identical on every rank).

So every rank keeps the same pools, global best and statistics, and the solve
equals the solve of all P islands on one device (same seed, budget, target),
bit for bit: a search's results depend only on its index s and on the pools
of the previous generation.  The exchange carries S results per generation
(S x (4 words(n) + 12) bytes); with R ranks each runs S/R searches.

`IslandSolve` drives one rank through an engine with the stages above (the
CUDA library's context: `ContextEngine`) and a `gather` callable that returns
every rank's contribution in rank order (`torch.distributed.all_gather_object`
for a process group; an in-process list for ranks driven from one process).
"""
from __future__ import annotations

import numpy as np


def island_range(P: int, ranks: int, rank: int):
    """Islands [lo, hi) of one rank: a contiguous block, the first P mod R ranks
    holding one more."""
    if not (1 <= ranks <= P) or not (0 <= rank < ranks):
        raise ValueError("need 1 <= ranks <= islands and 0 <= rank < ranks")
    base, extra = divmod(P, ranks)
    lo = rank * base + min(rank, extra)
    return lo, lo + base + (1 if rank < extra else 0)


def search_slots(S: int, P: int, lo: int, hi: int) -> np.ndarray:
    """The searches s < S of islands [lo, hi): lo <= s mod P < hi."""
    s = np.arange(S)
    return s[(s % P >= lo) & (s % P < hi)]


class ContextEngine:
    """The stages of one generation on a `dabs.Context`, its searches restricted
    to one rank's islands."""

    def __init__(self, ctx, lo: int, hi: int):
        from paper_2207_03069_gb300 import dabs
        self.dabs = dabs
        self.ctx = ctx
        self.S, self.P = ctx.S, ctx.P
        ctx.set_search_slots(self.P, lo, hi)

    def begin(self, seed, budget, target):
        self.ctx.solve_begin(seed, budget=budget, target=target)

    def search(self):
        self.ctx.run_stage(self.dabs.STAGE_OFFSPRING)
        self.ctx.run_stage(self.dabs.STAGE_SEARCH)

    def results(self):
        """(best_X words [S][w], best_E [S], flips [S], algo [S], op [S]) of every slot
        (valid for this rank's slots)."""
        D, a, o, bX, bE, f = self.ctx.read_generation()
        return bX, bE, f, a, o

    def merge(self, bX, bE, f, a, o):
        self.ctx.write_results(bX, bE, f, a, o)
        self.ctx.run_stage(self.dabs.STAGE_MERGE)
        self.ctx.run_stage(self.dabs.STAGE_FINALIZE)

    def status(self):
        return self.ctx.solve_status()

    def best(self):
        return self.ctx.solve_best()

    def close(self):
        self.ctx.set_search_slots(0)


class IslandSolve:
    """One rank of a solve split by island.  `gather(obj)` must return the list
    of every rank's `obj` in rank order."""

    def __init__(self, engine, rank: int, ranks: int, gather):
        self.engine, self.rank, self.ranks, self.gather = engine, rank, ranks, gather
        self.lo, self.hi = island_range(engine.P, ranks, rank)
        self.slots = search_slots(engine.S, engine.P, self.lo, self.hi)

    def begin(self, seed: int, budget: int = 2**64 - 1, target: int | None = None):
        self.engine.begin(seed, budget, target)

    def search_part(self):
        """Stages 0 and 1; returns this rank's contribution to the exchange."""
        self.engine.search()
        bX, bE, f, a, o = self.engine.results()
        s = self.slots
        return (self.rank, s, bX[s], bE[s], f[s])

    def merge_part(self, parts):
        """Stages 2 and 3 on the results of every rank (a list of search_part
        outputs, any order); returns True once the solve has stopped."""
        bX, bE, f, a, o = self.engine.results()  # algo/op: bred here from the same pools
        bX, bE, f = bX.copy(), bE.copy(), f.copy()
        seen = np.zeros(len(bE), bool)
        for _, s, px, pe, pf in parts:
            bX[s], bE[s], f[s] = px, pe, pf
            seen[s] = True
        if not seen.all():
            raise RuntimeError("the exchange did not cover every search")
        self.engine.merge(bX, bE, f, a, o)
        return bool(self.engine.status()["done"])

    def generation(self) -> bool:
        return self.merge_part(self.gather(self.search_part()))

    def solve(self, budget: int, seed: int, target: int | None = None, max_generations=None):
        self.begin(seed, budget, target)
        g = 0
        while not self.generation():
            g += 1
            if max_generations is not None and g >= max_generations:
                break
        X, E = self.engine.best()
        return X, E, self.engine.status()["flips"]


def torch_gather(group=None):
    """all_gather_object over a torch.distributed process group."""
    import torch.distributed as dist

    def gather(obj):
        out = [None] * dist.get_world_size(group)
        dist.all_gather_object(out, obj, group=group)
        return out
    return gather
