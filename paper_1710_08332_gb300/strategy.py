"""Reduction strategy descriptor (mirror of ``dpia_reduce_strategy``).

A strategy spells out the paper's strategy annotations (Section 2.1: split
sizes, which hierarchy level runs each map, which reduce is sequential) as
plain fields; see include/dpia.h for the meaning of each field.
"""
from __future__ import annotations

from dataclasses import asdict, dataclass, replace

from . import _native as N

LEVELS = {"grid": N.LVL_GRID, "block": N.LVL_BLOCK, "warp": N.LVL_WARP, "thread": N.LVL_THREAD,
          "seq": N.LVL_SEQ}


@dataclass(frozen=True)
class ReduceStrategy:
    split: int
    threads: int = 256
    vec: int = 4
    map_level: str = "block"
    inner_level: str = "thread"
    thread_map: str = "interleaved"
    second: str = "seq"
    threads2: int = 32
    compensated: bool = False
    pad: bool = False
    grid: int = 0
    stage: str = "private"   # "private" (registers) or "local" (shared memory, bulk copies)

    def to_c(self) -> N.ReduceStrategyC:
        return N.ReduceStrategyC(
            int(self.split), int(self.threads), int(self.vec), LEVELS[self.map_level],
            LEVELS[self.inner_level],
            N.MAP_INTERLEAVED if self.thread_map == "interleaved" else N.MAP_CONTIG,
            N.SECOND_TREE if self.second == "tree" else N.SECOND_SEQ, int(self.threads2),
            int(bool(self.compensated)), int(bool(self.pad)), int(self.grid),
            N.STAGE_LOCAL if self.stage == "local" else N.STAGE_PRIVATE)

    @property
    def chunk_threads(self) -> int:
        """Threads that cooperate on one chunk (the value-defining T)."""
        return {"block": self.threads, "warp": 32, "grid": 1}[self.map_level]

    def with_(self, **kw) -> "ReduceStrategy":
        return replace(self, **kw)

    def as_dict(self):
        return asdict(self)


def default_dot_strategy(n: int) -> ReduceStrategy:
    """A coalesced block-per-chunk strategy with a tree second level."""
    s = 8192 if n >= 8192 else max(1024, 1 << max(n - 1, 1).bit_length())
    return ReduceStrategy(split=s, threads=256, vec=4, second="tree", threads2=256, pad=n % s != 0)
