"""Partition of independent subcarriers over ranks (one process per GPU).

OCD detection is independent per subcarrier (Section IV: subcarriers are
interleaved through one pipeline because nothing couples them), so ranks
take disjoint contiguous blocks and exchange nothing.
"""
from __future__ import annotations


def shard_range(n: int, rank: int, world: int) -> tuple[int, int]:
    """Contiguous block [start, stop) of n units for `rank` out of `world`;
    block sizes differ by at most one."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError(f"bad rank {rank} / world {world}")
    if n < 0:
        raise ValueError("n must be >= 0")
    q, rem = divmod(n, world)
    start = rank * q + min(rank, rem)
    return start, start + q + (1 if rank < rem else 0)
