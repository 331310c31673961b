"""Frequency sharding across ranks (one process per GPU, no collective on the data path).

Frequencies are independent, so a sweep is weak-scaled by giving each rank its own
batches of the frequency grid: step s of rank r takes the batch
[(s * world + r) * B, (s * world + r + 1) * B) of the grid, wrapping around its end.
Within a step the ranks' batches are disjoint as long as world * B <= len(grid).
"""
import numpy as np


def batch_indices(n_freqs: int, batch: int, world: int, rank: int, step: int) -> np.ndarray:
    """Grid indices of rank `rank`'s batch in step `step`."""
    if not (n_freqs > 0 and batch > 0 and 0 <= rank < world):
        raise ValueError("bad sharding arguments")
    return (np.arange(batch) + (step * world + rank) * batch) % n_freqs
