"""One band (or several) split by rows across the ranks of a process group.

Pass 1 and pass 2 work on each rank's own rows; the stretch needs the whole
band's histogram, so the one exchange is a sum of the per-band histograms
(2^bits counts per band) between the passes.  Every other step stays local.
With NCCL each rank's rows, histogram and output live on its GPU.
"""
from __future__ import annotations

import torch
import torch.distributed as dist


def row_range(height: int, world: int, rank: int) -> tuple[int, int]:
    """Rows [r0, r1) of `rank` when `height` rows are split as evenly as possible over `world` ranks."""
    if world < 1 or not 0 <= rank < world or height < 0:
        raise ValueError("bad split")
    return height * rank // world, height * (rank + 1) // world


def _cuda_steps():
    import paper_1505_05655_gb300 as lutc

    def hist(raw, A, G, O, bits):
        return lutc.hist(raw, A, G, O, bits)

    def stretch(h, bits):
        return lutc.stretch(h, bits)[0]

    def apply(raw, A, G, O, bits, S):
        return lutc.apply_stretch(raw, A, G, O, bits, S)

    return hist, stretch, apply


def correct_rows(raw_rows: torch.Tensor, A: torch.Tensor, G: torch.Tensor, O: torch.Tensor, bits: int,
                 group=None, steps=None) -> torch.Tensor:
    """The fused correction of this rank's rows ``[bands, rows, W]`` of bands split across `group`.

    Equal, row for row, to correcting the whole bands on one device.  `steps` = (hist, stretch, apply)
    replaces the library's entry points (the host-side tests run them on the CPU oracle).
    """
    hist, stretch, apply = steps if steps is not None else _cuda_steps()
    h = hist(raw_rows, A, G, O, bits)                    # [bands, 2^bits] counts of this rank's rows
    counts = h.view(torch.int64) if h.dtype == torch.uint64 else h
    if dist.is_available() and dist.is_initialized() and dist.get_world_size(group) > 1:
        dist.all_reduce(counts, op=dist.ReduceOp.SUM, group=group)
    S = stretch(counts.view(h.dtype), bits)
    return apply(raw_rows, A, G, O, bits, S)
