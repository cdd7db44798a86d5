"""The row split across ranks, with its CUDA steps run on one device (GPU).

When the rows of each band are split across ranks, every rank runs pass 1 on
its own rows, the ranks sum their per-band histograms (the one exchange), and
every rank builds S from the sum and runs pass 2 on its own rows.  The
multi-rank host tests cover that flow with the oracle in place of the device
steps; here the device steps themselves (``sharded._cuda_steps``: lutc_hist,
lutc_stretch, lutc_apply_stretch) run for two row ranges on one GPU, the test
sums the two histograms where the all-reduce would (through the same int64
view of the uint64 counts that the all-reduce uses), and the stacked result
must equal the oracle's correction of the whole raster, element by element.
"""
import numpy as np
import pytest
import torch

import oracle
import synth
from paper_1505_05655_gb300 import sharded

pytestmark = pytest.mark.gpu

import paper_1505_05655_gb300 as lutc  # noqa: E402


def _d(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.mark.parametrize("bands,h,w,bits,world,pad", [
    (3, 517, 2304, 14, 2, 0),    # 14-bit, aligned rows: TMA-staged kernels on both ranks
    (2, 301, 1001, 12, 2, 0),    # odd width: strip kernels
    (1, 64, 1024, 16, 3, 0),     # 16-bit (histogram in global memory), three ranks
    (4, 9, 768, 10, 4, 8),       # a rank of two rows, pitched rows
    (1, 5, 300, 12, 7, 0),       # more ranks than some ranks have rows: empty slices
])
def test_row_split_device_steps_equal_whole_raster(bands, h, w, bits, world, pad):
    raw = synth.raster(8800 + h, bands, h, w, bits, dead_frac=0.01, sat_frac=0.001)
    A, G, O = synth.coeff_set(8800 + h, bands, w)
    dA, dG, dO = _d(A), _d(G), _d(O)
    hist, stretch, apply = sharded._cuda_steps()
    ranges = [sharded.row_range(h, world, r) for r in range(world)]
    parts = []
    for r0, r1 in ranges:
        rows = np.zeros((bands, r1 - r0, w + pad), np.uint16)
        rows[:, :, :w] = raw[:, r0:r1]
        parts.append(_d(rows)[:, :, :w])  # each rank holds its own rows, in its own (pitched) buffer
    # pass 1 on every rank, then the exchange: a sum of the counts viewed as int64
    counts = [hist(p, dA, dG, dO, bits) for p in parts]
    tma = (2 * (w + pad)) % 16 == 0 and w >= 256
    from paper_1505_05655_gb300._lib import LUTC_PATH_STRIP, LUTC_PATH_TMA
    assert lutc.last_path() == (LUTC_PATH_TMA if tma else LUTC_PATH_STRIP)
    assert all(c.dtype == torch.uint64 and c.shape == (bands, 1 << bits) for c in counts)
    total = counts[0].view(torch.int64).clone()
    for c in counts[1:]:
        total += c.view(torch.int64)
    ref, (ref_hist, ref_S, ref_lohi) = oracle.correct_image(raw, A, G, O, bits, stretch=True, with_tables=True)
    np.testing.assert_array_equal(total.cpu().numpy(), ref_hist.astype(np.int64))
    # every rank builds S from the summed counts and corrects its own rows
    S = stretch(total.view(torch.uint64), bits)
    np.testing.assert_array_equal(S.cpu().numpy(), ref_S)
    outs = [apply(p, dA, dG, dO, bits, S) for p in parts]
    got = torch.cat([o.reshape(bands, -1, w) for o in outs], dim=1).cpu().numpy()
    np.testing.assert_array_equal(got, ref)
    # without the exchange a rank's own counts give another S (the exchange is needed)
    if world == 2 and h > 100:
        alone = stretch(counts[0], bits)
        assert not torch.equal(alone, S)


def test_correct_rows_without_a_process_group_is_the_single_device_correction():
    # with no process group (one rank), correct_rows on all rows is lutc_correct_image
    bands, h, w, bits = 2, 200, 1536, 12
    raw = synth.raster(8900, bands, h, w, bits)
    A, G, O = synth.coeff_set(8900, bands, w)
    got = sharded.correct_rows(_d(raw), _d(A), _d(G), _d(O), bits)
    np.testing.assert_array_equal(got.cpu().numpy(), oracle.correct_image(raw, A, G, O, bits, stretch=True))
