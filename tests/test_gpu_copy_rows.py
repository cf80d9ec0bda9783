"""gf2x_copy_rows (the serving loop's operand staging): every entry's limbs
land at its destination, padding entries (limbs = 0) and the words around
each destination row are untouched; one launch, also captured in a graph."""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


def test_rows_copied_padding_skipped_neighbours_untouched():
    from paper_2201_10473_gb300 import Context
    ctx = Context(0)
    try:
        rng = np.random.default_rng(77)
        src = torch.from_numpy(rng.integers(0, 2**63, size=50000, dtype=np.int64)).cuda()
        dst = torch.full((60000,), -7, dtype=torch.int64, device="cuda")
        entries, expect = [], dst.clone().cpu().numpy()
        s_off = d_off = 0
        for i in range(300):
            L = int(rng.integers(1, 120))
            if i % 17 == 0:
                entries.append((0, 0, 0))                       # padding entry
                continue
            entries.append((src.data_ptr() + 8 * s_off, dst.data_ptr() + 8 * (d_off + 1), L))
            expect[d_off + 1: d_off + 1 + L] = src[s_off: s_off + L].cpu().numpy()
            s_off += L
            d_off += L + 3                                      # gaps between destination rows
        rows = torch.tensor(entries, dtype=torch.int64).cuda()
        side = torch.cuda.Stream()
        side.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(side):
            ctx.copy_rows(rows, len(entries))
        torch.cuda.current_stream().wait_stream(side)
        torch.cuda.synchronize()
        assert np.array_equal(dst.cpu().numpy(), expect)
        dst.fill_(-7)
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            ctx.copy_rows(rows, len(entries))
        g.replay()
        torch.cuda.synchronize()
        assert np.array_equal(dst.cpu().numpy(), expect)
        ctx.sync_status()
    finally:
        ctx.close()
