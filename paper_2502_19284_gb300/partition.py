"""Row partition of one product over several GPUs (host logic; no GPU work here).

A row-partitioned y = A x: rank g of G holds the rows [r_g, r_g+1) of A and the whole x, forms
its slice of y with any of the library's products, and one all-gather of the slices gives y
(the next x in iterative use).  The cut points are the merge-path split of Section 3.3 (the
path of row ends and nonzero indices cut into equal lengths) taken at GPU granularity: the
cut on diagonal d = g (m + nnz) / G falls after the largest number i of row ends with
row_ptr[i] <= d - i (on a tie the row end is consumed first, as in the merge-path figure), so
every rank's rows plus nonzeros are within one row of the mean.  A row never spans two ranks,
so the products need no exchange of partial sums.
"""
from __future__ import annotations

import numpy as np


def row_ranges(row_ptr, parts: int) -> np.ndarray:
    """First row of every part (parts + 1 entries, the last = m) for a CRS row_ptr."""
    rp = np.asarray(row_ptr, dtype=np.int64)
    m = rp.size - 1
    nnz = int(rp[-1]) if m >= 0 else 0
    if parts < 1:
        raise ValueError("parts must be >= 1")
    cuts = np.empty(parts + 1, dtype=np.int64)
    for g in range(parts + 1):
        d = g * (m + nnz) // parts
        lo, hi = max(0, d - nnz), min(d, m)
        while lo < hi:                       # largest i with row_ptr[i] <= d - i
            mid = (lo + hi + 1) // 2
            if rp[mid] <= d - mid:
                lo = mid
            else:
                hi = mid - 1
        cuts[g] = lo
    cuts[0], cuts[-1] = 0, m
    return cuts


def local_rows(row_ptr, col, val, r0: int, r1: int):
    """The CRS arrays of rows [r0, r1) with row_ptr rebased to 0 (columns stay global)."""
    rp = np.asarray(row_ptr, dtype=np.int64)
    k0, k1 = int(rp[r0]), int(rp[r1])
    lrp = (rp[r0:r1 + 1] - k0).astype(np.int32)
    return lrp, np.asarray(col)[k0:k1], None if val is None else np.asarray(val)[k0:k1]


def gather_y(dist, y_local, cuts, device="cpu"):
    """All-gather of the ranks' y slices into the full y (torch.distributed; slices padded to
    the longest so that every rank sends the same count)."""
    import torch
    world = len(cuts) - 1
    lens = np.diff(cuts)
    width = int(lens.max()) if world else 0
    buf = torch.zeros(width, dtype=torch.float64, device=device)
    yl = torch.as_tensor(np.asarray(y_local), dtype=torch.float64, device=device)
    buf[: yl.numel()] = yl
    out = [torch.empty(width, dtype=torch.float64, device=device) for _ in range(world)]
    dist.all_gather(out, buf)
    return torch.cat([o[: int(n)] for o, n in zip(out, lens)]).cpu().numpy()
