"""Break-even count of a storage-format conversion (Section 6.2 and the conclusion).

The paper quotes how many SpMV multiplications pay back converting to a blocked format
instead of CRS, without stating the formula.  The count that reproduces its quoted
numbers from its own tables is

    N* = (C_fmt - C_CRS) / (1 - S_CRS / S_fmt)

with C the mean conversion cost in units of one parallel CRS multiplication and S the mean
parallel speedup.  On measured times (one GPU) the same quantity is

    N*_GPU = (T_to_fmt - T_to_CRS) / (T_spmv_CRS - T_spmv_fmt),

the extra conversion time divided by the time saved per multiplication; it is None
("never") when the blocked product is not faster.
"""
from __future__ import annotations


def n_star_relative(conv_fmt: float, conv_crs: float, speedup_crs: float, speedup_fmt: float):
    """N* from the paper's relative units (conversion in CRS SpMVs, mean speedups)."""
    if speedup_fmt <= speedup_crs:
        return None
    return (conv_fmt - conv_crs) / (1.0 - speedup_crs / speedup_fmt)


def n_star_times(t_to_fmt: float, t_to_crs: float, t_spmv_crs: float, t_spmv_fmt: float):
    """N* from measured times (any one unit)."""
    saved = t_spmv_crs - t_spmv_fmt
    if saved <= 0:
        return None
    return max(0.0, t_to_fmt - t_to_crs) / saved
