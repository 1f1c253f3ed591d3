"""CPU oracle for Triple State QuickSort (arXiv 1505.00558) -- TEST INFRASTRUCTURE.

Only the test suite, ``__graft_entry__.smoke()`` and the CPU legs of ``bench.py``
(``cpu_baseline`` and ``--impl reference``) may import this package.  The product
path (``paper_1505_00558_gb300``) never imports it and shares no code with it.

The C source ``tsqs_oracle.c`` implements the paper's algorithm step by step
(Sections III-V); this module compiles it with gcc on first use and wraps it with
ctypes over numpy arrays.
"""
from .oracle import (  # noqa: F401
    KIND_I32, KIND_U32, KIND_F32, KIND_I64, KIND_U64, KIND_F64, KIND_REC,
    PIVOT_TIERED, PIVOT_RANDOM, STATE_NAMES,
    OracleCfg, build, lib, tsqs_sort, tsqs_sort_rows, tsqs_sort_segments,
    classical_sort, juggle_sort, median3, choose_pivot, lower_median, three_way_split, compare,
    wide_sort, std_sort_i32,
)
