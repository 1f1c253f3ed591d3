"""Seeded synthetic inputs shaped like the paper's test patterns.

This package holds input generation only -- no sorting, partitioning or pivot
arithmetic -- so both the CPU oracle's tests and the CUDA path's tests and bench
can use it without sharing any of the method's code.
"""
from .patterns import (  # noqa: F401
    PATTERNS, splitmix64, rand_u64, int32_pattern, records_u64, floats_normal_specials,
    batched_segments, serving_requests, total_order_key_f32, total_order_key_f64,
)
