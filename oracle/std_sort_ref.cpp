// std_sort_ref.cpp -- the C++ standard library's sort, timed beside the oracle as a
// second CPU reference (TEST INFRASTRUCTURE, like the oracle itself: only the test
// suite and the CPU legs of bench.py load it; it checks nothing and is only timed).
#include <algorithm>
#include <cstddef>
#include <cstdint>

extern "C" void orc_std_sort_i32(int32_t *a, size_t n) { std::sort(a, a + n); }
