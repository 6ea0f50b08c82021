"""Table 3 (Sec. 3.3.1): key/payload semantics of the check-point sort.  The
fixture pins a stable key sort followed by a scatter of the payload by the
shuffled index; the GPU radix sort is checked against the same fixture in
the GPU suite."""
import numpy as np

from tests.golden_table3 import load


def test_table3_is_a_stable_key_sort():
    t = load()
    M = np.array(t["unsorted_M"])
    order = np.argsort(M, kind="stable")
    assert list(M[order]) == t["sorted_M"]
    assert list(np.array(t["unsorted_Ic"])[order]) == t["sorted_Ic"]
    assert list(np.array(t["unsorted_Icb"])[order]) == t["scatter_Icb"]
    assert list(np.array(t["unsorted_dat"])[order]) == t["scatter_dat"]
