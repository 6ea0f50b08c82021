"""Reader of the Table 3 fixture (test infrastructure)."""
import os


def load():
    rows = {}
    with open(os.path.join(os.path.dirname(__file__), "golden", "table3_sort.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            k, *v = line.split()
            rows[k] = v
    out = {k: v for k, v in rows.items()}
    for k in ("unsorted_M", "sorted_M"):
        out[k] = [int(x, 2) for x in rows[k]]
    for k in ("unsorted_Ic", "unsorted_Icb", "sorted_Ic", "scatter_Icb"):
        out[k] = [int(x) for x in rows[k]]
    return out
