"""Host logic of the leaf-size autotuner: bins and table lookup."""
import numpy as np

from paper_2502_01496_gb300 import autotune


def test_bins_cover_the_ranges():
    te, ne = autotune.THETA_EDGES, autotune.N_EDGES
    assert autotune._bin(0.0, te) == 0 and autotune._bin(1.0, te) == len(te) - 2
    assert autotune._bin(0.39, te) == 0 and autotune._bin(0.4, te) == 1
    assert autotune._bin(2048, ne) == 0 and autotune._bin(262144, ne) == len(ne) - 2


def test_choose_reads_the_table_and_falls_back():
    table = {"theta_edges": [0.0, 0.5, 1.0], "n_edges": [1, 10000, 1 << 30],
             "best": {"0,0": 8, "1,1": 32}}
    sizes = [5000, 50000, 5000, 50000]
    thetas = [0.3, 0.9, 0.9, 0.3]
    got = autotune.choose(sizes, thetas, table)
    assert got.dtype == np.int32
    assert list(got) == [8, 32, autotune.DEFAULT_LEAF, autotune.DEFAULT_LEAF]
    assert list(autotune.choose(sizes, thetas, {})) == [autotune.DEFAULT_LEAF] * 4
