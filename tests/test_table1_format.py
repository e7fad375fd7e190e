"""Pins the output format (reading 10: int32 cell ranges over every cell and
int32 object references over every pair) against the paper's Table 1
(Sec. 5), tests/golden/table1_grid_attributes.txt: for each scene the
printed memory equals 4 (cells + pairs) bytes in MiB, with the pair count
taken from either of the table's two routes (triangles x cells per object,
or non-empty cells x objects per non-empty cell), and the cell count is the
product of the printed dimensions.  Then the oracle's own grid of a scene
has exactly that layout: ncells + 1 int32 ranges and NO int32 references."""
import os

import numpy as np
import pytest

import oracle
import scenes

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "table1_grid_attributes.txt")


def _rows():
    rows = []
    for line in open(GOLDEN):
        if not line.strip() or line.startswith("#"):
            continue
        name, tris, dims, cells, empty, per_cell, per_item, mem = line.split()
        dx, dy, dz = (int(v) for v in dims.split("x"))
        rows.append(dict(name=name, tris=float(tris), dims=(dx, dy, dz), cells=float(cells), empty=float(empty) / 100,
                         per_cell=float(per_cell), per_item=float(per_item), mem=float(mem)))
    return rows


@pytest.mark.parametrize("row", _rows(), ids=lambda r: r["name"])
def test_table1_columns_agree_with_the_int32_compact_format(row):
    dx, dy, dz = row["dims"]
    cells = dx * dy * dz
    assert abs(cells - row["cells"]) <= 0.005 * row["cells"] + 10, (cells, row["cells"])   # printed to 3-4 digits
    pairs_by_items = row["tris"] * row["per_item"]
    pairs_by_cells = cells * (1 - row["empty"]) * row["per_cell"]
    assert abs(pairs_by_items - pairs_by_cells) <= 0.01 * pairs_by_items, (pairs_by_items, pairs_by_cells)
    mem = 4 * (cells + pairs_by_items) / 2**20
    assert abs(mem - row["mem"]) <= 0.01 * row["mem"], (mem, row["mem"])
    # a different element size does not fit the column
    assert abs(8 * (cells + pairs_by_items) / 2**20 - row["mem"]) > 0.3 * row["mem"]


def test_oracle_grid_has_the_table1_layout():
    s = scenes.uniform_soup(3000, seed=991)
    o = oracle.build_grid(s.verts, s.tris, s.lam)
    assert o.G.dtype == np.int32 and o.refs.dtype == np.int32
    assert o.G.shape == (o.plan.ncells + 1,) and o.refs.shape == (o.NO,)
    assert o.G.nbytes + o.refs.nbytes == 4 * (o.plan.ncells + 1 + o.NO)
