"""The paper's storage model (Sec. 4.4, eqs. memory_diffusion /
memory_convection) against the values printed in its Tables 4-6
(tests/golden/memory_tables.txt): Table 4 is in units of 1e9 bytes, Tables 5
and 6 in GiB, each rounded as printed; and the problem sizes of Table 1
(tests/golden/problem_sizes.txt)."""
import os

import pytest

from paper_1805_11930_gb300 import footprint

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "memory_tables.txt")


def rows():
    out = []
    for line in open(GOLDEN):
        if line.startswith("#") or not line.strip():
            continue
        t, p, nx, ny, nz, mx, pmf, mf = line.split()
        out.append((int(t), int(p), int(nx) * int(ny) * int(nz), float(mx), float(pmf), float(mf), mf))
    return out


@pytest.mark.parametrize("row", rows(), ids=lambda r: f"table{r[0]}_p{r[1]}")
def test_memory_tables(row):
    t, p, ncell, mx, pmf, mf, mf_text = row
    if t == 4:
        kw, unit = dict(problem="diffusion"), 1e9
    elif t == 5:
        kw, unit = dict(problem="convection", n_out=100, n_blk=100), 2.0 ** 30
    else:
        kw, unit = dict(problem="convection", n_out=15, n_blk=12), 2.0 ** 30
    val = {v: footprint.paper_model(p, ncell, variant=v, **kw) * 8 / unit for v in ("MX", "PMF", "MF")}
    assert abs(val["MX"] - mx) <= 0.05 + 1e-9
    assert abs(val["PMF"] - pmf) <= 0.05 + 1e-9
    decimals = len(mf_text.split(".")[1])
    assert abs(val["MF"] - mf) <= 0.5 * 10 ** (-decimals) + 1e-9


SIZES = os.path.join(os.path.dirname(__file__), "golden", "problem_sizes.txt")


def size_rows():
    out = []
    for line in open(SIZES):
        if line.startswith("#") or not line.strip():
            continue
        p, npc, nx, ny, nz, mdofs, gib, ratio = line.split()
        out.append((int(p), int(npc), int(nx) * int(ny) * int(nz), float(mdofs), float(gib), int(ratio)))
    return out


@pytest.mark.parametrize("row", size_rows(), ids=lambda r: f"table1_p{r[0]}")
def test_problem_size_table(row):
    p, npc, ncell, mdofs, gib, ratio = row
    ndof = ncell * (p + 1) ** 3
    assert (p + 1) ** 3 == npc
    assert round(ndof / 1e6, 1) == mdofs
    assert abs(footprint.matrix_bytes(p, ncell) / 2.0 ** 30 - gib) <= 0.05 + 1e-9
    assert footprint.matrix_bytes(p, ncell) // (8 * ndof) == ratio
