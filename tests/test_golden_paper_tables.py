"""The bench's rate and energy arithmetic against the numbers the paper prints
(tests/golden/paper_tables.txt: Tables 2 and 3 of §4.3, with the Eq. 1 rates
of §4.2).  No GPU: these are the unit conversions every reported figure goes
through, pinned to the paper's own quotients rather than to a retyped formula."""
import os

import pytest

import bench

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "paper_tables.txt")


def _rows():
    rows = []
    for line in open(GOLDEN):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        table, prec, platform, gflops, watt, ratio = line.split()
        rows.append((table, prec, platform, float(gflops), float(watt), float(ratio)))
    return rows


def test_fixture_holds_both_tables():
    rows = _rows()
    assert len(rows) == 8
    assert {r[0] for r in rows} == {"table2", "table3"}
    # the best rates are the same in both tables; only the watt column differs
    rates = {}
    for table, prec, platform, g, _, _ in rows:
        rates.setdefault((prec, platform), set()).add(g)
    assert all(len(v) == 1 for v in rates.values())


@pytest.mark.parametrize("row", _rows(), ids=lambda r: f"{r[0]}-{r[1]}-{r[2]}")
def test_gflops_per_watt_reproduces_the_papers_quotients(row):
    _, _, _, gflops, watt, ratio = row
    assert round(bench.gflops_per_watt(gflops, watt), 2) == ratio


@pytest.mark.parametrize("row", _rows(), ids=lambda r: f"{r[0]}-{r[1]}-{r[2]}")
def test_eq1_round_trip_from_relaxations(row):
    """Eq. 1 counts two operations per relaxation: the paper's GFLOPS are
    gflops / 2 * 1e9 relaxations per second, and the bench maps them back."""
    gflops = row[3]
    relax = gflops / 2 * 1e9
    assert bench.eq1_gflops(relax) == pytest.approx(gflops, rel=1e-15)
    # the energy figure the bench prints is the paper's quotient for the same rate
    assert round(bench.gflops_per_watt(bench.eq1_gflops(relax), row[4]), 2) == row[5]

