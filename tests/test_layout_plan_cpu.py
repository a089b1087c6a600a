"""The host plan of the tiled split-CSR layout (rhpdhg_plan_layout, no device) against the rule
restated in Python (layout_rule.py), on row-length patterns that reach every branch: long rows by
length and by the segment budget (ties included), empty rows, ragged last tiles, and each choice
of tiles per work item."""
import os
import shutil

import numpy as np
import pytest

import layout_rule
from paper_2407_16144_gb300 import rhpdhg as rh

pytestmark = pytest.mark.skipif(shutil.which("nvcc") is None and
                                not os.path.exists("/usr/local/cuda/bin/nvcc"),
                                reason="nvcc not available")


@pytest.fixture(scope="module")
def rh_lib():
    """The library, built here; the plan is host code, so no device is needed."""
    from paper_2407_16144_gb300 import _build
    _build.build()
    return rh.load()


def _rp(lengths):
    return np.concatenate([[0], np.cumsum(np.asarray(lengths, dtype=np.int64))])


def _cases():
    rng = np.random.default_rng(7)
    yield "empty", []
    yield "one_row", [5]
    yield "all_empty_rows", [0] * 100
    yield "single_entry_rows_ragged", [1] * 4001            # mult 4, ragged last group
    yield "two_entry_rows", [2] * 4001                      # mean 64 per tile: mult 4 at the bound
    yield "three_entry_rows", [3] * 40000                   # mult 2
    yield "dense_short_rows", [25] * 1000                   # mult 1
    yield "long_by_length", [129, 1, 300, 5000, 0, 128] * 50
    yield "budget_ties", [40] * 32 * 10                     # 1280 per tile: ties broken by order
    yield "budget_mixed", list(rng.integers(0, 129, size=32 * 37 + 11))
    yield "power_law", list(np.minimum(rng.zipf(2.1, size=20000), 5000))
    yield "few_tiles", [1] * 100                             # 4 tiles: too few for 4 per item
    yield "bimodal", ([1] * 31 + [1000]) * 50               # long rows keep groups short


@pytest.mark.parametrize("name,lengths", list(_cases()), ids=[c[0] for c in _cases()])
def test_plan_matches_rule(rh_lib, name, lengths):
    rp = _rp(lengths)
    rc, got = rh.rhpdhg_plan_layout(rp)
    assert rc == 0
    assert got == layout_rule.plan(rp), name


def test_wide_row_sums_only_where_rows_are_skewed(rh_lib):
    """The warp-wide FP64 row sums are chosen for skewed tiles (one long row among short ones,
    a power law) and not for even row lengths, where they would save nothing."""
    rng = np.random.default_rng(11)
    skewed = ([2] * 31 + [100]) * 64
    even = [25] * 32 * 64
    power = list(np.minimum(rng.zipf(2.1, size=32 * 200), 128))
    for lengths, want in ((skewed, 1), (even, 0), (power, 1), ([40] * 32 * 8, 0)):
        rc, got = rh.rhpdhg_plan_layout(_rp(lengths))
        assert rc == 0 and got["wide_rows"] == want == layout_rule.plan(_rp(lengths))["wide_rows"]


def test_plan_rejects_bad_row_pointers(rh_lib):
    assert rh.rhpdhg_plan_layout(np.array([1, 2, 3]))[0] == rh.ERR_INVALID_ARG
    assert rh.rhpdhg_plan_layout(np.array([0, 3, 2]))[0] == rh.ERR_INVALID_ARG
