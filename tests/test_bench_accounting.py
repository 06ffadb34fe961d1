"""The algorithmic-byte accounting behind the bench's rooflines (CPU only):
vector streams of the adjoint schedule, counted by hand for small M."""
import pytest

import bench


def test_adjoint_streams_one_step_per_launch_m5():
    # M = 5: S = 3, two segments.  Forward: copies of j0, j1 (4 streams), steps
    # j2, j3, j4 (3 x 3), checkpoint 1 = (j3, j4) copied (4) -> 17.  Recompute:
    # segment 1 copies j3, j4 (4); segment 0 copies j0, j1 (4) and one step
    # for j2 (3) -> 11.  Reverse: lam4 is its source; lam3, lam2, lam1 are
    # three steps (9) and lam4 .. lam1 four accumulations (8) -> 17.
    assert bench.adjoint_streams(5) == 17 + 11 + 17


def test_adjoint_streams_multi_step_m5():
    # Forward: copies (4), one three-step pass in place j1 -> j4 (4 streams),
    # checkpoint copies (4) -> 12.  Recompute: 4 + (4 + 3) -> 11.  Reverse:
    # lam3, lam2, lam1 in one pass writing three levels (2 + 3) and four
    # accumulations (8) -> 13.
    assert bench.adjoint_streams(5, multi=True) == 12 + 11 + 13


@pytest.mark.parametrize("M", [2, 3, 7, 40, 64, 101, 512])
def test_multi_step_schedule_never_moves_more(M):
    assert bench.adjoint_streams(M, multi=True) <= bench.adjoint_streams(M)


def test_headline_traffic_record_matches_the_kernel_source():
    """The bench reports the dominant kernel's DRAM traffic from the committed
    ncu summary only while the kernel's source is the one those counters were
    taken with; a change to the three-step pass without a recapture shows up
    here rather than as a silent null in the bench line."""
    traffic, src = bench.recorded_traffic(("step_multi.cu", "multi_pass.cuh"), "step_multi_kernel_fp32_*.md")
    assert src is not None and src.startswith("profiles/")
    # four vector streams of 2N x B x 4 B per launch (128 x 128, all 16384 columns): within 1%
    algorithmic = 4 * 2 * 16384 * 16384 * 4
    assert abs(traffic / algorithmic - 1.0) < 0.01


def test_profiles_hold_text_summaries_with_unlocked_clocks():
    """profiles/ holds short text summaries; every ncu command in them leaves
    the clocks alone (--clock-control none) and names committed files only."""
    import glob
    import os
    import re
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    paths = sorted(glob.glob(os.path.join(root, "profiles", "*")))
    assert paths
    for path in paths:
        assert path.endswith((".md", ".txt")), path
        assert os.path.getsize(path) < 64 * 1024, path
        text = open(path).read()
        assert "_work" not in text, path
        # an ncu command may continue over backslash-ended lines
        for cmd in re.findall(r"(?m)^\s*ncu\b(?:[^\n]*\\\n)*[^\n]*", text):
            assert "--clock-control none" in cmd, (path, cmd)
