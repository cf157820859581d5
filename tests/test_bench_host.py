"""Host-side arithmetic of bench.py, on CPU: the scaling of the headline's
sampled per-kernel profile."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def test_sampled_profile_scaled_to_every_generation():
    """The headline's tensor-core kinds are timed on one inner generation in
    PROFILE_STRIDE: their totals are the mean per sampled launch times the
    run's launches, the counts those launches; the per-launch mean is kept and
    the size-bucket kinds (timed on every launch) and the near-tie count are
    left as read."""
    import bench
    prof = {"fused_small": (3.0, 2), "tc_trial": (10.0, 50), "tc_sel": (6.0, 50), "tc_generation": (20.0, 50),
            "tc_gemm": (0.0, 0), "near_ties": (0.0, 1234)}
    out = bench.scale_sampled(prof, 200)
    assert out["tc_trial"] == (40.0, 200) and out["tc_sel"] == (24.0, 200) and out["tc_generation"] == (80.0, 200)
    assert out["fused_small"] == (3.0, 2) and out["near_ties"] == (0.0, 1234) and out["tc_gemm"] == (0.0, 0)
    for k in ("tc_trial", "tc_sel"):
        assert out[k][0] / out[k][1] == prof[k][0] / prof[k][1]
    assert prof["tc_trial"] == (10.0, 50)  # the profile read is not modified in place
    assert bench.PROFILE_STRIDE >= 1 and set(bench.TC_KINDS) >= {"tc_trial", "tc_sel", "tc_ties", "tc_prologue"}
