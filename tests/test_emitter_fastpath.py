"""Host-side checks of the emitted float32 path of the float-pair rate
kernels (no GPU): the path is a warp-wide vote on float32 estimates against
2^-40 of the state's scale anchor, emitted for the elementary, three-body,
falloff and chemically activated classes of the production-rate kernels
only (never in the rates-of-progress kernel, whose bar is each reaction's
own rate), and kx_options.rates_negligible = 1 removes it."""
import re

import pytest

from paper_2411_02640_gb300 import kx, synth


def _src(tmp_path, kernel, **opts):
    path = synth.mechanism_file("gri_53_325", str(tmp_path))
    m = kx.Mechanism(path, cache_dir=str(tmp_path / "cache"), compile_only=1, lazy=1, **opts)
    return m.kernel_source(kernel)


def test_thread_per_state_vote(tmp_path):
    src = _src(tmp_path, "wdot_fp64", rates_layout=1)
    votes = re.findall(r"__all_sync\(__activemask\(\), lme < __fmul_rn\(kx_i2f\(S \+ 22\), 0\.693147182f\)\)", src)
    # one vote per eligible class loop, in both copies of the main pass (signed and sign-free)
    assert len(votes) >= 2 and len(votes) % 2 == 0
    assert "__expf(lfe - sl)" in src


def test_warp_cooperative_vote(tmp_path):
    src = _src(tmp_path, "wdot_fp64", rates_layout=2)
    assert "__reduce_max_sync(__activemask(), emax)" in src
    assert re.search(r"__all_sync\(__activemask\(\), lme < __fmul_rn\(kx_i2f\(emx - 40\), 0\.693147182f\)\)", src)


@pytest.mark.parametrize("kernel,layout", [("wdot_fp64", 1), ("wdot_fp64", 2)])
def test_rates_negligible_removes_the_path(tmp_path, kernel, layout):
    src = _src(tmp_path, kernel, rates_layout=layout, rates_negligible=1)
    assert "lme <" not in src and "__expf(lfe" not in src


def test_rates_of_progress_never_take_it(tmp_path):
    src = _src(tmp_path, "rop_fp64")
    assert "lme <" not in src and "__expf(lfe" not in src


def test_running_scale_rescales_in_two_steps(tmp_path):
    """The thread-per-state kernel's running scale applies a rescale's power of two as two factors
    of at least 2^-126 each (a single factor is zero below 2^-126 and zeroed sums that would
    still be representable after a jump of more than 2^126)."""
    src = _src(tmp_path, "wdot_fp64", rates_layout=1)
    assert "d1 = max(d, -126), d2 = d - d1" in src
    assert re.search(r"w\[k\] = kx_mk\(__fmul_rn\(__fmul_rn\(w\[k\]\.hi, f1\), f2\)", src)
