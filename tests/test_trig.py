"""Accuracy of the rollout step's branch-free sin / cos and Box-Muller
logarithm (csrc/trig.cuh), built for the host with nvcc and compared against
double-precision libm: the Taylor pair on |e| <= pi/4 and the Cody-Waite
reduced state angle on [-2^16, 2^16] stay within 1.5 ulp of 1.0f, sin
keeps its relative accuracy near zero, results stay in [-1, 1] up to 2^24
and NaN propagates; -2 ln u is within 2 ulp of the exact value on all 2^23
uniforms the noise maps to (the host divides exactly; the device's MUFU
reciprocal adds about 2 ulp, bounded on the GPU by the noise-stream test),
and sin / cos of 2 pi u from the uniform's bits within 1 ulp of 1.0f on
all of them."""
import json
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2508_05773_gb300", "csrc")


def _nvcc():
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    return None


@pytest.fixture(scope="module")
def errors(tmp_path_factory):
    nvcc = _nvcc()
    if nvcc is None:
        pytest.skip("nvcc not available")
    exe = str(tmp_path_factory.mktemp("trig") / "trig_check")
    src = os.path.join(ROOT, "tests", "trig_check.cu")
    subprocess.run([nvcc, "-O2", "-std=c++17", "-Xcompiler", "-ffp-contract=off", "-I", CSRC, src, "-o", exe],
                   check=True, capture_output=True, text=True)
    out = subprocess.run([exe], check=True, capture_output=True, text=True).stdout
    return json.loads(out.strip().splitlines()[-1])


def test_turn_pair_within_bound(errors):
    assert errors["turn_sin_ulp"] <= 1.5 and errors["turn_cos_ulp"] <= 1.5, errors


def test_state_angles_within_bound(errors):
    assert errors["state_sin_ulp"] <= 1.5 and errors["state_cos_ulp"] <= 1.5, errors
    assert errors["state_sin_rel"] <= 3e-7, errors


def test_far_arguments_bounded_and_nan(errors):
    assert errors["far_max_abs"] <= 1.0 + 1e-6, errors
    assert errors["nan_propagates"] == 1, errors


def test_box_muller_log_within_bound(errors):
    assert errors["neg2_log_ulp"] <= 2.0, errors


def test_box_muller_angle_within_bound(errors):
    assert errors["unit_sin_ulp"] <= 1.0 and errors["unit_cos_ulp"] <= 1.0, errors
