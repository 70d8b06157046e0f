"""Host-side tests of the serving scheduler (the continuous-batching loop of gm_sched.h) with a stub engine, on the
CPU: results in a mix equal results alone, batches respect the slot capacity, and the failure paths -- unknown
image, over-budget request, failed launch, bounded poll timeout, full queue, cancellation at shutdown -- return
their status without a GPU; admission follows the engine's capacity of the moment (the budget share left after
images put since the server started)."""
import json
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))

OK, NOT_FOUND, BUDGET, CUDA, TIMEOUT, CANCELLED, BUSY = 0, -4, -3, -5, -6, -7, -8


@pytest.fixture(scope="module")
def harness(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no C++ compiler")
    exe = str(tmp_path_factory.mktemp("sched") / "sched_harness")
    subprocess.run([cxx, "-std=c++17", "-O1", "-pthread", os.path.join(HERE, "sched_harness.cpp"), "-o", exe],
                   check=True)
    return lambda mode: json.loads(subprocess.run([exe, mode], check=True, capture_output=True, text=True,
                                                  timeout=120).stdout)


def test_mix_equals_alone(harness):
    r = harness("mix")
    assert r["bad"] == 0 and r["completed"] == 2000
    assert r["batches"] < 2000 and r["max_batch"] >= 2   # requests shared batches


def test_failure_paths(harness):
    r = harness("faults")
    assert r["unknown"] == NOT_FOUND and r["fits"] == OK and r["budget"] == BUDGET
    assert r["launch_fail"] == CUDA and r["failed"] >= 1
    assert r["timeout"] == TIMEOUT and r["after_release"] == OK
    assert r["busy"] >= 1 and r["rejected_busy"] == r["busy"] and r["rejected_budget"] == 0


def test_cancellation_at_stop(harness):
    r = harness("cancel")
    assert r["cancelled"] == 5 and r["ok"] == 1 and r["other"] == 0
    assert r["after_stop"] == CANCELLED


def test_admission_follows_current_capacity(harness):
    r = harness("shrink")
    assert r["bad"] == 0 and r["completed"] == 300
    assert 0 < r["max_multi_cost"] <= 4   # batches of several requests fit the capacity of the moment
