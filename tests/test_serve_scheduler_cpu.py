"""Serving admission logic on the CPU: the scheduler the library's serving
loop uses, driven by a fake executor (batches take a modelled time)."""
import os
import subprocess

import numpy as np
import pytest

from conftest import ROOT

HARNESS = os.path.join(ROOT, "tests", "sched_harness.cpp")


@pytest.fixture(scope="module")
def harness(tmp_path_factory):
    exe = str(tmp_path_factory.mktemp("sched") / "sched")
    subprocess.run(["g++", "-O2", "-std=c++17", "-o", exe, HARNESS], check=True)
    return exe


def run(exe, arrivals, sizes, budget, slots, max_batch, per_byte=1e-9, fixed=1e-3):
    lines = [f"{len(arrivals)} {budget} {slots} {max_batch} {per_byte} {fixed}"]
    lines += [f"{a:.9f} {b}" for a, b in zip(arrivals, sizes)]
    out = subprocess.run([exe], input="\n".join(lines), capture_output=True, text=True,
                         check=True).stdout.splitlines()
    head = out[0].split()
    rows = np.array([[float(x) for x in ln.split()] for ln in out[1:]])
    return dict(violations=int(head[1]), peak=int(head[3]), peak_batches=int(head[5]),
                done=int(head[7])), rows


def test_budget_slots_and_batch_limits_hold(harness):
    g = np.random.default_rng(0)
    n = 300
    arrivals = np.cumsum(g.exponential(1e-3, n))
    sizes = g.integers(10_000_000, 200_000_000, n)
    budget = 1_000_000_000
    info, rows = run(harness, arrivals, sizes, budget, slots=4, max_batch=8)
    assert info["violations"] == 0 and info["done"] == 1
    assert info["peak"] <= budget
    admit, finish = rows[:, 1], rows[:, 2]
    assert np.all(admit >= arrivals - 1e-8) and np.all(finish > admit)   # 9-decimal I/O


def test_admission_is_fifo_and_batches_overlap(harness):
    g = np.random.default_rng(1)
    n = 200
    arrivals = np.cumsum(g.exponential(5e-4, n))
    sizes = g.integers(1_000_000, 50_000_000, n)
    info, rows = run(harness, arrivals, sizes, 10_000_000_000, slots=3, max_batch=4)
    admit = rows[:, 1]
    order = np.argsort(arrivals, kind="stable")
    assert np.all(np.diff(admit[order]) >= -1e-12)      # never admitted out of arrival order
    assert info["peak_batches"] > 1                      # continuous batching: overlap happens


def test_requests_arriving_while_busy_join_later_batches(harness):
    # a burst: the first batch is admitted alone, the rest queue and are
    # admitted as slots free up (several per batch)
    arrivals = [0.0] + [1e-6] * 20
    sizes = [100] * 21
    info, rows = run(harness, arrivals, sizes, 10 ** 9, slots=1, max_batch=8, fixed=1e-3)
    admit = rows[:, 1]
    assert admit[0] == 0.0
    assert len(np.unique(admit[1:])) == 3                 # 8 + 8 + 4 per batch


def test_oversized_request_is_rejected_others_served(harness):
    arrivals = [0.0, 0.001, 0.002]
    sizes = [100, 5_000, 100]
    info, rows = run(harness, arrivals, sizes, 1_000, slots=2, max_batch=4)
    assert info["done"] == 1
    assert rows[1, 3] == 1 and rows[0, 3] == 0 and rows[2, 3] == 0
    assert rows[0, 2] > 0 and rows[2, 2] > 0


def test_budget_limits_concurrency(harness):
    # each request takes 40 % of the budget: at most two can be in flight
    arrivals = [0.0] * 10
    sizes = [400] * 10
    info, rows = run(harness, arrivals, sizes, 1000, slots=8, max_batch=1)
    assert info["peak"] <= 1000 and info["peak_batches"] == 2
