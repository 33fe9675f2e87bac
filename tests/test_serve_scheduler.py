"""Scheduling of the exchange server, without a device.

tests/serve_scheduler_driver.cpp runs the server's scheduler
(paper_1801_09263_gb300/csrc/serve_core.h, the code liblace's lace_server_*
calls run) with a fake executor that sleeps for each request, and prints what
ran when.  The checks: requests of different systems overlap up to the slot
count; one system's requests run in submission order; an apply before the
first rebuild fails with the state error; memory admission makes a request
wait while its growth does not fit and fails it with the out-of-memory status
when it can never fit; removing a system frees its memory; a rebuild-slot
limit keeps slots free for applies; a REBUILD starts together with a queued
REBUILD on the same grid as one group in one rebuild slot (so that the two
can share pass launches), but only within the memory budget; the
rebuild cadence reports a rebuild as due once the block energy of
consecutive applies has converged.
"""
import json
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(os.path.dirname(HERE), "paper_1801_09263_gb300", "csrc")
OK, ERR_ARG, ERR_STATE, ERR_OOM = 0, 1, 2, 3
REBUILD, APPLY = 0, 1


@pytest.fixture(scope="module")
def runs(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    if not cxx:
        pytest.skip("no C++ compiler")
    exe = str(tmp_path_factory.mktemp("sched") / "driver")
    subprocess.run([cxx, "-std=c++17", "-O1", "-pthread", "-I", CSRC,
                    os.path.join(HERE, "serve_scheduler_driver.cpp"), "-o", exe], check=True)
    out = subprocess.run([exe], check=True, capture_output=True, text=True, timeout=120).stdout
    return {d["name"]: d for d in map(json.loads, out.strip().splitlines())}


def _per_system_order(reqs):
    by = {}
    for r in reqs:
        by.setdefault(r["sys"], []).append(r)
    for rs in by.values():
        for a, b in zip(rs, rs[1:]):
            assert b["start"] >= a["end"] - 1e-3, (a, b)


def test_requests_of_different_systems_overlap(runs):
    r = runs["overlap"]
    assert all(q["status"] == OK and q["done"] for q in r["requests"])
    assert r["max_running"] == 4
    _per_system_order(r["requests"])
    # 12 requests of 50 ms on 4 slots: about 150 ms, far below 600 ms serial
    assert max(q["end"] for q in r["requests"]) < 450
    for q in r["requests"]:
        if q["kind"] == REBUILD:
            assert q["ex"] == -(q["sys"] + 1) and q["n_pairs"] == 10 * (q["sys"] + 1)
        else:
            assert q["out0"] == 3.0


def test_one_slot_runs_in_submission_order(runs):
    r = runs["serial"]
    assert r["max_running"] == 1
    ends = [q["end"] for q in r["requests"]]
    assert ends == sorted(ends)
    assert all(q["status"] == OK for q in r["requests"])


def test_apply_before_rebuild_is_a_state_error(runs):
    st = [q["status"] for q in runs["state"]["requests"]]
    assert st == [ERR_STATE, OK, OK]
    _per_system_order(runs["state"]["requests"])


def test_memory_admission_waits_then_refuses(runs):
    q = runs["memory"]["requests"]
    assert [x["status"] for x in q] == [OK, OK, OK, OK, ERR_OOM]
    a, b = q[0], q[1]
    assert b["start"] >= a["end"] - 1e-3  # B's rebuild waited for A's transient memory
    assert q[4]["latency"] >= a["end"] - 1e-3  # refused only once nothing else could free memory


def test_removed_system_frees_memory(runs):
    q = runs["remove"]["requests"]
    assert [x["status"] for x in q] == [OK, OK, OK, -ERR_ARG]


def test_rebuild_slots_leave_room_for_applies(runs):
    r = runs["rebuild_slots"]
    q = r["requests"]
    assert all(x["status"] == OK for x in q)
    assert r["max_rebuilding"] == 1
    # system 0's applies ran while the later rebuilds were still running
    last_rebuild_end = max(x["end"] for x in q if x["kind"] == REBUILD)
    assert all(x["end"] < last_rebuild_end for x in q if x["kind"] == APPLY)


def test_rebuild_is_due_once_the_inner_loop_has_converged(runs):
    """The double loop of the paper (Sec. 2): the inputs of the inner loop
    converge (factor 1 + 0.5^k); an APPLY reports a rebuild as due when its
    block energy differs from the previous APPLY's by at most the tolerance
    (1e-3 relative), and never right after a REBUILD."""
    q = runs["cadence"]["requests"]
    assert all(x["status"] == OK for x in q)
    applies = [x for x in q[1:15]]
    e = [x["e_block"] for x in applies]
    assert e == sorted(e)  # |e| shrinks toward its limit
    expect = [False] + [abs(b - a) <= 1e-3 * abs(b) for a, b in zip(e, e[1:])]
    assert [bool(x["rebuild_due"]) for x in applies] == expect
    first_due = expect.index(True)
    assert 9 <= first_due <= 12 and all(expect[first_due:])
    assert q[15]["kind"] == REBUILD
    assert [bool(x["rebuild_due"]) for x in q[16:]] == [False, True]  # the same block twice after the rebuild


def test_rebuilds_on_one_grid_start_together_as_one_group(runs):
    """REBUILD groups: with one rebuild slot, system 2 (system 0's grid)
    starts with system 0 as one group once the slot frees, ahead of system 1
    submitted before it, and 1 waits for the group's slot.  Every request
    runs once and succeeds."""
    run = runs["group"]
    q = {x["sys"]: x for x in run["requests"]}
    assert all(x["status"] == OK for x in q.values())
    assert q[0]["start"] >= q[3]["end"] - 1e-3
    assert abs(q[2]["start"] - q[0]["start"]) < 20
    assert q[1]["start"] >= max(q[0]["end"], q[2]["end"]) - 1e-3
    assert run["max_rebuilding"] == 2  # the group ran at once in one slot


def test_rebuild_group_stays_within_the_memory_budget(runs):
    """Two REBUILDs on one grid that do not fit the budget together run one
    after the other, not as a group."""
    q = {x["sys"]: x for x in runs["group_memory"]["requests"]}
    assert all(x["status"] == OK for x in q.values())
    first, second = sorted(q.values(), key=lambda x: x["start"])
    assert second["start"] >= first["end"] - 1e-3
