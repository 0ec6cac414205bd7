"""Pins of the event-labeling oracle (paper Sec. 3.3, Appendix A.5).

tests/golden/label_modes.json holds one hand-built trajectory per success and
failure mode of the four subtasks, each acting out the mode's plain-text
description (cited per case), with the event list the appendix's event
definitions give for it. The oracle must reproduce both the events and the
mode. Random trajectories then check the partition: a trajectory gets a
success mode exactly when its list holds a success event.
"""
import json
import os

import numpy as np
import pytest

from oracle import labels as L
from paper_2412_13211_b300 import trajectories as TR

HERE = os.path.dirname(os.path.abspath(__file__))
TASK = {"pick": L.PICK, "place": L.PLACE, "open": L.OPEN, "close": L.CLOSE}
CASES = json.load(open(os.path.join(HERE, "golden", "label_modes.json")))["cases"]


@pytest.mark.parametrize("case", CASES, ids=[f"{c['task']}-{c['mode']}" for c in CASES])
def test_mode_examples(case):
    task = TASK[case["task"]]
    n = len(case["cumcol"])
    rec = {k: [float(x) for x in case[k]] for k in ("force", "dist", "artq", "cumcol") if k in case}
    rec["grasped"] = [bool(x) for x in case.get("grasped", [0] * n)]
    rec["success"] = [bool(x) for x in case["success"]]
    E = L.events(task, rec, n)
    assert E == case["events"]
    d0 = rec["dist"][0] if task == L.PLACE else None
    assert L.label(task, E, d0) == case["mode"]


def test_every_mode_has_an_example():
    seen = {(c["task"], c["mode"]) for c in CASES}
    for task, modes in (("pick", 9), ("place", 12), ("open", 9), ("close", 9)):
        for m in range(1, modes + 1):
            assert (task, m) in seen, (task, m)


def test_last_occurrence_index():
    assert L.idx(["contact", "grasped", "dropped", "grasped"], "grasped") == 3
    assert L.idx([], "grasped") == -1


@pytest.mark.parametrize("task", [L.PICK, L.PLACE, L.OPEN, L.CLOSE])
def test_random_trajectories_partition(task):
    traj = TR.make(task, num=400, steps=60, seed=3)
    E, lab = L.label_batch(task, traj)
    success_modes = {L.PICK: range(1, 5), L.PLACE: range(1, 6), L.OPEN: range(1, 4), L.CLOSE: range(1, 4)}[task]
    for ev, lb in zip(E, lab):
        if "success" in ev:
            assert lb in success_modes or lb == 0
        else:
            assert lb not in success_modes
    # the generator reaches most modes
    assert len(set(lab)) >= 5
    assert np.mean(np.asarray(lab) == 0) < 0.3      # lists no mode describes (reading L7)
