"""C-ABI checks that need no GPU: the library builds for sm_103a, loads,
exports every entry point declared in include/msh.h, and rejects invalid
arguments on the host with a message (no device call is made)."""
import ctypes as C
import os
import re

import numpy as np
import pytest

from paper_2412_13211_b300 import _lib, scenes
from paper_2412_13211_b300.sim import make_cfg, make_desc

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    src = open(os.path.join(ROOT, "include", "msh.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(msh_[a-z_]+)\s*\(", src)))


def test_library_exports_every_declared_symbol():
    lib = _lib.load()
    names = declared_symbols()
    assert len(names) >= 12
    for n in names:
        assert hasattr(lib, n), n
    assert set(names) == set(_lib.EXPORTS)


def _create(desc, cfg):
    lib = _lib.load()
    h = C.c_void_p()
    rc = lib.msh_create(C.byref(desc) if desc is not None else None, C.byref(cfg) if cfg is not None else None,
                        C.byref(h))
    return rc, h, lib.msh_last_error().decode()


def _scene():
    return scenes.make_config(2, num_envs=2)


def test_rejects_null_and_bad_config():
    sc, cfg = _scene()
    desc, keep = make_desc(sc)
    rc, h, msg = _create(None, make_cfg(cfg))
    assert rc == _lib.MSH_ERR_INVALID_ARG and not h.value
    bad = make_cfg(cfg)
    bad.substeps = 0
    rc, h, msg = _create(desc, bad)
    assert rc == _lib.MSH_ERR_INVALID_ARG and "substeps" in msg
    bad = make_cfg(cfg)
    bad.max_contacts = 5000
    rc, h, msg = _create(desc, bad)
    assert rc == _lib.MSH_ERR_INVALID_ARG and "max_contacts" in msg
    del keep


@pytest.mark.parametrize("field,value,needle", [
    ("body_mass", 0.0, "mass"),
    ("body_mass", np.nan, "mass"),
    ("body_shape", 7, "shape"),
    ("body_dims", -1.0, "dims"),
    ("joint_parent", 99, "parent"),
    ("joint_type", 5, "type"),
    ("joint_dof", 50, "dof"),
])
def test_rejects_invalid_descriptor(field, value, needle):
    sc, cfg = _scene()
    arr = getattr(sc, field).copy()
    arr.reshape(-1)[0] = value
    setattr(sc, field, arr)
    desc, keep = make_desc(sc)
    rc, h, msg = _create(desc, make_cfg(cfg))
    assert rc == _lib.MSH_ERR_INVALID_ARG, (rc, msg)
    assert needle in msg
    assert not h.value
    del keep


def test_rejects_non_monotone_offsets():
    sc, cfg = _scene()
    sc.body_off = sc.body_off.copy()
    sc.body_off[1] = sc.body_off[2] + 1
    desc, keep = make_desc(sc)
    rc, h, msg = _create(desc, make_cfg(cfg))
    assert rc == _lib.MSH_ERR_INVALID_ARG
    del keep


def test_null_handle_calls_fail_cleanly():
    lib = _lib.load()
    st = _lib.State()
    assert lib.msh_step(None, C.byref(st), None, 0.01, 1, None) == _lib.MSH_ERR_INVALID_ARG
    assert lib.msh_set_exec(None, 0, 128, 0) == _lib.MSH_ERR_INVALID_ARG
    assert lib.msh_get_status(None, None, None) == _lib.MSH_ERR_INVALID_ARG
    assert lib.msh_scratch_bytes(None) == 0
    assert lib.msh_set_report(None, None) == _lib.MSH_ERR_INVALID_ARG
    assert lib.msh_set_controller(None, None) == _lib.MSH_ERR_INVALID_ARG
    assert lib.msh_control_step(None, C.byref(st), None, None, None) == _lib.MSH_ERR_INVALID_ARG
    lib.msh_destroy(None)


def test_label_events_rejects_bad_arguments_before_any_launch():
    lib = _lib.load()
    b = _lib.TrajBatch()
    assert lib.msh_label_events(0, None, 8, None, None, None, None) == _lib.MSH_ERR_INVALID_ARG
    b.num_traj, b.num_steps = 4, 10
    out = (C.c_int8 * 32)()
    n = (C.c_int32 * 4)()
    lab = (C.c_int32 * 4)()
    assert lib.msh_label_events(7, C.byref(b), 8, out, n, lab, None) == _lib.MSH_ERR_INVALID_ARG   # unknown task
    assert lib.msh_label_events(0, C.byref(b), 8, out, n, lab, None) == _lib.MSH_ERR_INVALID_ARG   # no records
    assert lib.msh_label_events(0, C.byref(b), 0, out, n, lab, None) == _lib.MSH_ERR_INVALID_ARG   # max_events
    assert b"records" in lib.msh_last_error() or b"max_events" in lib.msh_last_error()
