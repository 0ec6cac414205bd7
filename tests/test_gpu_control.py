"""The CUDA control wrapper (msh_set_controller, msh_control_step) against the
oracle (Sec. 4.1 normalised actions; Sec. 4.2 five 100 Hz physics steps per
20 Hz action).

Tolerances: the controller's arithmetic is FP32 in the oracle's order without
FMA contraction, so every column but the base's x and y is bit-exact; those
two take cosf/sinf of the yaw target (a few ulp from the correctly rounded
value the oracle uses) and agree within 1e-6 m. After one control step (five
physics steps) body states agree with the FP32 oracle within 5e-5 m and
5e-4 m/s: five times the one-step bound. The graph and the direct launches,
and every execution form, agree bit for bit; the physics part equals five
msh_step calls with the controller's targets.
"""
import ctypes as C

import numpy as np
import pytest

import oracle
from oracle import control as K
from paper_2412_13211_b300 import scenes as S

pytestmark = pytest.mark.gpu
SMALL = {2: 8, 3: 8, 4: 8, 6: 8}


def _sim(sc, cfg, spec, **kw):
    from paper_2412_13211_b300.sim import MshSim
    sim = MshSim(sc, cfg, **kw)
    sim.set_controller(spec)
    return sim


def bits(a):
    return np.ascontiguousarray(a, np.float32).view(np.int32)


def _err(a, b):
    return float(np.abs(np.asarray(a, np.float64) - np.asarray(b, np.float64)).max()) if np.size(a) else 0.0


@pytest.mark.parametrize("idx", [2, 3, 6])
def test_controller_targets_match_oracle(idx):
    import torch
    sc, cfg = S.make_config(idx, num_envs=SMALL[idx])
    spec = sc.controller_spec()
    acts = sc.random_actions(6, spec.action_dim, seed=1, amp=1.3)        # some components beyond [-1, 1]
    acts[0, 0, 0] = np.nan                                                # counts as -1
    sim = _sim(sc, cfg, spec)
    t_ref = sc.targets0.astype(np.float32)
    base = np.isin(spec.kind, [K.BASE_X, K.BASE_Y])
    dtc = K.control_dt(spec.steps_per_action, cfg.dt, "f32")
    for a in acts:
        sim.control_step(torch.as_tensor(a).cuda())
        t_ref = K.controller(spec, a, t_ref, dtc, "f32")
        # the oracle continues from the GPU's targets so that ulp differences in x, y do not accumulate
        got = sim.ctrl_targets.cpu().numpy()
        assert np.array_equal(bits(got[:, ~base]), bits(t_ref[:, ~base]))
        assert _err(got[:, base], t_ref[:, base]) <= 1e-6
        t_ref = got.copy()
    assert not sim.status().any()
    sim.close()


@pytest.mark.parametrize("idx", [2, 3, 4, 6])
def test_one_control_step_parity(idx, record_property):
    import torch
    sc, cfg = S.make_config(idx, num_envs=SMALL[idx])
    spec = sc.controller_spec()
    a = sc.random_actions(1, spec.action_dim, seed=2)[0]
    sim = _sim(sc, cfg, spec)
    sim.control_step(torch.as_tensor(a).cuda())
    gpu = sim.state_numpy()
    status = sim.status()
    o32, t32, st32 = K.control_step(sc, cfg, spec, sc.state(), a, sc.targets0, "f32")
    o64, _, _ = K.control_step(sc, cfg, spec, sc.state(), a, sc.targets0, "f64")
    assert np.array_equal(status, st32)
    errs = [_err(gpu[k], o32[k]) for k in range(4)]
    record_property("err_vs_fp32", errs)
    record_property("err_vs_fp64", [_err(gpu[k], o64[k]) for k in range(4)])
    assert errs[0] <= 5e-5 and errs[1] <= 5e-5
    assert errs[2] <= 5e-4 and errs[3] <= 5e-4
    assert _err(sim.ctrl_targets.cpu().numpy(), t32) <= 1e-6
    sim.close()


@pytest.mark.parametrize("idx", [3, 6])
def test_forms_graph_and_step_calls_bitwise_equal(idx):
    import torch
    sc, cfg = S.make_config(idx, num_envs=SMALL[idx])
    spec = sc.controller_spec()
    acts = torch.as_tensor(sc.random_actions(3, spec.action_dim, seed=3)).cuda()
    results = []
    for kw in (dict(exec_form="fused"), dict(exec_form="fused", use_graph=True),
               dict(exec_form="plain", use_graph=True), dict(exec_form="substep"),
               dict(exec_form="fused", threads_per_env=16, use_graph=True)):
        sim = _sim(sc, cfg, spec, **kw)
        for k in range(3):
            sim.control_step(acts[k].contiguous())
        results.append(sim.state_numpy() + (sim.ctrl_targets.cpu().numpy(),))
        sim.close()
    for r in results[1:]:
        for x, y in zip(results[0], r):
            assert np.array_equal(bits(x), bits(y))
    # the physics part: five msh_step calls with the controller's targets
    sim = _sim(sc, cfg, spec)
    sim.control_step(acts[0].contiguous())
    ref = sim.state_numpy()
    tg = sim.ctrl_targets.clone()
    sim.close()
    from paper_2412_13211_b300.sim import MshSim
    plain = MshSim(sc, cfg)
    for _ in range(spec.steps_per_action):
        plain.step(tg)
    for x, y in zip(ref, plain.state_numpy()):
        assert np.array_equal(bits(x), bits(y))
    plain.close()


def test_recording_handle_records_every_physics_step():
    import torch
    sc, cfg = S.make_config(4, num_envs=4)
    spec = sc.controller_spec()
    sim = _sim(sc, cfg, spec)
    sim.set_tape(12)
    a = torch.as_tensor(sc.random_actions(1, spec.action_dim)[0]).cuda()
    sim.control_step(a)
    sim.control_step(a)
    assert int(sim.lib.msh_tape_count(sim.handle)) == 10
    with pytest.raises(RuntimeError):
        sim.control_step(a)                              # 15 > 12: refused before any launch
    sim.close()


def test_controller_argument_checks():
    import torch
    from paper_2412_13211_b300 import _lib
    sc, cfg = S.make_config(3, num_envs=2)
    spec = sc.controller_spec()
    from paper_2412_13211_b300.sim import MshSim
    sim = MshSim(sc, cfg)
    st = sim._state()
    a = torch.zeros((2, spec.action_dim), device="cuda")
    rc = sim.lib.msh_control_step(sim.handle, C.byref(st), C.c_void_p(a.data_ptr()),
                                  C.c_void_p(sim.targets.data_ptr()), None)
    assert rc == _lib.MSH_ERR_INVALID_ARG                 # no controller yet

    def bad(**kw):
        s = S.ControllerSpec(**{**spec.__dict__, **{k: v for k, v in kw.items()}})
        with pytest.raises(RuntimeError):
            sim.set_controller(s)
    kind = spec.kind.copy()
    kind[3] = 9
    bad(kind=kind)
    col = spec.action.copy()
    col[3] = spec.action_dim
    bad(action=col)
    lo = spec.lo.copy()
    lo[3] = spec.hi[3] + 1
    bad(lo=lo)
    bad(yaw_dof=-1)
    bad(steps_per_action=0)
    sim.set_controller(spec)
    assert sim.lib.msh_control_step(sim.handle, C.byref(st), None, C.c_void_p(sim.targets.data_ptr()),
                                    None) == _lib.MSH_ERR_INVALID_ARG
    sim.close()
