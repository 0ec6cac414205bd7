"""Differentiable rollouts through the CUDA adjoint (msh_backward).

The rollout gradient of the goal loss w.r.t. the initial velocities, the
per-step joint targets and the masses: a closed form for free fall; bitwise
independence of the checkpoint interval, of the execution form that recorded
the steps, and of whether the forward pass kept its last segment; a central
difference of the GPU step itself for one recorded step. The adjoint of every
step is compared with the oracle element by element in
test_gpu_adjoint_parity.py.
"""
import numpy as np
import pytest

import oracle
from paper_2412_13211_b300 import scenes as S

pytestmark = pytest.mark.gpu


def _gpu_grads(sc, cfg, tg, nsteps, k, **sim_kw):
    import torch
    from paper_2412_13211_b300.autograd import goal_loss, rollout
    from paper_2412_13211_b300.sim import MshSim
    sim = MshSim(sc, cfg, **sim_kw)
    st = [torch.tensor(np.asarray(a, np.float32), device="cuda", requires_grad=True) for a in sc.state()]
    mass = torch.tensor(np.asarray(sc.body_mass, np.float32), device="cuda", requires_grad=True)
    targets = torch.tensor(np.asarray(tg[:nsteps], np.float32), device="cuda", requires_grad=True)
    out = rollout(sim, st, targets, mass, k)
    L = goal_loss(sim, out[0])
    L.sum().backward()
    res = dict(L=L.detach().cpu().numpy(), v=st[2].grad.cpu().numpy(), w=st[3].grad.cpu().numpy(),
               tg=targets.grad.cpu().numpy(), m=mass.grad.cpu().numpy(), status=sim.status())
    sim.close()
    return res


def test_free_fall_gradient_closed_form():
    from helpers import env, scene_from_envs
    e = env()
    e.body(S.SPHERE, (0.05,), 0.7, (0.1, -0.2, 50.0), linvel=(0.3, -0.1, 2.0))
    e.goal_body, e.goal_pos = 0, (0.5, 0.2, 49.0)
    sc = scene_from_envs([e])
    cfg = S.SolverCfg(substeps=3, iterations=4)
    n = 12
    g = _gpu_grads(sc, cfg, np.zeros((n, 1, 1), np.float32), n, 4)
    out, _ = oracle.step(sc, cfg, sc.state(), None, n, "f64")
    k, h = n * 3, 0.01 / 3
    r = out[0][0] - np.array(e.goal_pos)
    np.testing.assert_allclose(g["v"][0], 2 * r * k * h, rtol=1e-4, atol=1e-6)
    np.testing.assert_allclose(g["w"][0], 0.0, atol=1e-7)
    assert abs(g["m"][0]) < 1e-6


@pytest.fixture(scope="module")
def diff_case():
    sc, cfg = S.make_config(4, num_envs=16)
    nsteps = 8
    tg = sc.target_walk(nsteps, 3)
    g = _gpu_grads(sc, cfg, tg, nsteps, 4)
    return sc, cfg, tg, nsteps, g


def test_checkpoint_interval_does_not_change_gradients(diff_case):
    sc, cfg, tg, nsteps, g4 = diff_case
    for k in (1, 3, 8):
        gk = _gpu_grads(sc, cfg, tg, nsteps, k)
        for key in ("v", "w", "tg", "m"):
            assert np.array_equal(gk[key], g4[key]), (k, key)


def test_steps_recorded_by_every_form_give_the_same_gradients(diff_case):
    """The recorded steps (state, lambdas and the collision stage's results)
    of the plain, substep and fused forms are bitwise equal, so are the
    gradients."""
    sc, cfg, tg, nsteps, g4 = diff_case
    assert not g4["status"].any() and np.abs(g4["tg"]).max() > 0
    for kw in (dict(exec_form="plain"), dict(exec_form="substep"), dict(exec_form="fused", threads_per_env=16)):
        gk = _gpu_grads(sc, cfg, tg, nsteps, 4, **kw)
        for key in ("v", "w", "tg", "m"):
            assert np.array_equal(gk[key], g4[key]), (kw, key)


def test_backward_through_c_abi_directly():
    """msh_backward on a recorded step; the adjoint of the start state for a
    linear seed equals the step's Jacobian transpose applied to it, checked
    against a central difference of the GPU step itself along a random
    direction (free bodies only: a clean linear map)."""
    import torch
    from paper_2412_13211_b300.sim import MshSim
    from helpers import env, scene_from_envs
    e = env()
    e.body(S.BOX, (0.05, 0.04, 0.03), 0.8, (0.0, 0.0, 5.0), linvel=(0.1, 0.2, 0.3), angvel=(1.0, -0.5, 0.25))
    e.body(S.SPHERE, (0.05,), 0.5, (1.0, 0.0, 5.0), linvel=(0.0, 0.0, -1.0))
    sc = scene_from_envs([e])
    cfg = S.SolverCfg(substeps=2, iterations=3)
    sim = MshSim(sc, cfg)
    sim.set_tape(1)
    sim.step()
    assert sim.tape_count == 1
    rng = np.random.default_rng(0)
    seed = [torch.tensor(rng.normal(size=a.shape).astype(np.float32), device="cuda") for a in sc.state()]
    adj = sim.backward(seed)
    assert sim.tape_count == 0
    # <seed, d out> = <adj, d in> for the velocity direction (positions respond linearly)
    d = rng.normal(size=(2, 3))
    outs = []
    for sgn in (1.0, -1.0):
        s2 = MshSim(sc, cfg)
        lv = sc.linvel.astype(np.float64) + sgn * 1e-3 * d
        s2.set_state(sc.pos, sc.quat, lv.astype(np.float32), sc.angvel)
        s2.step()
        outs.append([x.astype(np.float64) for x in s2.state_numpy()])
    dout = [(a - b) / 2e-3 for a, b in zip(*outs)]
    lhs = sum(float((s.cpu().numpy().astype(np.float64) * o).sum()) for s, o in zip(seed, dout))
    rhs = float((adj[2].cpu().numpy().astype(np.float64) * d).sum())
    assert abs(lhs - rhs) <= 1e-3 * abs(lhs) + 1e-4


def test_steps_after_backward_do_not_record():
    import torch
    from paper_2412_13211_b300.autograd import goal_loss, rollout
    from paper_2412_13211_b300.sim import MshSim
    sc, cfg = S.make_config(4, num_envs=4)
    sim = MshSim(sc, cfg)
    st = [torch.tensor(np.asarray(a, np.float32), device="cuda", requires_grad=True) for a in sc.state()]
    mass = torch.tensor(np.asarray(sc.body_mass, np.float32), device="cuda", requires_grad=True)
    tg = torch.tensor(sc.target_walk(4), device="cuda", requires_grad=True)
    out = rollout(sim, st, tg, mass, 2)
    goal_loss(sim, out[0]).sum().backward()
    for _ in range(20):
        sim.step(tg[0].detach())
    assert sim.tape_count == 0
    sim.set_tape(-1)


def test_forward_pass_keeps_the_last_segment_for_the_backward_pass():
    """The forward pass records its last segment and pauses the tape: steps in
    between are not recorded, and the gradients equal those of a backward
    pass that re-runs every segment (forced by touching the tape)."""
    import torch
    from paper_2412_13211_b300.autograd import goal_loss, rollout
    from paper_2412_13211_b300.sim import MshSim
    sc, cfg = S.make_config(4, num_envs=4)
    tgn = sc.target_walk(5)
    grads = []
    for touch in (False, True):
        sim = MshSim(sc, cfg)
        st = [torch.tensor(np.asarray(a, np.float32), device="cuda", requires_grad=True) for a in sc.state()]
        mass = torch.tensor(np.asarray(sc.body_mass, np.float32), device="cuda", requires_grad=True)
        tg = torch.tensor(tgn, device="cuda", requires_grad=True)
        out = rollout(sim, st, tg, mass, 2)
        assert sim.tape_count == 1                      # the last segment (step 4) is kept
        loss = goal_loss(sim, out[0]).sum()
        if touch:
            sim.tape_reset()                            # the backward pass must re-run it
        else:
            snap = tuple(x.clone() for x in (sim.pos, sim.quat, sim.linvel, sim.angvel))
            sim.step(tg[0].detach())                    # paused: not recorded
            assert sim.tape_count == 1
            for x, y in zip((sim.pos, sim.quat, sim.linvel, sim.angvel), snap):
                x.copy_(y)
        loss.backward()
        grads.append([t.grad.cpu().numpy() for t in (st[2], st[3], tg, mass)])
        assert sim.tape_count == 0
        sim.close()
    for a, b in zip(*grads):
        assert np.array_equal(a, b)
