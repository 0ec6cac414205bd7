"""The CUDA adjoint of one step (msh_backward) against the oracle, element by
element.

For a step from state x with joint targets u and masses m, the GPU records
the step and reverses it for a seed w on the stepped state; the oracle's
reverse mode (oracle.step_vjp, FP32 primal arithmetic as the FP32 oracle,
adjoints in double) computes w^T dx'/d(x, u, m) from the same FP32 inputs.

The step is piecewise smooth, and both sides differentiate the piece their
own primal values select. Resting contacts sit exactly on a kink of the
contact bias (speculative s/h above s = 0, nothing down to -slop, Baumgarte
below): a contact that lands is stopped at s = 0 to rounding. From the
second substep of a step on, the two sides' poses differ in the last bits
(the solvers round differently), so they pick different pieces there and
both derivatives are correct one-sided ones. The comparisons therefore run
the configurations' scenes with one substep per step (dt = the configured
substep, the configured iterations): every branch of the row set-up and of
the collision stage is then decided on identical FP32 start poses, and the
only remaining decisions, the impulse clamps, count as active at an exact tie
on both sides.

Every element of the adjoints of positions, velocities, angular velocities,
joint targets and masses is compared; for the quaternion only its component
tangent to the unit sphere is unique (the step is defined on unit
quaternions, and the two sides may extend their formulas off the sphere
differently), so that part is compared. The tolerance of an element is
RTOL of its own size plus ATOL of the largest element of its kind in the
same env plus FLOOR of the largest of its kind in the batch (an FP32 adjoint
through N sweeps against a double-precision one).

Inputs: the oracle's own FP32 trajectory (the GPU is given the oracle's
state at each compared step), seeded random seeds, and for the
differentiation workload the goal loss's adjoints chained back over its
whole horizon by the oracle.
"""
import numpy as np
import pytest

import oracle
from paper_2412_13211_b300 import scenes as S

pytestmark = pytest.mark.gpu

RTOL, ATOL, FLOOR = 2e-3, 2e-3, 1e-6
KINDS = ("pos", "quat", "linvel", "angvel", "targets", "mass")


def gpu_vjp(sim, state, targets, seed):
    """Records one step from `state` and reverses it for `seed`."""
    import torch
    dev = sim.device
    sim.set_state(*state)
    sim.set_tape(1)
    sim.step(None if targets is None else torch.as_tensor(np.asarray(targets, np.float32)).to(dev))
    E, md = sim.scene.num_envs, max(sim.scene.max_dof, 1)
    adj_tg = torch.zeros((E, md), dtype=torch.float32, device=dev)
    adj_m = torch.zeros(max(sim.scene.num_bodies, 1), dtype=torch.float32, device=dev)
    w = [torch.as_tensor(np.asarray(a, np.float32)).to(dev) for a in seed]
    adj = sim.backward(w, adj_tg, adj_m)
    torch.cuda.synchronize(dev)
    out = dict(pos=adj[0].cpu().numpy(), quat=adj[1].cpu().numpy(), linvel=adj[2].cpu().numpy(),
               angvel=adj[3].cpu().numpy(), targets=adj_tg.cpu().numpy()[:, :sim.scene.max_dof],
               mass=adj_m.cpu().numpy()[:sim.scene.num_bodies])
    assert sim.tape_count == 0
    return out


def tangential(g, q):
    q = np.asarray(q, np.float64)
    q = q / np.linalg.norm(q, axis=1, keepdims=True)
    return g - (g * q).sum(1, keepdims=True) * q


def compare(sc, envs, ref, got, quat):
    """Worst ratio of |got - ref| to its tolerance over the given envs and
    every kind; returns (ratio, where)."""
    ref = dict(ref)
    got = dict(got)
    ref["quat"] = tangential(ref["quat"], quat)
    got["quat"] = tangential(np.asarray(got["quat"], np.float64), quat)
    worst, where = 0.0, None
    floor = {k: FLOOR * float(np.abs(np.asarray(ref[k], np.float64)).max(initial=0.0)) for k in KINDS}
    for e in envs:
        b0, b1 = sc.body_off[e], sc.body_off[e + 1]
        for k in KINDS:
            if k == "targets":
                if sc.max_dof == 0:
                    continue
                r, g = ref[k][e], got[k][e]
            else:
                r, g = ref[k][b0:b1], got[k][b0:b1]
            r = np.asarray(r, np.float64)
            g = np.asarray(g, np.float64)
            if r.size == 0:
                continue
            tol = RTOL * np.abs(r) + ATOL * np.abs(r).max() + floor[k] + 1e-30
            ratio = float((np.abs(g - r) / tol).max())
            if ratio > worst or not np.isfinite(ratio):
                worst, where = ratio, (int(e), k)
    return worst, where


def oracle_vjp(sc, cfg, state, targets, seed):
    r = oracle.step_vjp(sc, cfg, state, targets, seed, "f32")
    return dict(pos=r.pos, quat=r.quat, linvel=r.linvel, angvel=r.angvel, targets=r.targets, mass=r.mass), r


def one_substep(idx, envs):
    """Configuration idx with one substep per step of the configured substep
    length (same h, same iterations)."""
    sc, cfg = S.make_config(idx, num_envs=envs)
    cfg.dt = cfg.dt / cfg.substeps
    cfg.substeps = 1
    return sc, cfg


def random_seed(sc, rng):
    B = sc.num_bodies
    return [rng.normal(size=(B, 3)), rng.normal(size=(B, 4)), rng.normal(size=(B, 3)), rng.normal(size=(B, 3))]


@pytest.mark.parametrize("idx,envs,mode", [(1, 64, 0), (2, 64, 0), (3, 64, 0), (4, 128, 0), (5, 32, 0), (6, 32, 0),
                                           (1, 64, 1), (2, 64, 1), (3, 64, 1), (4, 128, 1)])
def test_step_adjoint_elementwise(idx, envs, mode, record_property):
    """Random seeds at steps 0, 4 and 12 of the oracle's trajectory, in the
    coloured (mode 0) and the mass-split Jacobi (mode 1) solver."""
    from paper_2412_13211_b300.sim import MshSim
    sc, cfg = one_substep(idx, envs)
    cfg.mode = mode
    steps = (0, 4, 12, 40)
    tg = sc.target_walk(max(steps) + 1)
    xs, st = oracle.trajectory(sc, cfg, sc.state(), tg if sc.max_dof else None, max(steps))
    assert not st.any()
    sim = MshSim(sc, cfg)
    rng = np.random.default_rng(idx)
    worst = (0.0, None)
    for t in steps:
        w = random_seed(sc, rng)
        u = tg[t] if sc.max_dof else None
        ref, r = oracle_vjp(sc, cfg, xs[t], u, w)
        got = gpu_vjp(sim, xs[t], u, w)
        ratio, where = compare(sc, range(sc.num_envs), ref, got, xs[t][1])
        if ratio >= worst[0]:
            worst = (ratio, (t,) + (where or ()))
    record_property("worst_ratio", worst[0])
    record_property("worst_at", str(worst[1]))
    assert not sim.status().any()
    sim.close()
    assert worst[0] <= 1.0, worst


def test_differentiation_workload_rollout_adjoint_elementwise(record_property):
    """The differentiation workload (512 envs, arm pushing a box), its 64-step
    horizon at 4 substeps run as 256 one-substep steps with each step's
    targets held for 4 steps: the oracle chains the goal loss's adjoint back
    over all 256 steps along its FP32 trajectory; at every step the GPU,
    given the oracle's state and the oracle's adjoint of the step's output,
    must return the oracle's adjoint of the step's input, targets and
    masses."""
    from paper_2412_13211_b300.sim import MshSim
    sc, cfg = one_substep(4, 512)
    T = 256
    tg = np.repeat(sc.target_walk(T // 4), 4, axis=0)
    seed = lambda x: oracle.goal_seed(sc, x[0], sc.goal_body, sc.goal_pos)
    xs, st = oracle.trajectory(sc, cfg, sc.state(), tg, T)
    assert not st.any()
    sim = MshSim(sc, cfg)
    w = seed(xs[T])
    worst = (0.0, None)
    nonzero = 0
    for t in range(T - 1, -1, -1):
        ref, r = oracle_vjp(sc, cfg, xs[t], tg[t], w)
        got = gpu_vjp(sim, xs[t], tg[t], w)
        ratio, where = compare(sc, range(sc.num_envs), ref, got, xs[t][1])
        if ratio >= worst[0]:
            worst = (ratio, (t,) + (where or ()))
        w = [r.pos, r.quat, r.linvel, r.angvel]
        nonzero = max(nonzero, int((np.abs(r.targets).max(axis=1) > 0).sum()))
    record_property("worst_ratio", worst[0])
    record_property("worst_at", str(worst[1]))
    record_property("envs_with_target_gradient", nonzero)
    assert nonzero >= 256
    assert not sim.status().any()
    sim.close()
    assert worst[0] <= 1.0, worst


def _sample(sc, n_random, rng):
    nb = np.diff(sc.body_off)
    ns = np.diff(sc.static_off)
    cost = nb * (nb + ns)
    pick = {int(np.argmax(cost)), int(np.argmin(cost))}
    pick |= set(int(i) for i in rng.choice(sc.num_envs, n_random, replace=False))
    return np.array(sorted(pick))


@pytest.mark.parametrize("idx,envs", [(3, 4096), (5, 16384)])
def test_full_size_batch_sampled_step_adjoint(idx, envs, record_property):
    """The full batch on the GPU, in the launch configuration of its size
    (two envs per warp in the reversed sweeps, rows in device memory): the
    sampled envs (the costliest, the cheapest, random ones) start from the
    oracle's state after 32 steps, the others from the initial state; their
    adjoints are compared element by element (one substep per step, as
    above)."""
    from paper_2412_13211_b300.sim import MshSim
    sc, cfg = one_substep(idx, envs)
    rng = np.random.default_rng(idx + 100)
    pick = _sample(sc, 10, rng)
    sub = sc.subset(pick)
    T = 32
    tg = sc.target_walk(T + 1)
    xs, st = oracle.trajectory(sub, cfg, sub.state(), tg[:, pick], T)
    assert not st.any()
    full = [np.array(a, np.float32) for a in sc.state()]
    for j, e in enumerate(pick):
        b0, b1 = sc.body_off[e], sc.body_off[e + 1]
        s0 = sub.body_off[j]
        for k in range(4):
            full[k][b0:b1] = xs[T][k][s0:s0 + (b1 - b0)]
    w = random_seed(sc, rng)
    wsub = [np.concatenate([a[sc.body_off[e]:sc.body_off[e + 1]] for e in pick]) for a in w]
    ref, _ = oracle_vjp(sub, cfg, xs[T], tg[T][pick], wsub)
    sim = MshSim(sc, cfg)
    got_full = gpu_vjp(sim, full, tg[T], w)
    idx_b = np.concatenate([np.arange(sc.body_off[e], sc.body_off[e + 1]) for e in pick])
    got = {k: (v[pick] if k == "targets" else v[idx_b]) for k, v in got_full.items()}
    ratio, where = compare(sub, range(sub.num_envs), ref, got, xs[T][1])
    record_property("sampled_envs", len(pick))
    record_property("worst_ratio", ratio)
    record_property("worst_at", str(where))
    assert not sim.status().any()
    sim.close()
    assert ratio <= 1.0, (ratio, where)


@pytest.mark.parametrize("mode", [0, 1], ids=["coloured", "jacobi"])
def test_multi_substep_adjoint_without_contacts(mode, record_property):
    """Four substeps per step where no decision sits on a kink: the
    manipulator scene lifted 5 m into the air with its objects spread apart
    (no contact; joints with soft drives), so the substeps' poses differ only
    smoothly between the two sides. Checks the reverse over substeps (tape
    replay per substep, the pose and velocity adjoints carried from one
    substep to the one before) element by element."""
    from paper_2412_13211_b300.sim import MshSim
    sc, cfg = S.make_config(2, num_envs=8)
    cfg.mode = mode
    st = [a.copy() for a in sc.state()]
    st[0][:, 2] += 5.0
    for e in range(sc.num_envs):
        b = np.arange(sc.body_off[e], sc.body_off[e + 1])
        st[0][b[9:], 0] += 2.0 * np.arange(1, len(b) - 8)
    tg = sc.target_walk(13)
    xs, status = oracle.trajectory(sc, cfg, st, tg, 12)
    assert not status.any()
    for t in (0, 12):
        assert oracle.detect(sc, cfg, xs[t][0], xs[t][1]).contact_count.sum() == 0
    sim = MshSim(sc, cfg)
    rng = np.random.default_rng(mode)
    worst = (0.0, None)
    for t in (0, 6, 12):
        w = random_seed(sc, rng)
        ref, _ = oracle_vjp(sc, cfg, xs[t], tg[t], w)
        got = gpu_vjp(sim, xs[t], tg[t], w)
        ratio, where = compare(sc, range(sc.num_envs), ref, got, xs[t][1])
        if ratio >= worst[0]:
            worst = (ratio, (t,) + (where or ()))
    record_property("worst_ratio", worst[0])
    record_property("worst_at", str(worst[1]))
    sim.close()
    assert worst[0] <= 1.0, worst
