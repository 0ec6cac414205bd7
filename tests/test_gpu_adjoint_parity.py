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
only remaining decisions are the impulse clamps (active at an exact tie on
both sides). A clamp whose row has converged onto its bound (a friction row
on its cone, a normal impulse at zero) is still decided within rounding, and
the two solvers round differently; the oracle reports such fragile
decisions, and an env whose adjoint differs from the oracle's own piece must
agree element by element with the piece reached by re-deciding some of them
(tests/adjoint_pieces.py). No env is left out.

Every element of the adjoints of positions, velocities, angular velocities,
joint targets and masses is compared; for the quaternion only its component
tangent to the unit sphere is unique (the step is defined on unit
quaternions, and the two sides may extend their formulas off the sphere
differently), so that part is compared. The tolerance of an element
(adjoint_pieces.env_ratio) is 2e-3 of its own size plus 2e-3 of the largest
element of its kind in the same env plus 1e-5 of the env's largest element
of any kind: an FP32 adjoint through N sweeps against a double-precision one.

Inputs: the oracle's own FP32 trajectory (the GPU is given the oracle's
state at each compared step, every position moved by a seeded 1e-6 m so that
no resting contact sits exactly on the kink at s = 0; see off_kink), seeded
random seeds, and for the differentiation workload the goal loss's adjoints
chained back over its whole horizon by the oracle.
"""
import numpy as np
import pytest

import oracle
from paper_2412_13211_b300 import scenes as S

pytestmark = pytest.mark.gpu

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


def check_batch(sc, cfg, state, targets, seed, ref, got, stats):
    """Every env: the GPU adjoint against the oracle's own piece, else against
    a piece reached by re-deciding fragile decisions (adjoint_pieces).
    Updates stats (envs, direct, redecided, max_flips, worst) and returns the
    worst final ratio with its env."""
    import adjoint_pieces as AP
    worst = (0.0, None)
    for e in range(sc.num_envs):
        b0, b1 = sc.body_off[e], sc.body_off[e + 1]
        g = {k: (got[k][e] if k == "targets" else got[k][b0:b1]) for k in KINDS}
        r = {k: (ref[k][e] if k == "targets" else ref[k][b0:b1]) for k in KINDS}
        q, _ = AP.env_ratio(r, g, state[1][b0:b1])
        stats["envs"] += 1
        if q <= 1.0:
            stats["direct"] += 1
        else:
            sub = sc.subset(np.array([e]))
            xs = [a[b0:b1] for a in state]
            ws = [a[b0:b1] for a in seed]
            us = None if targets is None else targets[e:e + 1]
            q, flips = AP.check_env(sub, cfg, xs, us, ws, g)
            if q <= 1.0:
                stats["redecided"] += 1
                stats["max_flips"] = max(stats["max_flips"], len(flips))
        if q > worst[0]:
            worst = (q, e)
    stats["worst"] = max(stats["worst"], worst[0])
    return worst


def new_stats():
    return dict(envs=0, direct=0, redecided=0, max_flips=0, worst=0.0)


def record(record_property, stats):
    for k, v in stats.items():
        record_property(k, v)


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


def off_kink(state, rng):
    """The state with every position coordinate moved by a seeded 1e-6 m: a
    contact that the previous step brought to rest lands exactly on the kink
    of its bias at s = 0 (to 1e-17 m), where the step is not differentiable;
    the offset moves it clear of the kink by far more than any rounding."""
    pos = np.asarray(state[0], np.float32) + rng.uniform(-1e-6, 1e-6, size=np.shape(state[0])).astype(np.float32)
    return (pos,) + tuple(state[1:])


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
    stats = new_stats()
    bad = []
    for t in steps:
        w = random_seed(sc, rng)
        u = tg[t] if sc.max_dof else None
        x = off_kink(xs[t], rng)
        ref, r = oracle_vjp(sc, cfg, x, u, w)
        got = gpu_vjp(sim, x, u, w)
        q, e = check_batch(sc, cfg, x, u, w, ref, got, stats)
        if q > 1.0:
            bad.append((t, e, q))
    record(record_property, stats)
    assert not sim.status().any()
    sim.close()
    assert not bad, bad


def test_differentiation_workload_rollout_adjoint_elementwise(record_property):
    """The differentiation workload (512 envs, arm pushing a box), its 64-step
    horizon at 4 substeps run as 256 one-substep steps with each step's
    targets held for 4 steps: the oracle chains the goal loss's adjoint back
    over all 256 steps along its FP32 trajectory; at every step the GPU,
    given the oracle's state (moved off the kinks, see off_kink) and the
    oracle's adjoint of the step's output, must return the oracle's adjoint
    of the step's input, targets and masses."""
    from paper_2412_13211_b300.sim import MshSim
    sc, cfg = one_substep(4, 512)
    T = 256
    tg = np.repeat(sc.target_walk(T // 4), 4, axis=0)
    seed = lambda x: oracle.goal_seed(sc, x[0], sc.goal_body, sc.goal_pos)
    xs, st = oracle.trajectory(sc, cfg, sc.state(), tg, T)
    assert not st.any()
    sim = MshSim(sc, cfg)
    w = seed(xs[T])
    stats = new_stats()
    bad = []
    nonzero = 0
    rng = np.random.default_rng(4)
    for t in range(T - 1, -1, -1):
        x = off_kink(xs[t], rng)
        ref, r = oracle_vjp(sc, cfg, x, tg[t], w)
        got = gpu_vjp(sim, x, tg[t], w)
        q, e = check_batch(sc, cfg, x, tg[t], w, ref, got, stats)
        if q > 1.0:
            bad.append((t, e, q))
        w = [r.pos, r.quat, r.linvel, r.angvel]
        nonzero = max(nonzero, int((np.abs(r.targets).max(axis=1) > 0).sum()))
    record(record_property, stats)
    record_property("envs_with_target_gradient", nonzero)
    assert nonzero >= 256
    assert not sim.status().any()
    sim.close()
    assert not bad, bad[:5]


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
    xT = off_kink(xs[T], rng)
    full = [np.array(a, np.float32) for a in sc.state()]
    for j, e in enumerate(pick):
        b0, b1 = sc.body_off[e], sc.body_off[e + 1]
        s0 = sub.body_off[j]
        for k in range(4):
            full[k][b0:b1] = xT[k][s0:s0 + (b1 - b0)]
    w = random_seed(sc, rng)
    wsub = [np.concatenate([a[sc.body_off[e]:sc.body_off[e + 1]] for e in pick]) for a in w]
    ref, _ = oracle_vjp(sub, cfg, xT, tg[T][pick], wsub)
    sim = MshSim(sc, cfg)
    got_full = gpu_vjp(sim, full, tg[T], w)
    idx_b = np.concatenate([np.arange(sc.body_off[e], sc.body_off[e + 1]) for e in pick])
    got = {k: (v[pick] if k == "targets" else v[idx_b]) for k, v in got_full.items()}
    stats = new_stats()
    q, e = check_batch(sub, cfg, xT, tg[T][pick], wsub, ref, got, stats)
    record(record_property, stats)
    assert not sim.status().any()
    sim.close()
    assert q <= 1.0, (q, e)


@pytest.mark.parametrize("mode", [0, 1], ids=["coloured", "jacobi"])
def test_multi_substep_adjoint_without_contacts(mode, record_property):
    """Four substeps per step where no decision sits on a kink: the
    manipulator scene with its counter moved far away and its objects spread
    apart far from the arm (no contact; joints with soft drives), so the
    substeps' poses differ only smoothly between the two sides. Checks the
    reverse over substeps (tape replay per substep, the pose and velocity
    adjoints carried from one substep to the one before) element by
    element."""
    from paper_2412_13211_b300.sim import MshSim
    sc, cfg = S.make_config(2, num_envs=8)
    cfg.mode = mode
    sc.static_pose[:, 0] += 1000.0
    st = [a.copy() for a in sc.state()]
    for e in range(sc.num_envs):
        b = np.arange(sc.body_off[e], sc.body_off[e + 1])
        st[0][b[9:], 0] += 100.0 + 2.0 * np.arange(1, len(b) - 8)
    tg = sc.target_walk(13)
    xs, status = oracle.trajectory(sc, cfg, st, tg, 12)
    assert not status.any()
    for t in (0, 12):
        assert oracle.detect(sc, cfg, xs[t][0], xs[t][1]).contact_count.sum() == 0
    sim = MshSim(sc, cfg)
    rng = np.random.default_rng(mode)
    stats = new_stats()
    bad = []
    for t in (0, 6, 12):
        w = random_seed(sc, rng)
        ref, _ = oracle_vjp(sc, cfg, xs[t], tg[t], w)
        got = gpu_vjp(sim, xs[t], tg[t], w)
        q, e = check_batch(sc, cfg, xs[t], tg[t], w, ref, got, stats)
        if q > 1.0:
            bad.append((t, e, q))
    record(record_property, stats)
    sim.close()
    assert not bad, bad
