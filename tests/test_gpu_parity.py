"""Parity of the CUDA step (through the C ABI) with the CPU oracle.

Tolerances: the collision stage (AABBs, pairs, contacts, colours) is bit-exact
against the FP32 oracle from identical poses; body states agree within 1e-5 m
and 1e-4 m/s after one step and within 1e-3 m after 100 steps on envs that
are not chaotic (a 1e-7 m FP64 perturbation grows by less than 1e-4 m over
the horizon, and the FP32 oracle stays within 1e-4 m of the FP64 one). The forms of the step (plain per-stage launches, fused
persistent launch, CUDA graph, threads per env) agree bit for bit.
"""
import numpy as np
import pytest

import oracle
from paper_2412_13211_b300 import scenes as S

pytestmark = pytest.mark.gpu

SMALL = {1: 16, 2: 8, 3: 16, 4: 8, 5: 6, 6: 8}
TOL_X, TOL_V = 1e-5, 1e-4

_cache = {}


def scene(idx, n=None, **cfg_over):
    key = (idx, n)
    if key not in _cache:
        _cache[key] = S.make_config(idx, num_envs=n if n is not None else SMALL[idx])
    sc, cfg = _cache[key]
    cfg = S.SolverCfg(**{**cfg.__dict__, **cfg_over})
    return sc, cfg


def make_sim(sc, cfg, **kw):
    from paper_2412_13211_b300.sim import MshSim
    return MshSim(sc, cfg, **kw)


def bits(a):
    return np.ascontiguousarray(a, np.float32).view(np.int32)


def oracle_states(sc, cfg, steps):
    """Poses reached by the FP32 oracle after 0, steps/2, steps steps."""
    st = sc.state()
    out = [st]
    tg = sc.target_walk(steps)
    half = steps // 2
    a, _ = oracle.step(sc, cfg, st, tg[:half], half, "f32")
    b, _ = oracle.step(sc, cfg, a, tg[half:], steps - half, "f32")
    return out + [a, b]


@pytest.mark.parametrize("idx", [1, 2, 3, 4, 5, 6])
def test_collision_stage_bit_exact(idx):
    sc, cfg = scene(idx)
    sim = make_sim(sc, cfg)
    for st in oracle_states(sc, cfg, 20):
        sim.set_state(*st)
        g = sim.detect()
        o = oracle.detect(sc, cfg, st[0], st[1], "f32")
        assert np.array_equal(bits(g["aabb_body"]), bits(o.aabb_body))
        assert np.array_equal(bits(g["aabb_static"]), bits(o.aabb_static))
        assert np.array_equal(g["pair_count"], o.pair_count)
        assert np.array_equal(g["contact_count"], o.contact_count)
        assert np.array_equal(g["manifold_count"], o.manifold_count)
        assert np.array_equal(g["ncolours"], o.ncolours)
        for e in range(sc.num_envs):
            npair, nc = o.pair_count[e], o.contact_count[e]
            assert np.array_equal(g["pairs"][e, :npair], o.pairs[e, :npair])
            assert np.array_equal(g["contact_ids"][e, :nc], o.contact_ids[e, :nc])
            assert np.array_equal(bits(g["contact_geom"][e, :nc]), bits(o.contact_geom[e, :nc]))
        J = sc.num_joints
        assert np.array_equal(g["colours"][:J], o.colours[:J])
        for e in range(sc.num_envs):
            m = o.manifold_count[e]
            sl = slice(J + e * cfg.max_pairs, J + e * cfg.max_pairs + m)
            assert np.array_equal(g["colours"][sl], o.colours[sl])
    assert (o.contact_count > 0).any()


def _step_both(sc, cfg, nsteps, seed=0, **kw):
    tg = sc.target_walk(nsteps, seed)
    sim = make_sim(sc, cfg, **kw)
    import torch
    for t in range(nsteps):
        sim.step(torch.as_tensor(tg[t]).cuda())
    gpu = sim.state_numpy()
    status = sim.status()
    o32, st32 = oracle.step(sc, cfg, sc.state(), tg, nsteps, "f32")
    o64, _ = oracle.step(sc, cfg, sc.state(), tg, nsteps, "f64")
    return gpu, o32, o64, status, st32


def _err(a, b):
    return float(np.abs(np.asarray(a, np.float64) - np.asarray(b, np.float64)).max()) if np.size(a) else 0.0


@pytest.mark.parametrize("mode", [S.MODE_COLOURED, S.MODE_JACOBI])
@pytest.mark.parametrize("idx", [1, 2, 3, 4, 5, 6])
def test_one_step_parity(idx, mode, record_property):
    sc, cfg = scene(idx, mode=mode)
    gpu, o32, o64, status, st32 = _step_both(sc, cfg, 1)
    assert np.array_equal(status, st32)
    ex, eq, ev, ew = (_err(gpu[k], o32[k]) for k in range(4))
    record_property("err_vs_fp32", [ex, eq, ev, ew])
    record_property("err_vs_fp64", [_err(gpu[k], o64[k]) for k in range(4)])
    record_property("err_fp32_vs_fp64", [_err(o32[k], o64[k]) for k in range(4)])
    assert ex <= TOL_X and eq <= TOL_X
    assert ev <= TOL_V and ew <= TOL_V


def _non_chaotic(sc, cfg, tg, steps):
    """Envs that are insensitive to rounding over the horizon: a 1e-7 m FP64
    perturbation of every body position coordinate (seeded random signs)
    grows by less than 1e-4 m, and the FP32 oracle stays within 1e-4 m of the
    FP64 oracle."""
    a, _ = oracle.step(sc, cfg, sc.state(), tg, steps, "f64")
    st = sc.state()
    sign = np.random.default_rng(12345).choice([-1.0, 1.0], size=st[0].shape)
    pert = (st[0].astype(np.float64) + 1e-7 * sign, st[1], st[2], st[3])
    b, _ = oracle.step(sc, cfg, pert, tg, steps, "f64")
    c, _ = oracle.step(sc, cfg, sc.state(), tg, steps, "f32")
    d = np.maximum(np.abs(a[0] - b[0]).max(axis=1), np.abs(a[0] - c[0]).max(axis=1))
    return np.array([d[sc.body_off[e]:sc.body_off[e + 1]].max() < 1e-4 for e in range(sc.num_envs)])


def _errs(sc, envs, a, b):
    """Max |a - b| over the given envs' bodies, for x, q, v and omega."""
    idx = np.concatenate([np.arange(sc.body_off[e], sc.body_off[e + 1]) for e in envs]) if len(envs) else []
    return [_err(a[k][idx], b[k][idx]) for k in range(4)]


@pytest.mark.parametrize("idx", [1, 2, 3, 4, 5, 6])
def test_hundred_steps_non_chaotic(idx, record_property):
    """After 100 steps the non-chaotic envs are within 1e-3 m of the FP32
    oracle; the errors against the FP64 oracle (and the FP32 oracle's own
    against it) are recorded beside them."""
    sc, cfg = scene(idx)
    steps = 100
    tg = sc.target_walk(steps)
    calm = _non_chaotic(sc, cfg, tg, steps)
    record_property("non_chaotic_envs", f"{int(calm.sum())}/{sc.num_envs}")
    assert calm.sum() >= 1
    gpu, o32, o64, status, _ = _step_both(sc, cfg, steps)
    envs = np.nonzero(calm)[0]
    record_property("err100_gpu_vs_fp32", _errs(sc, envs, gpu, o32))
    record_property("err100_gpu_vs_fp64", _errs(sc, envs, gpu, o64))
    record_property("err100_fp32_vs_fp64", _errs(sc, envs, o32, o64))
    for e in envs:
        sl = slice(sc.body_off[e], sc.body_off[e + 1])
        assert _err(gpu[0][sl], o32[0][sl]) <= 1e-3, e
    assert not (status & 8).any()


@pytest.mark.parametrize("idx", [2, 3, 6])
def test_plain_fused_graph_and_block_sizes_bitwise_equal(idx):
    sc, cfg = scene(idx)
    import torch
    tg = sc.target_walk(3)
    results = []
    for kw in (dict(exec_form="fused"), dict(exec_form="plain"), dict(exec_form="fused", use_graph=True),
               dict(exec_form="plain", use_graph=True), dict(exec_form="substep"),
               dict(exec_form="substep", use_graph=True, threads_per_env=64),
               dict(exec_form="fused", threads_per_env=64), dict(exec_form="fused", threads_per_env=128),
               dict(exec_form="fused", threads_per_env=256), dict(exec_form="fused", threads_per_env=16),
               dict(exec_form="fused", threads_per_env=8, use_graph=True)):
        sim = make_sim(sc, cfg, **kw)
        for t in range(3):
            sim.step(torch.as_tensor(tg[t]).cuda())
        results.append(sim.state_numpy())
        sim.close()
    for r in results[1:]:
        for a, b in zip(results[0], r):
            assert np.array_equal(bits(a), bits(b))


def test_host_buffer_step_equals_device_step():
    sc, cfg = scene(3)
    import torch
    tg = sc.target_walk(2)
    sim = make_sim(sc, cfg)
    for t in range(2):
        sim.step(torch.as_tensor(tg[t]).cuda())
    dev = sim.state_numpy()
    host = [np.ascontiguousarray(a, np.float32).copy() for a in sc.state()]
    sim2 = make_sim(sc, cfg)
    for t in range(2):
        sim2.step_host(*host, np.ascontiguousarray(tg[t]))
    for a, b in zip(dev, host):
        assert np.array_equal(bits(a), bits(b))


FULL_ENVS = {1: 64, 2: 1024, 3: 4096, 4: 512, 5: 16384, 6: 4096}
FULL_HORIZON = {1: 100, 2: 100, 3: 100, 4: 100, 5: 100, 6: 100}


@pytest.mark.parametrize("idx", [1, 2, 3, 4, 5, 6])
def test_full_size_batch_sampled(idx, record_property):
    """Each configuration at its full batch size in the launch the benchmark
    times (autotuned form, CUDA graph): the whole batch status-clean and
    finite; sampled envs (random ones plus the largest and the smallest)
    within the one-step tolerances of the FP32 oracle, and, over a horizon,
    the sampled envs that are not chaotic within 1e-3 m."""
    import torch
    from paper_2412_13211_b300 import autotune
    sc, cfg = scene(idx, FULL_ENVS[idx])
    H = FULL_HORIZON[idx]
    tg = sc.target_walk(H)
    t0 = torch.as_tensor(tg[0]).cuda()
    sim = make_sim(sc, cfg, use_graph=True)
    tuning = autotune.tune(sim, t0, steps=2, warmup=1)
    record_property("form", tuning["best"])
    sim.set_state(*sc.state())
    sim.clear_status()
    sim.step(t0)
    one = sim.state_numpy()
    assert not sim.status().any()
    for t in range(1, H):
        sim.step(torch.as_tensor(tg[t]).cuda())
    last = sim.state_numpy()
    status = sim.status()
    assert not (status & 8).any()
    assert all(np.isfinite(a).all() for a in last)
    sim.close()

    rng = np.random.default_rng(idx)
    counts = np.diff(sc.body_off)
    sample = np.unique(np.concatenate([rng.choice(sc.num_envs, min(32, sc.num_envs), replace=False),
                                       [int(np.argmax(counts)), int(np.argmin(counts))]]))
    sub = sc.subset(sample)
    o1, _ = oracle.step(sub, cfg, sub.state(), tg[:1, sample], 1, "f32")
    o1d, _ = oracle.step(sub, cfg, sub.state(), tg[:1, sample], 1, "f64")
    oH, stH = oracle.step(sub, cfg, sub.state(), tg[:, sample], H, "f32")
    oHd, _ = oracle.step(sub, cfg, sub.state(), tg[:, sample], H, "f64")
    calm = _non_chaotic(sub, cfg, tg[:, sample], H)
    record_property("non_chaotic_sampled_envs", f"{int(calm.sum())}/{len(sample)}")
    gidx = np.concatenate([np.arange(sc.body_off[e], sc.body_off[e + 1]) for e in sample])
    g1 = [a[gidx] for a in one]
    gH = [a[gidx] for a in last]
    allk = range(len(sample))
    calmk = np.nonzero(calm)[0]
    record_property("err1_gpu_vs_fp32", _errs(sub, allk, g1, o1))
    record_property("err1_gpu_vs_fp64", _errs(sub, allk, g1, o1d))
    record_property("err1_fp32_vs_fp64", _errs(sub, allk, o1, o1d))
    record_property("err100_gpu_vs_fp32", _errs(sub, calmk, gH, oH))
    record_property("err100_gpu_vs_fp64", _errs(sub, calmk, gH, oHd))
    record_property("err100_fp32_vs_fp64", _errs(sub, calmk, oH, oHd))
    assert np.array_equal(status[sample][calm], stH[calm])
    for k, e in enumerate(sample):
        g = slice(sc.body_off[e], sc.body_off[e + 1])
        o = slice(sub.body_off[k], sub.body_off[k + 1])
        assert _err(one[0][g], o1[0][o]) <= TOL_X, e
        assert _err(one[1][g], o1[1][o]) <= TOL_X, e
        assert _err(one[2][g], o1[2][o]) <= TOL_V, e
        assert _err(one[3][g], o1[3][o]) <= TOL_V, e
        if calm[k]:
            assert _err(last[0][g], oH[0][o]) <= 1e-3, e
    assert calm.sum() >= 1


def test_capacity_overflow_sets_status_and_truncates_like_oracle():
    sc, cfg = scene(2, max_contacts=12, max_pairs=10)
    sim = make_sim(sc, cfg)
    g = sim.detect()
    o = oracle.detect(sc, cfg, sc.pos, sc.quat, "f32")
    assert np.array_equal(g["pair_count"], o.pair_count)
    assert np.array_equal(g["contact_count"], o.contact_count)
    assert (o.status & 1).any()
    import torch
    sim.step(torch.zeros((sc.num_envs, sc.max_dof)).cuda())
    st = sim.status()
    _, ost = oracle.step(sc, cfg, sc.state(), None, 1, "f32")
    assert np.array_equal(st, ost)
    assert (st & 1).any()


def test_nonfinite_state_sets_status_without_trap():
    sc, cfg = scene(1)
    sim = make_sim(sc, cfg)
    pos = sc.pos.copy()
    pos[sc.body_off[3]] = np.nan
    sim.set_state(pos, sc.quat, sc.linvel, sc.angvel)
    sim.step()
    st = sim.status()
    assert st[3] & 8
    assert not (np.delete(st, 3) & 8).any()
    sim.clear_status()
    assert not sim.status().any()


def test_degenerate_envs():
    """Env with one body and nothing else, env with no contacts (free flight),
    env with only statics nearby, joint-only env."""
    from helpers import env, scene_from_envs
    envs = []
    e = env(); e.body(S.SPHERE, (0.05,), 1.0, (0.0, 0.0, 3.0)); envs.append(e)
    e = env(); e.body(S.BOX, (0.1, 0.1, 0.1), 1.0, (0.0, 0.0, 0.1)); e.static((0.5, 0.0, 0.2), (0.2, 0.2, 0.2))
    envs.append(e)
    e = env()
    e.body(S.CAPSULE, (0.03, 0.1), 1.0, (0.0, 0.0, 1.0 + 0.1), S.Q_LINK)
    e.joint(S.REVOLUTE, -1, 0, (0.0, 0.0, 1.0) + S.QW_AXIS_Z, (-0.1, 0.0, 0.0) + S.QL_AXIS_Z, S.ARM_GAINS,
            (0.0, 0.0), [(0.0, 0.0, -3, 3)])
    envs.append(e)
    sc = scene_from_envs(envs)
    cfg = S.SolverCfg(substeps=4, iterations=8)
    gpu, o32, _, status, st32 = _step_both(sc, cfg, 3)
    assert np.array_equal(status, st32)
    assert _err(gpu[0], o32[0]) <= TOL_X and _err(gpu[2], o32[2]) <= TOL_V


def test_autotuner_picks_a_form_and_keeps_state():
    import torch
    from paper_2412_13211_b300 import autotune
    sc, cfg = scene(3)
    sim = make_sim(sc, cfg)
    before = sim.state_numpy()
    res = autotune.tune(sim, steps=2, warmup=1)
    after = sim.state_numpy()
    for a, b in zip(before, after):
        assert np.array_equal(bits(a), bits(b))
    assert res["best"][0] in ("fused", "substep", "plain") and len(res["ms"]) >= 3
    assert (sim.exec_form, sim.threads_per_env) == tuple(res["best"])
    sim.step(torch.zeros((sc.num_envs, sc.max_dof)).cuda())
    assert not sim.status().any()


def test_handles_with_different_workspaces_coexist():
    """A second handle with a smaller workspace must not break the first one's
    fused launches (kernel attributes are shared by all handles)."""
    import torch
    big_sc, big_cfg = scene(3)
    small_sc, small_cfg = scene(4)
    big = make_sim(big_sc, big_cfg)
    small = make_sim(small_sc, small_cfg)
    assert small.workspace_bytes < big.workspace_bytes
    big.step(torch.zeros((big_sc.num_envs, big_sc.max_dof)).cuda())
    small.step(torch.zeros((small_sc.num_envs, small_sc.max_dof)).cuda())
    small.close()
    big.step(torch.zeros((big_sc.num_envs, big_sc.max_dof)).cuda())
    assert not big.status().any()


def test_maximum_capacities_use_the_device_memory_workspace():
    """At the largest capacities (1024 contacts, 4096 pairs per env) one env's
    workspace takes 171 KB of shared memory (one env per SM); two envs per
    warp exceed it and the fused form runs on device-memory slabs. Both stay
    bitwise equal to the plain form and within the one-step tolerance of the
    oracle."""
    import torch
    sc, cfg = scene(2, max_contacts=1024, max_pairs=4096)
    tg = sc.target_walk(2)
    res = []
    for kw in (dict(exec_form="fused"), dict(exec_form="fused", threads_per_env=16), dict(exec_form="plain")):
        sim = make_sim(sc, cfg, **kw)
        assert sim.workspace_bytes > 113 * 1024      # two exceed the 227 KB of one CTA
        for t in range(2):
            sim.step(torch.as_tensor(tg[t]).cuda())
        res.append(sim.state_numpy())
        assert not sim.status().any()
        sim.close()
    for r in res[1:]:
        for a, b in zip(res[0], r):
            assert np.array_equal(bits(a), bits(b))
    o32, _ = oracle.step(sc, cfg, sc.state(), tg, 2, "f32")
    assert _err(res[0][0], o32[0]) <= 2 * TOL_X and _err(res[0][2], o32[2]) <= 2 * TOL_V


def test_empty_envs_in_a_batch():
    """Envs without any body (statics only, or nothing at all) between
    ordinary ones: they step as no-ops and leave their neighbours intact."""
    from helpers import env, scene_from_envs
    envs = []
    e = env(); e.body(S.SPHERE, (0.05,), 1.0, (0.0, 0.0, 0.049)); envs.append(e)
    envs.append(env())
    e = env(); e.static((0.0, 0.0, 0.5), (0.2, 0.2, 0.5)); envs.append(e)
    e = env(); e.body(S.BOX, (0.05, 0.05, 0.05), 1.0, (0.0, 0.0, 0.3)); envs.append(e)
    sc = scene_from_envs(envs)
    cfg = S.SolverCfg(substeps=2, iterations=8)
    gpu, o32, _, status, st32 = _step_both(sc, cfg, 3)
    assert np.array_equal(status, st32) and not status.any()
    assert _err(gpu[0], o32[0]) <= TOL_X and _err(gpu[2], o32[2]) <= TOL_V


def test_chunked_host_step_equals_device_step():
    """Large batches step from host buffers in env chunks whose copies overlap
    the other chunks' launches: bitwise the device step, report included."""
    import torch
    sc, cfg = S.make_config(3, num_envs=1536)
    tg = sc.target_walk(2)
    sim = make_sim(sc, cfg)
    sim.set_report(*sc.report_spec())
    for t in range(2):
        sim.step(torch.as_tensor(tg[t]).cuda())
    dev = sim.state_numpy()
    rep_dev = sim.report()
    host = [np.ascontiguousarray(a, np.float32).copy() for a in sc.state()]
    sim2 = make_sim(sc, cfg)
    sim2.set_report(*sc.report_spec())
    for t in range(2):
        sim2.step_host(*host, np.ascontiguousarray(tg[t]))
    for a, b in zip(dev, host):
        assert np.array_equal(bits(a), bits(b))
    rep_host = sim2.report()
    for k in rep_dev:
        assert np.array_equal(np.asarray(rep_dev[k]).view(np.int32), np.asarray(rep_host[k]).view(np.int32)), k
    assert not sim2.status().any()


@pytest.mark.parametrize("mode", [S.MODE_COLOURED, S.MODE_JACOBI])
@pytest.mark.parametrize("idx", [1, 2, 3, 4, 5, 6])
def test_recorded_impulses_match_oracle_per_sweep(idx, mode, record_property):
    """The impulses a recorded step holds after every sweep of every substep
    (msh_tape_lambdas) against the FP32 oracle's, row by row, from the FP32
    oracle's state after 30 steps: within 1e-3 of the env's largest impulse
    plus 1e-3 of the row's own. The regrouped per-point update and the fused
    multiply-adds round differently, and on a statically indeterminate
    contact set (a box on four points) the split of the load among the rows
    is not unique, so rounding differences along it are not damped."""
    import torch
    sc, cfg = scene(idx, mode=mode)
    tg = sc.target_walk(31)
    x30, _ = oracle.step(sc, cfg, sc.state(), tg[:30], 30, "f32")
    sim = make_sim(sc, cfg)
    sim.set_state(*x30)
    sim.set_tape(1)
    sim.step(torch.as_tensor(tg[30]).cuda())
    got = sim.tape_lambdas(0)
    sim.set_tape(-1)
    _, ref = oracle.step_lambdas(sc, cfg, x30, tg[30])
    assert got.shape == ref.shape
    used = np.isfinite(ref)
    assert used.any()
    worst = 0.0
    for e in range(sc.num_envs):
        r, g, m = ref[e], got[e], used[e]
        if not m.any():
            continue
        tol = 1e-3 * np.abs(r[m]).max() + 1e-3 * np.abs(r[m])
        worst = max(worst, float((np.abs(g[m] - r[m]) / np.maximum(tol, 1e-30)).max()))
    record_property("worst_ratio", worst)
    assert worst <= 1.0, worst


@pytest.mark.parametrize("mode", [S.MODE_COLOURED, S.MODE_JACOBI])
def test_one_step_parity_with_restitution(mode, record_property):
    """Restitution 0.5 (reading C5: contacts approaching faster than 1 m/s
    target the rebound e * v_n): one step of the falling-sphere scene from the
    FP32 oracle's state after 25 steps, when spheres strike the boxes and the
    plane at 1-4 m/s, within the one-step tolerances of the FP32 oracle; the
    oracle's own step with e = 0 differs, so restitution acted."""
    sc, cfg = scene(1, 64, mode=mode, restitution=0.5)
    x25, _ = oracle.step(sc, cfg, sc.state(), None, 25, "f32")
    sim = make_sim(sc, cfg)
    sim.set_state(*x25)
    sim.step()
    gpu = sim.state_numpy()
    o32, st = oracle.step(sc, cfg, x25, None, 1, "f32")
    plain, _ = oracle.step(sc, S.SolverCfg(**{**cfg.__dict__, "restitution": 0.0}), x25, None, 1, "f32")
    assert _err(o32[2], plain[2]) > 0.1
    assert np.array_equal(sim.status(), st)
    ex, ev = _err(gpu[0], o32[0]), _err(gpu[2], o32[2])
    record_property("err_vs_fp32", [ex, ev])
    assert ex <= TOL_X and _err(gpu[1], o32[1]) <= TOL_X
    assert ev <= TOL_V and _err(gpu[3], o32[3]) <= TOL_V
