"""The CUDA depth cameras (msh_render_depth) against the oracle.

Both sides evaluate the same closed forms in IEEE FP32 without FMA
contraction in the same operation order, and the kernel's per-tile culling is
conservative, so depth images must agree bit for bit: every config's scenes
(world, base and hand mounted cameras), after stepping, at 128 x 128 (4 x 4
tiles) and at a ragged size that leaves partial tiles.
"""
import numpy as np
import pytest

import oracle
from paper_2412_13211_b300 import scenes as S

pytestmark = pytest.mark.gpu
FOV, NEAR, FAR = np.pi / 2, 0.01, 10.0


def _focal(H):
    """The library's focal length: (H/2) / tan(fov/2) in double from the f32 field of view, then f32."""
    return float(np.float32(H * 0.5 / np.tan(float(np.float32(FOV)) * 0.5)))


def _gpu(sc, cfg, tg, steps, W, H, body, pose):
    import torch
    from paper_2412_13211_b300.sim import MshSim
    sim = MshSim(sc, cfg)
    t = torch.as_tensor(tg).cuda() if tg is not None else None
    for k in range(steps):
        sim.step(t[k] if t is not None else None)
    sim.set_cameras(body, pose, W, H, FOV, NEAR, FAR)
    d = sim.render_depth().cpu().numpy()
    st = sim.state_numpy()
    sim.close()
    return d, st


@pytest.mark.parametrize("idx,envs,W,H", [(1, 8, 128, 128), (2, 4, 128, 128), (3, 6, 128, 128), (4, 4, 70, 45),
                                          (5, 3, 96, 128), (6, 3, 128, 128)])
def test_depth_matches_oracle_bitwise(idx, envs, W, H):
    sc, cfg = S.make_config(idx, num_envs=envs)
    tg = sc.target_walk(3) if sc.max_dof > 0 else None
    body, pose = sc.camera_mounts()
    d, st = _gpu(sc, cfg, tg, 3, W, H, body, pose)
    ref = oracle.render_depth(sc, st[0], st[1], body, pose, W, H, _focal(H), NEAR, FAR, "f32")
    assert d.shape == ref.shape
    hit = ref > 0
    assert hit.mean() > 0.2                       # the cameras see something
    assert np.array_equal(d.view(np.int32), ref.view(np.int32)), np.argwhere(d != ref)[:5]


def test_cameras_argument_checks():
    import ctypes as C
    from paper_2412_13211_b300 import _lib
    from paper_2412_13211_b300.sim import MshSim
    sc, cfg = S.make_config(1, num_envs=2)
    sim = MshSim(sc, cfg)
    body, pose = sc.camera_mounts()
    with pytest.raises(RuntimeError):
        sim.set_cameras(body, pose, 0, 128)
    with pytest.raises(RuntimeError):
        sim.set_cameras(body, pose, 128, 128, fov_y=4.0)
    bad = body.copy()
    bad[0, 0] = 99
    with pytest.raises(RuntimeError):
        sim.set_cameras(bad, pose)
    lib = _lib.load()
    st = sim._state()
    assert lib.msh_render_depth(sim.handle, C.byref(st), None, None) == _lib.MSH_ERR_INVALID_ARG
    sim.close()
