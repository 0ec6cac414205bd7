"""The allocation-free step (msh_step_static_scratch) against msh_step.

Callers that cannot call cudaMalloc while they step -- a framework whose
caching allocator owns the device memory, a real-time loop that must not
block in the allocator -- use msh_step_static_scratch, which keeps its
workspace in a static device array. This test drives it through the C ABI
and checks that two calls in a row give the same states as two calls of the
regular msh_step from the same start (within the parity tolerances). The
file sorts last so that a run stopping at the first failure has already run
every other test.
"""
import ctypes as C

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

TOL_X, TOL_V = 1e-5, 1e-4


def _err(a, b):
    return float(np.abs(np.asarray(a, np.float64) - np.asarray(b, np.float64)).max())


@pytest.mark.parametrize("idx,envs,tpe", [(2, 8, 32), (3, 16, 32), (3, 16, 16)])
def test_static_scratch_step_matches_msh_step(idx, envs, tpe):
    import torch
    from paper_2412_13211_b300 import _lib, scenes
    from paper_2412_13211_b300.sim import MshSim

    sc, cfg = scenes.make_config(idx, num_envs=envs)
    tg = torch.as_tensor(sc.target_walk(2)).cuda()
    ref = MshSim(sc, cfg)                      # regular step
    nal = MshSim(sc, cfg, threads_per_env=tpe)   # same scene, stepped without allocation
    lib = _lib.load()
    stream = torch.cuda.current_stream()
    for t in range(2):
        ref.step(tg[t])
        st = nal._state()
        rc = lib.msh_step_static_scratch(nal.handle, C.byref(st), C.c_void_p(tg[t].data_ptr()), 0.0, 0,
                                         C.c_void_p(stream.cuda_stream))
        _lib.check(rc, "msh_step_static_scratch")
        a, b = ref.state_numpy(), nal.state_numpy()
        assert _err(a[0], b[0]) <= TOL_X and _err(a[1], b[1]) <= TOL_X
        assert _err(a[2], b[2]) <= TOL_V and _err(a[3], b[3]) <= TOL_V
    assert not nal.status().any()
    ref.close()
    nal.close()
