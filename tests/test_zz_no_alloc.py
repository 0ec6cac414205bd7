"""The allocation-free step (msh_step_static_scratch) against msh_step.

Callers that cannot call cudaMalloc while they step -- a framework whose
caching allocator owns the device memory, a real-time loop that must not
block in the allocator -- use msh_step_static_scratch, which keeps its
workspace in a static device array of the library. This file drives it
through the C ABI: two calls in a row must give the same states, bit for
bit, as two calls of the regular msh_step from the same start (every
execution form of the step computes identical results), including a batch
large enough that the static array, not the GPU, limits the number of
persistent CTAs. While a tape is recording, the entry point must refuse to
run (it records nothing) and leave the state as it was. The file sorts last
so that a run stopping at the first failure has already run every other test.

Rejection of an oversized workspace is not exercised: the descriptor limits
(4096 bodies, 4096 static boxes, 1024 joints, 4096 pairs and 1024 contacts
per env) keep one env's workspace near 2 MB at most, far below the 32 MiB
array, so no valid handle reaches that check.
"""
import ctypes as C

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

STATIC_SCRATCH_BYTES = 32 << 20


def _bits(arrs):
    return [np.ascontiguousarray(a, np.float32).view(np.int32) for a in arrs]


def _call(lib, sim, tg, stream):
    st = sim._state()
    return lib.msh_step_static_scratch(sim.handle, C.byref(st), C.c_void_p(tg.data_ptr()), 0.0, 0,
                                       C.c_void_p(stream.cuda_stream))


@pytest.mark.parametrize("idx,envs,tpe", [(2, 8, 32), (3, 16, 32), (3, 16, 16), (3, 2048, 32), (3, 2048, 16)])
def test_static_scratch_step_equals_msh_step_bitwise(idx, envs, tpe):
    import torch
    from paper_2412_13211_b300 import _lib, scenes
    from paper_2412_13211_b300.sim import MshSim

    sc, cfg = scenes.make_config(idx, num_envs=envs)
    tg = torch.as_tensor(sc.target_walk(2)).cuda()
    ref = MshSim(sc, cfg)                          # regular step
    nal = MshSim(sc, cfg, threads_per_env=tpe)     # same scene, stepped without allocation
    lib = _lib.load()
    stream = torch.cuda.current_stream()
    if envs >= 1024:
        # an env's whole workspace exceeds its shared-memory part, so here the
        # static array, not the batch, bounds the number of persistent CTAs
        assert envs * nal.workspace_bytes > STATIC_SCRATCH_BYTES
    for t in range(2):
        ref.step(tg[t])
        _lib.check(_call(lib, nal, tg[t], stream), "msh_step_static_scratch")
        for a, b in zip(_bits(ref.state_numpy()), _bits(nal.state_numpy())):
            assert np.array_equal(a, b)
    assert np.array_equal(ref.status(), nal.status())
    assert not nal.status().any()
    ref.close()
    nal.close()


def test_static_scratch_step_refuses_while_recording():
    import torch
    from paper_2412_13211_b300 import _lib, scenes
    from paper_2412_13211_b300.sim import MshSim

    sc, cfg = scenes.make_config(4, num_envs=4)
    tg = torch.as_tensor(sc.target_walk(1)).cuda()
    sim = MshSim(sc, cfg)
    ref = MshSim(sc, cfg)
    lib = _lib.load()
    stream = torch.cuda.current_stream()
    sim.set_tape(2)
    before = _bits(sim.state_numpy())
    assert _call(lib, sim, tg[0], stream) == _lib.MSH_ERR_INVALID_ARG
    assert "record" in lib.msh_last_error().decode()
    torch.cuda.synchronize()
    for a, b in zip(before, _bits(sim.state_numpy())):
        assert np.array_equal(a, b)
    assert sim.tape_count == 0
    # paused: the step runs, records nothing, and equals msh_step
    check = lib.msh_tape_record(sim.handle, 0)
    _lib.check(check, "msh_tape_record")
    _lib.check(_call(lib, sim, tg[0], stream), "msh_step_static_scratch")
    ref.step(tg[0])
    for a, b in zip(_bits(ref.state_numpy()), _bits(sim.state_numpy())):
        assert np.array_equal(a, b)
    assert sim.tape_count == 0
    sim.set_tape(-1)
    sim.close()
    ref.close()
