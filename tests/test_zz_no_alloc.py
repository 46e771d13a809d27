"""tensorsketch_apply_static_scratch: the entry point that allocates nothing.

Some callers cannot allocate device memory when they call in (a plug-in inside an
application whose framework owns the device memory, a latency-critical path that
cannot afford cudaMalloc's implicit synchronisation).  This variant keeps its
scratch in a fixed device array inside the library.  It must agree with
tensorsketch_apply (caller scratch) on consecutive calls, whatever the previous
call left in the shared array.  This file is collected last on purpose.
"""

import numpy as np
import pytest
import torch

from oracle import rng

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ts():
    from paper_2104_01101_gb300 import build, tsketch
    build.build_library()
    tsketch.lib()
    return tsketch


def _case(dims, ranks, m, dtype, seed):
    g = np.random.default_rng(seed)
    facs = [torch.from_numpy(np.linalg.qr(g.standard_normal((s, R)))[0]).to(dtype).cuda()
            for s, R in zip(dims, ranks)]
    tabs = [torch.from_numpy(rng.pack_table(*rng.hash_table(seed, 1, 0, 0, j, s, m))).cuda()
            for j, s in enumerate(dims)]
    return facs, tabs


@pytest.mark.parametrize("dtype,tol", [(torch.float32, 1e-5), (torch.float64, 1e-12)])
def test_static_scratch_matches_caller_scratch_on_consecutive_calls(ts, dtype, tol):
    # two calls in a row with different shapes: the second must not see the first's leftovers
    cases = [((400, 400), (10, 10), 2000), ((33, 29, 17), (3, 4, 2), 210)]
    for i, (dims, ranks, m) in enumerate(cases):
        facs, tabs = _case(dims, ranks, m, dtype, seed=10 + i)
        want = ts.tensorsketch_apply(facs, tabs, m)
        got = ts.tensorsketch_apply_static_scratch(facs, tabs, m)
        torch.cuda.synchronize()
        err = float(torch.linalg.norm(got - want) / torch.linalg.norm(want))
        assert err <= tol, (dims, err)
    # and the first shape again, after the second one used the array
    facs, tabs = _case(*cases[0][:2], cases[0][2], dtype, seed=10)
    want = ts.tensorsketch_apply(facs, tabs, cases[0][2])
    got = ts.tensorsketch_apply_static_scratch(facs, tabs, cases[0][2])
    torch.cuda.synchronize()
    assert float(torch.linalg.norm(got - want) / torch.linalg.norm(want)) <= tol


def test_static_scratch_rejects_problems_beyond_its_capacity(ts):
    cap = int(ts.lib().tensorsketch_apply_static_scratch_capacity())
    assert cap == 8 << 20
    # FP32, m = 12288, 48 + 48 factor columns: 12288 * (1 + 96) * 8 bytes = 9.5 MB > 8 MiB
    facs2, tabs2 = _case((64, 64), (48, 48), 12288, torch.float32, seed=3)
    with pytest.raises(ts.TsError) as e:
        ts.tensorsketch_apply_static_scratch(facs2, tabs2, 12288)
    assert e.value.status == 3
    assert "fixed" in str(e.value)
