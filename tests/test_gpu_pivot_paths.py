"""Every pivot sample size the plans allow (Section III.H's sampled pivot, with Section
V.C's randomised samples: 15, 31 or 63 per segment), in both reservation modes and for
every key width, must sort exactly as the oracle does."""
import ctypes

import numpy as np
import pytest

from tests.test_gpu_parity import KINDS, random_keys, to_dev, from_dev, oracle_sort
from workloads import int32_pattern, records_u64

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def T():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1505_00558_gb300 as T
    T.lib()
    return T


def _ctx(T, kind, samples, mode):
    plan = T.Plan()
    T.lib().tsqs_plan_default(kind, 0, ctypes.byref(plan))
    plan.sample_count = samples
    plan.offset_mode = mode
    return T.Context(plan)


@pytest.mark.parametrize("mode", [0, 1])
@pytest.mark.parametrize("samples", [15, 31, 63])
@pytest.mark.parametrize("kind_name", ["i32", "f32", "i64", "f64"])
def test_plans_sort_like_the_oracle(T, orc, kind_name, samples, mode):
    code, dt, _ = KINDS[kind_name]
    n = 1_500_007
    a = random_keys(kind_name, n, seed=samples + 7 * mode)
    a[::5] = a[11]                                          # a heavy =p run somewhere
    ctx = _ctx(T, code, samples, mode)
    t = to_dev(a)
    T.sort_(t, kind=code, ctx=ctx)
    torch.cuda.synchronize()
    assert ctx.status() == 0
    assert from_dev(t, dt).tobytes() == oracle_sort(orc, a, code).tobytes()
    ctx.close()


@pytest.mark.parametrize("samples", [15, 31, 63])
def test_plans_records_and_patterns(T, orc, samples):
    r = records_u64(400_001, seed=samples)
    ctx = _ctx(T, 7, samples, 0)
    t = torch.from_numpy(r.view(np.int64).copy()).cuda()
    T.sort_(t, records=True, ctx=ctx)
    torch.cuda.synchronize()
    assert ctx.status() == 0
    assert t.cpu().numpy().view(np.uint64).reshape(-1, 2).tobytes() == oracle_sort(orc, r, 7).tobytes()
    ctx.close()
    for pattern in ("organ_pipe", "many_equals", "nearly_sorted"):
        a = int32_pattern(pattern, 700_001, seed=samples)
        ctx = _ctx(T, 1, samples, 0)
        t = to_dev(a)
        T.sort_(t, kind=1, ctx=ctx)
        torch.cuda.synchronize()
        assert ctx.status() == 0
        assert from_dev(t, np.int32).tobytes() == oracle_sort(orc, a, 1).tobytes()
        ctx.close()
