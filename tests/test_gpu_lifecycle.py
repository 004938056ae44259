"""Handle life cycle on the GPU: checkpoint and resume of the online state,
and an injected device-allocation failure (the failure is made on the host:
nothing faults or hangs the GPU)."""
import os

import numpy as np
import pytest

from paper_2312_08684_gb300 import Estimator, _binding as abi, workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    abi.load()
    return torch


def _steps(est, wl, t0, t1):
    for t in range(t0, t1):
        est.step(np.ascontiguousarray(wl.y[:, t]), active=(wl.T > t).astype(np.uint8))


@pytest.mark.parametrize("make", [
    lambda: W.make_clutter_cv(B=4, Tmin=8, Tmax=14, N=40, L=4),
    lambda: W.make_planar_arm(B=2, T=10, N=24, L=3),
])
def test_resume_from_a_checkpoint_gives_the_same_bits(torch, make):
    """Half the steps, save, the other half: a fresh handle that loads the
    checkpoint and runs the other half ends with the same MAP paths and J,
    bit for bit; the saved handle itself is unchanged by the save."""
    wl = make()
    half = wl.maxT // 2
    with Estimator.from_workload(wl) as a:
        _steps(a, wl, 0, half)
        size = abi.smap_state_size(a.h)
        state = abi.smap_save(a.h)
        assert state.nbytes == size
        _steps(a, wl, half, wl.maxT)
        path_a, J_a = a.map_sequence()
        hist_a = a.history()
    with Estimator.from_workload(wl) as b:
        abi.smap_load(b.h, state)
        steps = np.empty(wl.B, np.int32)
        abi.smap_get_steps(b.h, steps)
        assert np.array_equal(steps, np.minimum(wl.T, half))
        _steps(b, wl, half, wl.maxT)
        path_b, J_b = b.map_sequence()
        hist_b = b.history()
    assert np.array_equal(np.nan_to_num(path_a, nan=1e30), np.nan_to_num(path_b, nan=1e30))
    assert np.array_equal(J_a, J_b)
    for s in range(wl.B):
        T = int(wl.T[s])
        assert np.array_equal(hist_a[s, :T], hist_b[s, :T])


def test_checkpoint_of_another_configuration_is_rejected(torch):
    wl = W.make_range_cv(B=2, T=6, N=32, L=2, dropout=None)
    with Estimator.from_workload(wl) as a:
        _steps(a, wl, 0, 3)
        state = abi.smap_save(a.h)
    for over in ({"N": 48}, {"L": 3}, {"seed": 99}):
        with Estimator.from_workload(wl, **over) as b:
            with pytest.raises(abi.SmapError) as e:
                abi.smap_load(b.h, state)
            assert e.value.status == abi.SMAP_E_INVAL
    with Estimator.from_workload(wl) as b:
        with pytest.raises(abi.SmapError) as e:
            abi.smap_load(b.h, state[: state.nbytes // 2])
        assert e.value.status == abi.SMAP_E_INVAL
        abi.smap_load(b.h, state)       # the handle is still usable


@pytest.mark.parametrize("k", [1, 5, 18])
def test_injected_allocation_failure(torch, monkeypatch, k):
    """SMAP_FAIL_ALLOC=k fails the k-th device allocation of smap_create:
    SMAP_E_NOMEM, no handle, nothing left allocated; without the variable the
    same configuration is created and runs."""
    wl = W.make_range_cv(B=64, T=50, N=128, L=2, dropout=None)
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    monkeypatch.setenv("SMAP_FAIL_ALLOC", str(k))
    with pytest.raises(abi.SmapError) as e:
        Estimator.from_workload(wl)
    assert e.value.status == abi.SMAP_E_NOMEM
    monkeypatch.delenv("SMAP_FAIL_ALLOC")
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 >= free0 - (2 << 20)        # the partial allocations were freed
    with Estimator.from_workload(wl) as est:
        path, J = est.run_batch(wl.y)
    assert np.all(np.isfinite(J))
