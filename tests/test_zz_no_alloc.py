"""The allocation-free emission entry point gives the same results as the allocating one.

pic_emission_eval_noalloc exists for callers that cannot take device memory (a process whose
device memory belongs to another framework's pool, or a latency-bound loop that cannot afford
cudaFree's device-wide synchronisation); it stages through a fixed array inside the library.
This file is collected last so that a failure here comes after every other test has run.
"""
import os

import numpy as np
import pytest

from paper_2402_08404_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sim():
    from paper_2402_08404_gb300 import _build
    if not os.path.exists(_build.LIB):
        _build.build()
    from paper_2402_08404_gb300 import pic
    cfg = dict(synth.CONFIGS["small"])
    s = pic.Pic(cfg, capacity=16, V0=20.0)
    yield s
    s.close()


def test_noalloc_matches_allocating_entry_point_twice(sim):
    # two calls in a row with different inputs: the shared staging array must not leak
    # anything from the first call into the second
    for seed, n in ((3, 3000), (4, 1700)):
        F, T, W, R = synth.face_tuples(n, seed=seed)
        R = np.where(np.arange(n) % 4 == 0, -1.0, R * 1e-9)
        J_ref, P_ref = sim.emission_eval(F * 1e9, T, W, R)
        J, P = sim.emission_eval_noalloc(F * 1e9, T, W, R)
        assert np.all(np.isfinite(J)) and np.all(np.isfinite(P))
        assert np.allclose(J, J_ref, rtol=1e-12, atol=0.0)
        assert np.allclose(P, P_ref, rtol=1e-12, atol=1e-30)


def test_noalloc_at_its_full_size(sim):
    # n equal to the array's size: the last slot of every staged sub-array is used
    n = 32768
    F, T, W, R = synth.face_tuples(n, seed=9)
    R = np.where(np.arange(n) % 5 == 0, -1.0, R * 1e-9)
    J_ref, P_ref = sim.emission_eval(F * 1e9, T, W, R)
    J, P = sim.emission_eval_noalloc(F * 1e9, T, W, R)
    assert np.allclose(J, J_ref, rtol=1e-12, atol=0.0)
    assert np.allclose(P, P_ref, rtol=1e-12, atol=1e-30)
    assert J[-1] == J_ref[-1] and P[-1] == P_ref[-1]


def test_noalloc_rejects_sizes_beyond_its_array(sim):
    from paper_2402_08404_gb300 import pic
    n = 32768 + 1
    with pytest.raises(pic.PicError) as e:
        sim.emission_eval_noalloc(np.full(n, 5e9), np.full(n, 300.0), np.full(n, 4.5), np.full(n, -1.0))
    assert e.value.code == pic.PIC_E_INVALID and "exceeds" in str(e.value)
