"""Emission surrogate on the GPU: forward/backward of the BF16 tensor-core MLP against the FP64
oracle MLP on the same (BF16-rounded) weights, then training on the full integral and the
held-out accuracy |dlog10 J| of the installed network against the oracle's integral."""
import math

import numpy as np
import pytest

from oracle import emission as em, mlp
from paper_2402_08404_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sim():
    import os
    from paper_2402_08404_gb300 import _build
    if not os.path.exists(_build.LIB):
        _build.build()
    from paper_2402_08404_gb300 import pic
    s = pic.Pic(dict(synth.CONFIGS["small"]), capacity=16, V0=20.0)
    yield s
    s.close()


def bf16(a):
    """Round float32 values to bfloat16 (nearest even), returned as float64."""
    u = np.asarray(a, dtype=np.float32).view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def unflatten(p):
    out, q = [], 0
    for a, b in zip(mlp.SIZES[:-1], mlp.SIZES[1:]):
        W = p[q:q + a * b].reshape(b, a); q += a * b
        c = p[q:q + b]; q += b
        out.append((W, c))
    return out


def test_mlp_forward_backward_matches_fp64_oracle(sim):
    rng = np.random.default_rng(0)
    params = mlp.init_params(rng)
    flat = np.concatenate([np.concatenate([W.ravel(), b]) for W, b in params]).astype(np.float32)
    flat[np.r_[256:320, 4416:4480, 8576:8640, 8768:8770]] = rng.normal(0, 0.1, 64 * 3 + 2)   # nonzero biases
    sim.set_mlp_params(flat)
    assert np.array_equal(sim.mlp_params(), flat)
    x = rng.normal(size=(1000, 4)).astype(np.float32)
    t = rng.normal(size=(1000, 2)).astype(np.float32)
    y, loss, g = sim.mlp_forward_backward(x, t)
    # oracle on the BF16 operands the tensor cores see (weights and inputs), in float64
    ref = [(bf16(W), b.astype(np.float64)) for W, b in unflatten(flat.astype(np.float64))]
    yr, _ = mlp.forward(ref, bf16(x))
    lr_, gr = mlp.loss_and_grad(ref, bf16(x), t.astype(np.float64))
    assert np.linalg.norm(y - yr) <= 1e-2 * np.linalg.norm(yr)
    assert loss == pytest.approx(lr_, rel=2e-2)
    gflat = np.concatenate([np.concatenate([gW.ravel(), gb]) for gW, gb in gr])
    gg = unflatten(g.astype(np.float64))
    for li, ((gW, gb), (rW, rb)) in enumerate(zip(gg, gr)):
        assert np.linalg.norm(gW - rW) <= 3e-2 * np.linalg.norm(rW), li
        assert np.linalg.norm(gb - rb) <= 3e-2 * np.linalg.norm(rb), li
    assert np.linalg.norm(g - gflat) <= 3e-2 * np.linalg.norm(gflat)


def test_surrogate_trains_to_the_integral(sim):
    st = sim.surrogate_train(nsamples=1_000_000, epochs=150, batch=8192, lr=3e-3, seed=3)
    print("surrogate training:", st)
    assert st["valid_sample_fraction"] > 0.3, st
    # fresh tuples over the surrogate workload ranges (F 3.5-15 GV/m, T, phi_w, R 1-20 nm)
    F, T, W, R = synth.face_tuples(9000, seed=21)
    keep = np.nonzero(F >= 3.5)[0][:3000]          # the part of the range where faces emit
    F, T, W, R = F[keep], T[keep], W[keep], R[keep]
    J, P, valid = sim.surrogate_eval(F * 1e9, T, W, R * 1e-9)
    Jr, Pr = em.current_density_fixed(F, T, W, R)
    lj_r = np.log10(np.maximum(Jr, 1e-300))
    lj = np.log10(np.maximum(J, 1e-300))
    rel = valid & (np.maximum(lj, lj_r) >= -5)
    assert rel.sum() > 500, (rel.sum(), st)
    err = np.abs(lj[rel] - lj_r[rel])
    assert np.quantile(err, 0.99) <= 0.02, (np.quantile(err, [0.5, 0.9, 0.99]), err.max(), st)
    assert err.max() <= 0.05
    # Nottingham heat follows the integral where J is relevant
    big = rel & (Jr > 1e6)
    assert np.median(np.abs(P[big] - Pr[big]) / (np.abs(Pr[big]) + Jr[big] * 0.05)) < 0.05
