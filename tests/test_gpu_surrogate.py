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
    s = pic.Pic(dict(synth.CONFIGS["small"]), capacity=200_000, V0=20.0)
    yield s
    s.close()


def unflatten(p):
    out, q = [], 0
    for a, b in zip(mlp.SIZES[:-1], mlp.SIZES[1:]):
        W = p[q:q + a * b].reshape(b, a); q += a * b
        c = p[q:q + b]; q += b
        out.append((W, c))
    return out


def bf16_params(flat):
    """The operands the GPU holds: BF16 weights in the two hidden (tensor-core) layers, FP32
    weights in the input and output layers."""
    return [(mlp.bf16(W) if li in mlp.BF16_LAYERS else W, b)
            for li, (W, b) in enumerate(unflatten(flat.astype(np.float64)))]


def output_bound(ref, x):
    """Per-element bound on |y_gpu - y_oracle| for the BF16-operand network, in units of the
    output's scale S (the absolute sum of the output layer's terms, plus that of the last hidden
    layer's terms carried through |W4| and the GELU slope bound 1.13): 2e-6 S from FP32
    accumulation (a few units of 2^-24 per term over 128-term sums), and 3e-5 S in rows where an
    activation fed to a BF16 layer lies so close to a rounding boundary that the GPU's FP32 value
    of it may round to the neighbouring BF16 value (one BF16 step of one of 128 activations moves
    the output by far less than 3e-5 S)."""
    out, cache = mlp.forward(ref, x, bf16_operands=True)
    (W1, b1), (W2, b2), (W3, b3), (W4, b4) = ref
    a2, a3 = cache[2][0], cache[3][0]                    # BF16 input of layer 2, FP32-kept input of layer 3
    z3_scale = np.abs(a2) @ np.abs(W3).T + np.abs(b3)
    scale = np.abs(a3) @ np.abs(W4).T + np.abs(b4) + (1.13 * z3_scale) @ np.abs(W4).T
    rows = mlp.bf16_ambiguous_rows(ref, x)
    return np.where(rows[:, None], 3e-5, 2e-6) * scale, out


def grad_bounds(ref, x, t):
    """Per-entry bounds on the weight and bias gradients.  With G the absolute sum of an entry's
    terms (one per row) and T its largest term: 2e-5 G for FP32 accumulation over the rows, plus
    2^-5 T for BF16 roundings that go the other way on the GPU (a rounded operand that differs by
    one BF16 step, 2^-7 relative, changes its term by at most 2^-7 T; four such steps)."""
    out, cache = mlp.forward(ref, x, bf16_operands=True)
    d = (out - t) / len(x)
    res = [None] * len(ref)
    for li in range(len(ref) - 1, -1, -1):
        h, z = cache[li]
        if li < len(ref) - 1:
            d = d * mlp.gelu_grad(z)
        dm = mlp.bf16(d) if li in mlp.BF16_LAYERS else d
        ad, ah = np.abs(dm), np.abs(h)
        G = ad.T @ ah
        T = np.max(ad[:, :, None] * ah[:, None, :], axis=0)
        Gb = np.abs(d).sum(axis=0)
        Tb = np.abs(d).max(axis=0)
        res[li] = (2e-5 * G + 2.0 ** -5 * T, 2e-5 * Gb + 2.0 ** -5 * Tb)
        d = dm @ ref[li][0]
    return res


def test_mlp_forward_backward_matches_fp64_oracle(sim):
    """Training forward and backward (mma.sync tiles) element by element against the oracle on
    the same BF16 operands: every output within output_bound, every gradient entry within
    grad_bounds, the loss to 1e-5."""
    rng = np.random.default_rng(0)
    params = mlp.init_params(rng)
    params = [(W, rng.normal(0, 0.1, b.size)) for W, b in params]        # nonzero biases
    flat = np.concatenate([np.concatenate([W.ravel(), b]) for W, b in params]).astype(np.float32)
    sim.set_mlp_params(flat)
    assert np.array_equal(sim.mlp_params(), flat)
    x = rng.normal(size=(1000, mlp.SIZES[0])).astype(np.float32)
    t = rng.normal(size=(1000, 2)).astype(np.float32)
    y, loss, g = sim.mlp_forward_backward(x, t)
    ref = bf16_params(flat)
    x64, t64 = x.astype(np.float64), t.astype(np.float64)
    bound, yr = output_bound(ref, x64)
    assert np.all(np.abs(y - yr) <= bound), np.max(np.abs(y - yr) / bound)
    lr_, gr = mlp.loss_and_grad(ref, x64, t64, bf16_operands=True)
    assert loss == pytest.approx(lr_, rel=1e-5)
    gg = unflatten(g.astype(np.float64))
    for li, ((gW, gb), (rW, rb), (BW, Bb)) in enumerate(zip(gg, gr, grad_bounds(ref, x64, t64))):
        assert np.all(np.abs(gW - rW) <= BW), (li, np.max(np.abs(gW - rW) / BW))
        assert np.all(np.abs(gb - rb) <= Bb), (li, np.max(np.abs(gb - rb) / Bb))


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


def test_production_emission_matches_integral(sim):
    """Emission stage in the production form (surrogate, FP32-Gamow fallback) on a hot tip in a
    calibrated Laplace field: every face's J within 0.02 in log10 J of the oracle's FP64 integral
    wherever J is above 1e-3 A/m^2 -- below it the step may take the network's value in bins that
    failed validation, since such a face emits an SP with probability < 1e-13 per step (runs
    after the training test on the same handle)."""
    from oracle import field, step as OS
    from oracle.grid import Grid
    from paper_2402_08404_gb300 import pic
    cfg = dict(synth.CONFIGS["small"])
    g = Grid(cfg["nx"], cfg["ny"], cfg["nz"], cfg["dx"], cfg["tip_radius"], cfg["tip_height"])
    V0 = field.calibrate_V0(g, cfg["apex_field"])
    phi = np.round(field.solve_poisson(g, V0) * 2.0 ** 40) / 2.0 ** 40   # the library's fixed-point grid
    sim.set_potential(phi)
    rng = np.random.default_rng(5)
    T = rng.uniform(1500.0, 3500.0, int(g.solid.sum()))
    sim.set_temperature(T)
    sim.set_flags(pic.F_PRODUCTION)
    sim.emit()
    F_got, J, _ = sim.face_emission()
    st = OS.State(g, dict(cfg, V0=V0, next_id=0), synth.plasma(dict(cfg, n_sp=100), seed=1), phi, T=T)
    Fv = field.face_field(g, phi)
    assert np.array_equal(F_got, Fv)
    pick = rng.choice(g.nface, size=min(400, g.nface), replace=False)
    Jr, _ = em.current_density_fixed(Fv[pick] * 1e-9, OS.face_temperature(st)[pick], cfg["work_function"],
                                     OS.face_radius_nm(g, st.prm)[pick])
    rel = Jr > 1e-3
    assert rel.sum() > 50
    err = np.abs(np.log10(np.maximum(J[pick][rel], 1e-300)) - np.log10(Jr[rel]))
    assert err.max() <= 0.02, (np.sort(err)[-5:],)


def test_surrogate_copy_serves_another_instance(sim):
    """pic_surrogate_copy installs the trained network and its validity map in a second instance
    (one training for an ensemble): its evaluations equal the source's bit for bit (runs after
    the training test on the same handle)."""
    from paper_2402_08404_gb300 import pic
    other = pic.Pic(dict(synth.CONFIGS["small"]), capacity=50_000, V0=20.0)
    F, T, W, R = synth.face_tuples(4000, seed=33)
    with pytest.raises(pic.PicError):
        sim.surrogate_copy_from(other)        # the source has no trained network
    other.surrogate_copy_from(sim)
    J1, P1, v1 = sim.surrogate_eval(F * 1e9, T, W, R * 1e-9)
    J2, P2, v2 = other.surrogate_eval(F * 1e9, T, W, R * 1e-9)
    assert v1.sum() > 100
    assert np.array_equal(v1, v2) and np.array_equal(J1, J2) and np.array_equal(P1, P2)
    other.close()


def test_tcgen05_inference_matches_reference_forward(sim):
    """Inference (forward without targets: the fused tcgen05/TMEM kernel the step uses) against the
    training path's forward (mma.sync tiles) and the FP64 oracle on the same BF16 operands: the
    two GPU paths differ only in the FP32 accumulation order inside the 128-term products."""
    rng = np.random.default_rng(4)
    params = mlp.init_params(rng)
    params = [(W, rng.normal(0, 0.1, b.size)) for W, b in params]
    flat = np.concatenate([np.concatenate([W.ravel(), b]) for W, b in params]).astype(np.float32)
    sim.set_mlp_params(flat)
    for n in (1, 127, 128, 1000, 70001):     # partial tiles, one tile, many tiles per CTA
        x = rng.normal(size=(n, mlp.SIZES[0])).astype(np.float32)
        (y_tc,) = sim.mlp_forward_backward(x)
        y_ref, _, _ = sim.mlp_forward_backward(x, np.zeros((n, 2), np.float32))
        assert np.all(np.isfinite(y_tc))
        assert np.max(np.abs(y_tc - y_ref)) <= 2e-3 * max(1.0, np.max(np.abs(y_ref))), n
        assert np.linalg.norm(y_tc - y_ref) <= 1e-4 * np.linalg.norm(y_ref) + 1e-6, n
        if n <= 1000:
            bound, yr = output_bound(bf16_params(flat), x.astype(np.float64))
            assert np.all(np.abs(y_tc - yr) <= bound), (n, np.max(np.abs(y_tc - yr) / bound))
