"""Oracle pins for the FP64 float colourise chain and its gradient.

F = bilinear(RGB(upsample(IDCT_f(c) + 128))) is affine in the coefficients c, so the
loss L = sum (F - T)^2 is quadratic: central differences are exact up to rounding for
any step, and <J dc, g> = <dc, J^T g> holds for the linear part J.
"""

import numpy as np

import oracle
import synth


def _setup(T=3, size=64, W=96, H=64, seed=9):
    ts = synth.make_texture_set(seed, [(size, size)] * T, [75] * T, [420] * T, full_chain=False, keep_coefs=True)
    m = size // 16
    coef = np.empty((T, m, m, 6, 64), np.float32)
    for t, lv in enumerate(ts.levels):
        e = lv[0]
        q = np.concatenate([np.repeat(e.qt[0][None], 4, 0), e.qt[1][None], e.qt[1][None]]).astype(np.float32)
        coef[t] = (e.qcoef.astype(np.float32) * q).reshape(m, m, 6, 64)
    pose = synth.Pose((0.0, 1.7, 0.0), 15.0, -25.0, 60.0, 0, 0.0)
    gb = synth.gbuffer_scene(seed, W, H, [(size, size)] * T, [1] * T, pose, nquads=0, use_mips=False)
    # squeeze the view onto the small textures: scale uv so the plane covers few repeats
    target = synth.noise_image(seed + 1, W, H)
    return ts, coef, gb, target


def test_fd_equals_analytic_gradient():
    ts, coef, gb, target = _setup()
    L, grad = oracle.float_loss_grad(coef, gb, target)
    rng = np.random.default_rng(1)
    nz = np.flatnonzero(grad)
    idx = np.concatenate([rng.choice(nz, 150, replace=False), rng.integers(0, coef.size, 50)])
    fd = oracle.float_fd(coef, gb, target, idx, h=1.0)
    g = grad.ravel()[idx]
    scale = np.abs(g).max()
    assert scale > 0
    np.testing.assert_allclose(fd, g, rtol=1e-7, atol=1e-9 * scale)


def test_fd_step_independent():
    """Quadratic loss: the central difference does not depend on the step."""
    ts, coef, gb, target = _setup()
    _, grad = oracle.float_loss_grad(coef, gb, target)
    idx = np.flatnonzero(grad)[:40]
    a = oracle.float_fd(coef, gb, target, idx, h=1.0)
    b = oracle.float_fd(coef, gb, target, idx, h=0.01)
    np.testing.assert_allclose(a, b, rtol=1e-6, atol=1e-9 * np.abs(a).max())


def test_adjoint_identity():
    ts, coef, gb, target = _setup()
    rng = np.random.default_rng(2)
    F0 = oracle.float_forward(np.zeros_like(coef), gb)
    dc = rng.standard_normal(coef.shape).astype(np.float32)
    Jdc = oracle.float_forward(dc, gb) - F0  # F is affine: J dc = F(dc) - F(0)
    g = rng.standard_normal(F0.shape)
    JTg = oracle.float_vjp(coef.shape, gb, g)
    lhs = float((Jdc * g).sum())
    rhs = float((dc.astype(np.float64) * JTg).sum())
    assert abs(lhs - rhs) <= 1e-9 * max(abs(lhs), 1.0)


def test_unneeded_mcus_have_zero_gradient():
    ts, coef, gb, target = _setup()
    _, grad = oracle.float_loss_grad(coef, gb, target)
    o = oracle.texset_from(ts)
    flags = o.mark(gb, 1)  # bilinear marking: every MCU a tap touches
    per_mcu = np.abs(grad).reshape(-1, 384).sum(axis=1)
    assert ((per_mcu > 0) <= (flags > 0)).all()
    assert (per_mcu[flags == 0] == 0).all()
    assert (per_mcu[flags > 0] > 0).mean() > 0.5


def test_float_chain_matches_integer_decode_at_texel_centres():
    """At texel centres bilinear weights are exact; the FP64 chain must agree with the
    integer decode of the same coefficients to within rounding (a transposed IDCT or a
    wrong colour constant would not)."""
    ts, coef, gb, target = _setup(T=2, size=64)
    T, m = coef.shape[0], coef.shape[1]
    size = m * 16
    xs, ys = np.meshgrid(np.arange(size), np.arange(size))
    uv = np.stack([(xs + 0.5) / size, (ys + 0.5) / size], axis=-1).astype(np.float32)
    for t in range(T):
        g = synth.GBuffer(size, size, uv, np.full((size, size), t, np.uint16), np.zeros((size, size), np.uint8))
        F = oracle.float_forward(coef, g)
        ref = oracle.Decoded(ts.levels[t][0].jfif).rgba[..., :3].astype(np.float64)
        inside = (F > 2) & (F < 253)  # away from the integer path's clamps
        err = np.abs(F - ref)[inside]
        assert err.max() < 3.0 and err.mean() < 0.8, (err.max(), err.mean())
