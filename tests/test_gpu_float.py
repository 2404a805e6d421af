"""GPU float chain (differentiable colourise): forward and adjoint through the C ABI against
the FP64 oracle.

Bars: forward F within fp32 rounding of the FP64 F; gradient rel. L2 < 1e-5 against the FP64
J^T 2(F - T); exact zeros for the coefficients of MCUs no tap touches; central differences
(exact for the quadratic loss) on 1000 coefficients."""

import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def jt():
    import paper_2510_08166_gb300 as m
    return m


def _coef_set(seed, T, size, q=75):
    ts = synth.make_texture_set(seed, [(size, size)] * T, [q] * T, [420] * T, full_chain=False, keep_coefs=True)
    m = size // 16
    coef = np.empty((T, m, m, 6, 64), np.float32)
    for t, lv in enumerate(ts.levels):
        e = lv[0]
        qt = np.concatenate([np.repeat(e.qt[0][None], 4, 0), e.qt[1][None], e.qt[1][None]]).astype(np.float32)
        coef[t] = (e.qcoef.astype(np.float32) * qt).reshape(m, m, 6, 64)
    return ts, coef


def _case(seed, T, size, W, H, kind="plane"):
    """kind "plane": the coefficient scene's perspective ground plane (touches most MCUs at these sizes);
    "bands": one rotated, magnified window per texture 0..T-2 (a part of each texture's MCUs),
    texture T-1 untouched, 3 % empty pixels."""
    ts, coef = _coef_set(seed, T, size)
    if kind == "plane":
        pose = synth.Pose((0.0, 1.7, 0.0), 15.0, -25.0, 60.0, 0, 0.0)
        gb = synth.gbuffer_scene(seed, W, H, [(size, size)] * T, [1] * T, pose, nquads=0, use_mips=False)
    else:
        hb = H // (T - 1)
        bands = [synth.gbuffer_affine(W, hb if t < T - 2 else H - hb * (T - 2), 11.0 + 23 * t, 0.25 + 0.1 * t, t)
                 for t in range(T - 1)]
        gb = synth.GBuffer(W, H, np.concatenate([b.uv for b in bands]), np.concatenate([b.tex_id for b in bands]),
                           np.concatenate([b.mip for b in bands]))
        gb.tex_id[np.random.default_rng(seed).random((H, W)) < 0.03] = 0xFFFF
    target = synth.noise_image(seed + 1, W, H)
    return ts, coef, gb, target


def _ctx(jt, coef, blocks=1 << 14):
    T, my, mx = coef.shape[:3]
    ctx = jt.Context(0, blocks)
    ctx.register_coeff_textures(0, T, mx * 16, my * 16)
    return ctx


def _rel_l2(a, b):
    return float(np.linalg.norm((a - b).ravel()) / max(np.linalg.norm(b.ravel()), 1e-300))


@pytest.mark.parametrize("seed,T,size,W,H,kind", [(9, 3, 64, 96, 64, "plane"), (4, 2, 128, 133, 77, "plane"),
                                                 (12, 5, 256, 256, 144, "plane"), (3, 4, 256, 200, 150, "bands"),
                                                 (8, 3, 512, 131, 97, "bands")])
def test_forward_and_gradient_match_fp64(jt, seed, T, size, W, H, kind):
    ts, coef, gb, target = _case(seed, T, size, W, H, kind)
    ctx = _ctx(jt, coef)
    dgb = jt.DeviceGBuffer.from_host(gb)
    c = torch.from_numpy(coef).cuda()
    F = torch.empty((H, W, 3), dtype=torch.float32, device="cuda")
    ctx.colorize_float(dgb, c, F)
    st = ctx.stats()
    F_ref = oracle.float_forward(coef, gb)
    assert _rel_l2(F.cpu().numpy().astype(np.float64), F_ref) < 1e-6
    assert np.abs(F.cpu().numpy() - F_ref).max() < 5e-3
    o_flags = oracle.texset_from(ts).mark(gb, 1)  # same gid layout: T textures, level 0
    assert st["needed_blocks"] == int((o_flags > 0).sum())
    # backward of L = sum (F - T)^2
    L_ref, g_ref = oracle.float_loss_grad(coef, gb, target)
    gF = 2.0 * (F - torch.from_numpy(target).cuda())
    gc = torch.full_like(c, float("nan"))
    ctx.colorize_backward(dgb, gF.contiguous(), gc)
    ctx.stats()
    g = gc.cpu().numpy().astype(np.float64)
    assert _rel_l2(g, g_ref) < 1e-5
    per_mcu_ref = np.abs(g_ref).reshape(-1, 384).sum(axis=1)
    per_mcu = np.abs(g).reshape(-1, 384).sum(axis=1)
    np.testing.assert_array_equal(per_mcu[per_mcu_ref == 0], 0.0)  # untouched MCUs: exactly zero
    assert (per_mcu[o_flags > 0] > 0).all()
    ctx.close()


def test_gradient_against_central_differences(jt):
    """L is quadratic in c, so (L(c + e_i) - L(c - e_i)) / 2 is its exact derivative: 1000
    coefficients, mostly of needed MCUs plus some of MCUs no tap touches (derivative 0)."""
    _, coef, gb, target = _case(21, 4, 256, 160, 96, "bands")
    ctx = _ctx(jt, coef)
    dgb = jt.DeviceGBuffer.from_host(gb)
    c = torch.from_numpy(coef).cuda().requires_grad_(True)
    F = ctx.colorize_float_autograd(dgb, c)
    loss = ((F - torch.from_numpy(target).cuda()) ** 2).sum()
    loss.backward()
    ctx.stats()
    g = c.grad.cpu().numpy().astype(np.float64).ravel()
    rng = np.random.default_rng(5)
    nz = np.flatnonzero(g)
    zero = np.flatnonzero(g == 0)
    assert zero.size > 1000  # the bands leave most MCUs untouched
    idx = np.concatenate([rng.choice(nz, 900, replace=False), rng.choice(zero, 100, replace=False)])
    fd = oracle.float_fd(coef, gb, target, idx, h=1.0)
    scale = np.abs(fd).max()
    assert scale > 0
    np.testing.assert_allclose(g[idx], fd, rtol=0, atol=2e-5 * scale)
    assert (fd[900:] == 0).all()
    assert _rel_l2(g[idx], fd) < 1e-5
    # the loss itself (through the autograd op's forward) matches FP64
    L_ref, _ = oracle.float_loss_grad(coef, gb, target, want_grad=False)
    assert abs(float(loss.detach()) - L_ref) <= 1e-5 * L_ref
    ctx.close()


def test_float_errors(jt):
    _, coef, gb, target = _case(9, 2, 64, 64, 48)
    ctx = jt.Context(0, 1 << 12)
    dgb = jt.DeviceGBuffer.from_host(gb)
    c = torch.from_numpy(coef).cuda()
    F = torch.empty((48, 64, 3), dtype=torch.float32, device="cuda")
    with pytest.raises(jt.JTError) as e:  # nothing registered
        ctx.colorize_float(dgb, c, F)
    assert e.value.status == 7
    with pytest.raises(jt.JTError):
        ctx.register_coeff_textures(0, 2, 60, 64)  # not a multiple of 16
    ctx.register_coeff_textures(0, 2, 64, 64)
    with pytest.raises(jt.JTError):
        ctx.register_coeff_textures(5, 1, 64, 64)  # only one registration per context
    ctx.colorize_float(dgb, c, F)
    assert ctx.stats()["status"] == 0
    # a float tile capacity smaller than the needed set is reported, not overrun
    small = jt.Context(0, 4)
    small.register_coeff_textures(0, 2, 64, 64)
    small.colorize_float(dgb, c, F)
    st = small.stats(check=False)
    assert st["status"] == 5 and st["error_bits"] & jt.DEVERR_CAPACITY
    # the same for the backward pass, whose gradient then covers only the MCUs that fit
    gC = torch.full_like(c, 7.0)
    small.colorize_backward(dgb, torch.ones_like(F), gC)
    st = small.stats(check=False)
    assert st["status"] == 5 and st["error_bits"] & jt.DEVERR_CAPACITY
    assert torch.isfinite(gC).all() and int((gC.abs().sum(dim=(3, 4)) != 0).sum()) <= 4
    small.close()
    ctx.close()
