"""Pins of the FP64 CNN oracle (the learned proposal's reference): finite
differences of the loss, closed forms of single layers, Adam's first step,
and the downsample against numpy."""
import math

import numpy as np
import pytest

import oracle
import scenegen as sg


@pytest.fixture(scope="module")
def net():
    r = sg.Rng(41)
    n = oracle.cnn_param_count()
    p = np.zeros(n)
    for wo, bo, shape in oracle.cnn_offsets():
        fan_in = int(np.prod(shape[1:]))
        p[wo:bo] = r.normal(bo - wo, 0.0, math.sqrt(2.0 / fan_in))
        p[bo:bo + shape[0]] = r.normal(shape[0], 0.0, 0.05)
    x = r.uniform(2 * 47 * 176 * 2).reshape(2, 47, 176, 2)
    y = np.array([7, 41], np.int32)
    return p, x, y


def test_param_count():
    assert oracle.cnn_param_count() == 1916960


def test_loss_gradient_matches_central_differences(net):
    p, x, y = net
    loss, g, gi = oracle.cnn_loss_grad(p, x, y, want_input_grad=True)
    r = sg.Rng(42)
    h = 1e-6
    checked = 0
    for wo, bo, shape in oracle.cnn_offsets():
        for lo, hi in ((wo, bo), (bo, bo + shape[0])):
            for _ in range(4):
                i = lo + int(r.uniform(1)[0] * (hi - lo))
                if abs(g[i]) < 1e-7:
                    continue
                pp, pm = p.copy(), p.copy()
                pp[i] += h; pm[i] -= h
                fd = (oracle.cnn_loss_grad(pp, x, y)[0] - oracle.cnn_loss_grad(pm, x, y)[0]) / (2 * h)
                assert abs(fd - g[i]) <= 1e-6 * max(abs(g[i]), 1e-3), (i, fd, g[i])
                checked += 1
    assert checked >= 20
    for _ in range(6):
        j = tuple(int(r.uniform(1)[0] * s) for s in x.shape)
        xp, xm = x.copy(), x.copy()
        xp[j] += h; xm[j] -= h
        fd = (oracle.cnn_loss_grad(p, xp, y)[0] - oracle.cnn_loss_grad(p, xm, y)[0]) / (2 * h)
        assert abs(fd - gi[j]) <= 1e-6 * max(abs(gi[j]), 1e-3)


def test_uniform_logits_give_log_classes():
    p = np.zeros(oracle.cnn_param_count())
    x = sg.Rng(3).uniform(3 * 47 * 176 * 2).reshape(3, 47, 176, 2)
    loss, g = oracle.cnn_loss_grad(p, x, np.array([0, 5, 63], np.int32))
    assert abs(loss - math.log(64)) < 1e-13
    wo, bo, shape = oracle.cnn_offsets()[6]
    db = g[bo:bo + 64]
    exp = np.full(64, 1 / 64.0)
    for c in (0, 5, 63):
        exp[c] -= 1 / 3.0
    assert np.allclose(db, exp, atol=1e-15)       # mean over the batch of p - onehot


def test_delta_kernel_convolution_is_strided_subsampling():
    x = sg.Rng(5).uniform(9 * 14 * 3).reshape(9, 14, 3)
    w = np.zeros((3, 3, 3, 3))
    for c in range(3):
        w[c, 1, 1, c] = 1.0                     # centre tap
    y = oracle.conv3x3s2(x, w, np.zeros(3))
    assert np.array_equal(y, x[::2, ::2, :])
    # a tap at (ky, kx) = (0, 0) reads (2 oy - 1, 2 ox - 1), zero-padded
    w2 = np.zeros((1, 3, 3, 3)); w2[0, 0, 0, 1] = 2.0
    y2 = oracle.conv3x3s2(x, w2, np.array([0.5]))
    ref = np.full((5, 7), 0.5)
    ref[1:, 1:] += 2.0 * x[1:8:2, 1:12:2, 1]
    assert np.allclose(y2[..., 0], ref)
    # ReLU
    y3 = oracle.conv3x3s2(x, w, np.full(3, -10.0))
    assert np.all(y3 == 0)


def test_adam_first_step_closed_form():
    r = sg.Rng(6)
    w = r.normal(50); g = r.normal(50)
    lr, eps = 1e-3, 1e-8
    w1, m1, v1 = oracle.adam(w, np.zeros(50), np.zeros(50), g, lr, 1, eps=eps)
    # m_hat = g, v_hat = g^2 after one step
    assert np.allclose(w1, w - lr * g / (np.abs(g) + eps), atol=1e-15)
    assert np.allclose(m1, 0.1 * g) and np.allclose(v1, 0.001 * g * g)


def test_downsample_gray_matches_numpy():
    img = sg.Rng(8).uniform(3 * 94 * 352).reshape(3, 94, 352).astype(np.float32)
    out = oracle.downsample_gray(img, 2)
    ref = img.astype(np.float64).mean(axis=0).reshape(47, 2, 176, 2).mean(axis=(1, 3))
    assert out.shape == (47, 176)
    assert np.allclose(out, ref, atol=1e-12)


# ---- BF16 activation storage (the BF16 network's reference) --------------------

def _bf16(a):
    """torch's FP32 -> BF16 conversion (round to nearest even), as FP64."""
    torch = pytest.importorskip("torch")
    return torch.tensor(np.asarray(a, np.float64), dtype=torch.float32).to(torch.bfloat16).double().numpy()


def test_bf16_round_ties_to_even_and_matches_torch():
    # exact ties between two BF16 neighbours go to the even significand
    assert oracle.bf16_round(1 + 2 ** -8) == 1.0
    assert oracle.bf16_round(1 + 3 * 2 ** -8) == 1 + 2 ** -6
    assert oracle.bf16_round(-(1 + 2 ** -8)) == -1.0
    assert oracle.bf16_round(1 + 2 ** -8 + 2 ** -20) == 1 + 2 ** -7
    assert oracle.bf16_round(0.0) == 0.0 and oracle.bf16_round(3.0e38) == float(_bf16([3.0e38])[0])
    vals = sg.Rng(5).normal(2000, 0.0, 3.0) * np.exp(sg.Rng(6).uniform(2000, -20, 20))
    got = np.array([oracle.bf16_round(v) for v in vals])
    assert np.array_equal(got, _bf16(vals))


def _forward_composed(p, x):
    """The network layer by layer from the oracle's single-layer convolution,
    every stored activation rounded to BF16; returns (x5, h1, logits)."""
    offs = oracle.cnn_offsets()
    outs = []
    for xb in x:
        a = xb
        for l in range(5):
            wo, bo, shape = offs[l]
            a = _bf16(oracle.conv3x3s2(a, p[wo:bo].reshape(shape), p[bo:bo + shape[0]]))
        x5 = a.reshape(-1)
        wo, bo, shape = offs[5]
        h1 = _bf16(np.maximum(p[wo:bo].reshape(shape) @ x5 + p[bo:bo + shape[0]], 0.0))
        wo, bo, shape = offs[6]
        z = p[wo:bo].reshape(shape) @ h1 + p[bo:bo + shape[0]]
        outs.append((x5, h1, z))
    return outs


def test_bf16_activation_forward_is_the_rounded_composition(net):
    p, x, y = net
    z = oracle.cnn_forward(p, x, act_bf16=True)
    ref = np.stack([o[2] for o in _forward_composed(p, x)])
    assert np.abs(z - ref).max() <= 1e-9 * np.abs(ref).max()
    # and the rounding matters: the plain forward differs
    assert np.abs(oracle.cnn_forward(p, x) - ref).max() > 1e-6


def test_bf16_activation_gradient_is_the_chain_rule_at_stored_values(net):
    """The last two layers' weight gradients in closed form at the rounded
    activations: dL/dW2 = dz h1^T, dL/dW1 = (W2^T dz * [h1 > 0]) x5^T."""
    p, x, y = net
    loss, g = oracle.cnn_loss_grad(p, x, y, act_bf16=True)
    offs = oracle.cnn_offsets()
    w2o, b2o, s2 = offs[6]
    w1o, b1o, s1 = offs[5]
    W2 = p[w2o:b2o].reshape(s2)
    gW2 = np.zeros(s2)
    gW1 = np.zeros(s1)
    ref_loss = 0.0
    for (x5, h1, z), lab in zip(_forward_composed(p, x), y):
        e = np.exp(z - z.max())
        pr = e / e.sum()
        ref_loss += (np.log(e.sum()) + z.max() - z[lab]) / len(y)
        dz = pr.copy()
        dz[lab] -= 1.0
        dz /= len(y)
        gW2 += np.outer(dz, h1)
        dh = (W2.T @ dz) * (h1 > 0)
        gW1 += np.outer(dh, x5)
    assert abs(loss - ref_loss) <= 1e-12 * ref_loss
    assert np.abs(g[w2o:b2o].reshape(s2) - gW2).max() <= 1e-12 * np.abs(gW2).max()
    assert np.abs(g[w1o:b1o].reshape(s1) - gW1).max() <= 1e-12 * np.abs(gW1).max()
