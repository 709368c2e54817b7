"""Pins of the oracle's Adam step on 3D Gaussian Splatting's latent
parameters (used against the GPU's reloc_train_step).

Closed forms of Adam's definition: at the first step m_hat = g and
v_hat = g^2, so every latent parameter moves by lr * sign(g) (eps -> 0):
mean, quaternion and colour by -lr sign(g), the scale by the factor
exp(-lr sign(g)), the opacity's logit by -lr sign(g); a zero gradient leaves a
parameter unchanged; with beta1 = beta2 = 0 every step is again
lr * g / |g|; the moments follow their recurrences."""
import numpy as np

import oracle
import scenegen as sg

LR = np.array([1e-3, 5e-3, 2e-3, 5e-2, 3e-3])
GROUP = np.array([0, 0, 0, 1, 1, 1, 2, 2, 2, 2, 3, 4, 4, 4])


def setup():
    g = sg.tiny_scene(n=50).gaussians
    prm = oracle.map_params(g)
    grad = sg.Rng(3).normal(50 * 14, 0.0, 1.0).reshape(50, 14)
    grad[::7, :] = 0.0
    return prm, grad


def expected_first_step(prm, grad, lr):
    s = np.sign(grad) * lr[GROUP][None, :]
    out = prm.copy()
    raw = [0, 1, 2, 6, 7, 8, 9, 11, 12, 13]
    out[:, raw] = prm[:, raw] - s[:, raw]
    out[:, 3:6] = prm[:, 3:6] * np.exp(-s[:, 3:6])
    o = prm[:, 10]
    out[:, 10] = 1.0 / (1.0 + np.exp(-(np.log(o / (1 - o)) - s[:, 10])))
    return out


def test_first_step_moves_each_latent_by_lr_sign():
    prm, grad = setup()
    out, m, v = oracle.adam_step(prm, grad, np.zeros_like(grad), np.zeros_like(grad), 1, LR, eps=1e-30)
    assert np.max(np.abs(out - expected_first_step(prm, grad, LR))) < 1e-12
    zero = np.all(grad == 0.0, axis=1)
    assert np.max(np.abs(out[zero] - prm[zero])) < 1e-15     # the opacity's logit round trip: an ulp


def test_no_momentum_repeats_the_sign_step():
    prm, grad = setup()
    p1, m, v = oracle.adam_step(prm, grad, np.zeros_like(grad), np.zeros_like(grad), 1, LR, 0.0, 0.0, 1e-30)
    p2, _, _ = oracle.adam_step(p1, grad, m, v, 2, LR, 0.0, 0.0, 1e-30)
    # the latent gradients of scale and opacity keep their signs (s > 0, o (1 - o) > 0)
    assert np.max(np.abs(p2 - expected_first_step(p1, grad, LR))) < 1e-12


def test_moments_follow_their_recurrences():
    prm, grad = setup()
    m0 = sg.Rng(4).normal(50 * 14, 0.0, 0.1).reshape(50, 14)
    v0 = np.abs(sg.Rng(5).normal(50 * 14, 0.0, 0.1).reshape(50, 14))
    _, m, v = oracle.adam_step(prm, grad, m0, v0, 3, LR, 0.8, 0.95)
    lat = grad.copy()
    lat[:, 3:6] *= prm[:, 3:6]
    lat[:, 10] *= prm[:, 10] * (1 - prm[:, 10])
    assert np.max(np.abs(m - (0.8 * m0 + 0.2 * lat))) < 1e-15
    assert np.max(np.abs(v - (0.95 * v0 + 0.05 * lat * lat))) < 1e-15
