"""Host side of map training and gray NCC (no GPU: only option defaults are
read through the C ABI): the defaults are the values include/reloc.h states
(the paper gives no lambda, omega_1, omega_2: 3D Gaussian Splatting's
lambda = 0.2 and weights of 1; Adam's usual betas), the binding rejects
option names the C struct does not have, and the gray NCC flag defaults to
the RGB reading."""
import pytest


@pytest.fixture(scope="module")
def R():
    from paper_2403_11367_gb300.build import build
    build()
    from paper_2403_11367_gb300 import reloc
    return reloc


def test_training_defaults(R):
    o = R.Context.train_options()
    assert (o.lambda_dssim, o.w_photo, o.w_reproj) == (0.2, 1.0, 1.0)
    assert (o.lr_mean, o.lr_scale, o.lr_quat, o.lr_opacity, o.lr_color) == (1.6e-4, 5e-3, 1e-3, 5e-2, 2.5e-3)
    assert (o.beta1, o.beta2, o.eps) == (0.9, 0.999, 1e-15)
    assert o.reproj_alpha_min == 0.5 and o.views_per_group == 16


def test_training_options_override_and_reject_unknown_names(R):
    o = R.Context.train_options(lambda_dssim=0.0, w_reproj=0.5, views_per_group=4)
    assert (o.lambda_dssim, o.w_reproj, o.views_per_group) == (0.0, 0.5, 4)
    with pytest.raises(TypeError):
        R.Context.train_options(lambda_ssim=0.1)


def test_gray_ncc_defaults_to_rgb(R):
    assert R.reloc_default_config().ncc_gray == 0
    assert R.reloc_default_config(ncc_gray=1).ncc_gray == 1
