"""Failure detection without a GPU fault.

The failures are made on the host (reloc_inject_faults): a tensor-core GEMM
whose MMA lanes wait on a barrier that nothing completes, and device
allocations that fail.  Each test checks the status the library returns
(RELOC_ETIMEOUT, RELOC_ENOMEM) and that the same context then computes the
same results as before -- the bounded waits gave up, the kernel released its
tensor memory and nothing it started was still running."""
import time

import numpy as np
import pytest

import scenegen as sg

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def R():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2403_11367_gb300.build import build
    build()
    from paper_2403_11367_gb300 import reloc
    yield reloc
    reloc.reloc_inject_faults(reloc.FAULT_GEMM_WAIT, 0)
    reloc.reloc_inject_faults(reloc.FAULT_ALLOC, 0)


def bf16(shape, seed):
    x = sg.Rng(seed).normal(int(np.prod(shape))).reshape(shape).astype(np.float32)
    t = torch.tensor(x).to(torch.bfloat16)
    return t.cuda(), t.float().numpy().astype(np.float64)


def test_gemm_wait_expiry_returns_etimeout_and_context_recovers(R):
    ctx = R.Context()
    A, a = bf16((256, 512), 5)        # two CTAs, eight K steps (more than the four stages)
    B, b = bf16((64, 512), 6)
    C = torch.full((256, 64), float("nan"), device="cuda:0")
    R.reloc_inject_faults(R.FAULT_GEMM_WAIT, 1)
    t0 = time.perf_counter()
    with pytest.raises(R.RelocError) as e:
        ctx.gemm_bf16(A, B, C)
    dt = time.perf_counter() - t0
    assert e.value.status == R.ETIMEOUT
    assert dt < 10.0                   # bounded waits (about a second each)
    # the next launch is not injected and computes the product
    ctx.gemm_bf16(A, B, C)
    ref = a @ b.T
    assert np.abs(C.cpu().numpy() - ref).max() < 1e-3 * np.abs(ref).max()
    # an unrelated kernel on the same context after the expiry
    s = sg.tiny_scene(n=2000)
    ctx.load_map(s.gaussians)
    rgb = torch.empty((1, 3, s.camera.height, s.camera.width), device="cuda:0")
    ctx.render([(0, ctx.n)], s.candidate_poses[:1], s.camera, rgb=rgb)
    torch.cuda.synchronize()
    assert torch.isfinite(rgb).all() and float(rgb.max()) > 0


def render(ctx, s, V):
    out = torch.empty((V, 3, s.camera.height, s.camera.width), device="cuda:0")
    ctx.render([(0, ctx.n)], s.candidate_poses[:V], s.camera, rgb=out)
    torch.cuda.synchronize()
    return out.cpu().numpy()


def test_allocation_failure_returns_enomem_and_context_recovers(R):
    s = sg.tiny_scene(n=4000)
    ref_ctx = R.Context()
    ref_ctx.load_map(s.gaussians)
    ref = render(ref_ctx, s, 8)
    ctx = R.Context()
    # the map upload's allocation fails; the next upload succeeds
    R.reloc_inject_faults(R.FAULT_ALLOC, 1)
    with pytest.raises(R.RelocError) as e:
        ctx.load_map(s.gaussians)
    assert e.value.status == R.ENOMEM
    ctx.load_map(s.gaussians)
    one = render(ctx, s, 1)
    assert np.array_equal(one[0], ref[0])
    # the workspace must grow for 8 views: that allocation fails, the retry works
    R.reloc_inject_faults(R.FAULT_ALLOC, 1)
    with pytest.raises(R.RelocError) as e:
        render(ctx, s, 8)
    assert e.value.status == R.ENOMEM
    assert np.array_equal(render(ctx, s, 8), ref)


def test_inject_faults_rejects_bad_arguments(R):
    with pytest.raises(R.RelocError) as e:
        R.reloc_inject_faults(7, 1)
    assert e.value.status == R.EINVAL
    with pytest.raises(R.RelocError) as e:
        R.reloc_inject_faults(R.FAULT_ALLOC, -1)
    assert e.value.status == R.EINVAL
