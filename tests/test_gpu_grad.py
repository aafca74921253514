"""Differentiation on the GPU: the loss kernel, the adjoint through the whole
path, and the torch.autograd wrapper, against the FP64 oracle.  (The FP64
finite-difference check of the oracle's own gradient is in test_oracle_pins.)"""
import numpy as np
import pytest

import oracle
from paper_1904_09409_gb300 import synth
from tests import _gpu
from tests._lines import true_cells

pytestmark = pytest.mark.gpu
TOL = 1e-5


@pytest.fixture(scope="module")
def torch():
    return _gpu.torch_cuda()


def workload(side, n, start=0):
    imgs, targets = [], []
    for i in range(n):
        si = synth.mixed_image(synth.WL_GRAD_512, start + i, side, side)
        imgs.append(si.img)
        targets.append(synth.blob_target(side, side, true_cells(si.lines, side, side, side, side)))
    return np.stack(imgs), np.stack(targets)


def test_loss_kernel_matches_oracle(torch):
    from paper_1904_09409_gb300 import funnel as f
    rng = np.random.default_rng(7)
    maps = (rng.standard_normal((3, 96, 128)) * 40).astype(np.float32)
    maps[0, 5, 7] = 0.0                                   # sign(0) = 0
    tgt = rng.random((3, 96, 128)).astype(np.float32)
    with f.Plan(96, 128, 128, 96) as plan:
        m = torch.from_numpy(maps).cuda()
        t = torch.from_numpy(tgt).cuda()
        loss, grad = f.ft_abs_mse_grad(plan, m, t, 2.0 / 128)
        loss2, _ = f.ft_abs_mse_grad(plan, m, t, 2.0 / 128, grad=False)
        torch.cuda.synchronize()
    assert torch.equal(loss, loss2)                       # deterministic
    ref_grad = np.empty_like(maps, dtype=np.float64)
    for i in range(3):
        l_ref, g_ref = oracle.map_loss_grad_ref(maps[i].astype(np.float64), tgt[i], 128)
        assert abs(float(loss[i]) - l_ref) <= 1e-6 * l_ref
        ref_grad[i] = g_ref / 3.0                         # gradient of the batch mean
    np.testing.assert_allclose(grad.cpu().numpy(), ref_grad, rtol=1e-6, atol=1e-12)


@pytest.mark.parametrize("side,n", [(64, 4), (512, 2)])
def test_forward_loss_backward_matches_oracle(torch, side, n):
    from paper_1904_09409_gb300 import funnel as f
    imgs, tgts = workload(side, n)
    with f.Plan(side, side, side, side) as plan:
        x = torch.from_numpy(imgs).cuda()
        t = torch.from_numpy(tgts).cuda()
        P = torch.empty_like(x)
        f.ft_forward(plan, x, P)
        loss, dP = f.ft_abs_mse_grad(plan, P, t, 2.0 / side)
        gx = torch.empty_like(x)
        f.ft_backward(plan, dP, gx)
        torch.cuda.synchronize()
        P, dP, gx, loss = P.cpu().numpy(), dP.cpu().numpy(), gx.cpu().numpy(), loss.cpu().numpy()
    for i in range(n):
        P_ref = oracle.funnel_ref(imgs[i], side, side)
        l_ref, _ = oracle.map_loss_grad_ref(P_ref, tgts[i], side)
        assert abs(loss[i] - l_ref) <= 1e-5 * l_ref
        # the adjoint of the GPU's own dP (exact up to FP32 rounding)
        g_adj = oracle.adjoint_ref(dP[i].astype(np.float64), side, side)
        assert _gpu.rel_l2(gx[i], g_adj) <= TOL
        # the full FP64 chain; cells where the two maps disagree in sign are tiny
        _, dP_ref = oracle.map_loss_grad_ref(P_ref, tgts[i], side)
        g_ref = oracle.adjoint_ref(dP_ref / n, side, side)
        assert _gpu.rel_l2(gx[i], g_ref) <= 1e-4


def test_autograd_wrapper(torch):
    from paper_1904_09409_gb300 import funnel as f
    imgs, tgts = workload(128, 3, start=50)
    with f.Plan(128, 128, 128, 128) as plan:
        x = torch.from_numpy(imgs).cuda().requires_grad_(True)
        t = torch.from_numpy(tgts).cuda()
        P = f.funnel_transform(x, plan)
        loss = ((P.abs() * (2.0 / 128) - t) ** 2).mean()
        loss.backward()
        # the same gradient through the C ABI calls
        _, dP = f.ft_abs_mse_grad(plan, P.detach().contiguous(), t, 2.0 / 128)
        gx = torch.empty_like(x)
        f.ft_backward(plan, dP, gx)
        torch.cuda.synchronize()
    assert _gpu.rel_l2(x.grad.cpu().numpy(), gx.cpu().numpy().astype(np.float64)) <= 1e-6


@pytest.mark.parametrize("side,n,space,Hp", [(64, 3, "regular", 64), (512, 2, "regular", 512),
                                             (128, 2, "inverse", 128), (96, 2, "regular", 216)])
def test_fused_loss_backward_equals_the_two_calls(torch, side, n, space, Hp):
    """ft_abs_mse_backward = ft_abs_mse_grad + ft_backward without storing the
    map gradient: the losses agree to FP32 rounding, the image gradients to the
    tolerance, and both are deterministic.  n_intercept 216 (no fixed-length
    kernel) takes the fallback through the workspace."""
    from paper_1904_09409_gb300 import funnel as f
    imgs, _ = workload(side, n)
    rng = np.random.default_rng(side + n)
    with f.Plan(side, side, side, Hp, space=space) as plan:
        x = torch.from_numpy(imgs).cuda()
        P = torch.empty((n, plan.Hp, plan.S), dtype=torch.float32, device="cuda")
        f.ft_forward(plan, x, P)
        t = torch.from_numpy(rng.random((n, plan.Hp, plan.S)).astype(np.float32)).cuda()
        loss_a, dP = f.ft_abs_mse_grad(plan, P, t, 2.0 / side)
        gx_a = torch.empty_like(x)
        f.ft_backward(plan, dP, gx_a)
        loss_b, gx_b = f.ft_abs_mse_backward(plan, P, t, 2.0 / side)
        loss_c, gx_c = f.ft_abs_mse_backward(plan, P, t, 2.0 / side)
        torch.cuda.synchronize()
    assert torch.equal(loss_b, loss_c) and torch.equal(gx_b, gx_c)
    la, lb = loss_a.cpu().numpy().astype(np.float64), loss_b.cpu().numpy().astype(np.float64)
    assert np.all(np.abs(la - lb) <= 2e-6 * la)
    for i in range(n):
        assert _gpu.rel_l2(gx_b[i].cpu().numpy(), gx_a[i].cpu().numpy().astype(np.float64)) <= 1e-6
        # and against the FP64 adjoint of the oracle's own loss gradient of this map
        _, dP_ref = oracle.map_loss_grad_ref(P[i].cpu().numpy().astype(np.float64),
                                             t[i].cpu().numpy().astype(np.float64), side)
        g_ref = oracle.adjoint_ref(dP_ref / n, side, side, "linear") if space == "regular" else None
        if g_ref is not None:
            assert _gpu.rel_l2(gx_b[i].cpu().numpy(), g_ref) <= TOL
