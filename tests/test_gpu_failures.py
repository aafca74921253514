"""Failure paths that a test can reach without faulting, trapping or hanging
the GPU: a device-side wait that runs out (the tensor-core kernels' bounded
mbarrier waits, with the plan's limit set to 0 cycles so that every wait gives
up before its first try) and device allocations that fail (injected on the
host, before cudaMalloc is called).  In both cases the call reports the error
and the plan and the CUDA context stay usable: the next call gives the right
answer."""
import numpy as np
import pytest

import oracle
from tests import _gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    return _gpu.torch_cuda()


def _images(n, H, W, seed):
    rng = np.random.default_rng(seed)
    return rng.standard_normal((n, H, W)).astype(np.float32)


# (H, W, S, H'): S = 4096 puts steps 2-3 on the tensor cores, H' = 4096 steps 1 and 4
@pytest.mark.parametrize("H,W,S,Hp", [(64, 64, 4096, 64), (64, 64, 64, 4096)])
@pytest.mark.parametrize("precision", ["bf16x3", "bf16x6"])
def test_tensor_core_wait_timeout(torch, H, W, S, Hp, precision):
    from paper_1904_09409_gb300 import funnel as f
    imgs = _images(2, H, W, seed=H + S)
    with f.Plan(H, W, S, Hp) as plan:
        f.ft_plan_set_precision(plan, precision)
        assert f.ft_plan_get_wait_cycles(plan) == f.FT_WAIT_CYCLES_DEFAULT
        with pytest.raises(f.FunnelError):
            f.ft_plan_set_wait_cycles(plan, -1)
        f.ft_plan_set_wait_cycles(plan, 0)              # every wait gives up at once
        _gpu.forward(plan, imgs)
        with pytest.raises(f.FunnelError) as e:
            f.ft_plan_tc_errors(plan)
        assert e.value.status == f.FT_ERR_TIMEOUT
        assert f.ft_plan_tc_errors(plan) == 0           # the flags were cleared
        # the context is still usable: the default bound gives the right map
        f.ft_plan_set_wait_cycles(plan, f.FT_WAIT_CYCLES_DEFAULT)
        got = _gpu.forward(plan, imgs)
        assert f.ft_plan_tc_errors(plan) == 0
    tol = 5e-5 if (precision == "bf16x3" and Hp == 4096) else 1e-5
    for i in range(2):
        assert _gpu.rel_l2(got[i], oracle.funnel_ref(imgs[i], S, Hp)) <= tol


def test_injected_allocation_failure_leaves_the_plan_usable(torch):
    from paper_1904_09409_gb300 import funnel as f
    H = W = 256
    imgs = _images(3, H, W, seed=1)
    with f.Plan(H, W, W, H) as plan:
        x = torch.from_numpy(imgs).cuda()
        m = torch.full((3, H, W), float("nan"), device="cuda")
        f.ft_plan_inject_alloc_failures(plan, 1)
        with pytest.raises(f.FunnelError) as e:
            f.ft_forward(plan, x, m)
        assert e.value.status == f.FT_ERR_OOM
        assert "workspace" in f.ft_last_error()
        torch.cuda.synchronize()
        assert bool(torch.isnan(m).all())               # nothing was launched
        f.ft_forward(plan, x, m)                        # allocates again
        torch.cuda.synchronize()
        got = m.cpu().numpy()
        # the host-buffer call: its first buffer fails, then everything works
        f.ft_plan_inject_alloc_failures(plan, 1)
        with pytest.raises(f.FunnelError) as e:
            f.ft_detect_host(plan, imgs, 5)
        assert e.value.status == f.FT_ERR_OOM
        assert "image" in f.ft_last_error()
        out, cnt = f.ft_detect_host(plan, imgs, 5)
        recs = out.numpy().view(f.PEAK_DTYPE).reshape(3, 5)
        cnt = cnt.numpy()
        f.ft_plan_inject_alloc_failures(plan, 3)
        f.ft_plan_inject_alloc_failures(plan, 0)        # cleared
        f.ft_forward(plan, x, m)
        torch.cuda.synchronize()
    for i in range(3):
        assert _gpu.rel_l2(got[i], oracle.funnel_ref(imgs[i], W, H)) <= 1e-5
        pk = [(int(p["t"]), int(p["s"]), float(p["value"])) for p in recs[i][:cnt[i]]]
        assert pk == oracle.peaks_ref(np.abs(got[i]).astype(np.float64), 5)


@pytest.mark.parametrize("interp", ["linear", "cubic"])
def test_bulk_copy_wait_timeout_fp32_rows(torch, interp):
    """Step 1 stages its image columns and step 4 its Hermitian halves with tensor
    copies, the row kernel its spectrum rows with bulk copies, all completing on
    an mbarrier; with the plan's wait limit at 0 every such wait gives up: the
    block drains its copies, writes nothing, and ft_plan_tc_errors returns
    FT_ERR_TIMEOUT with bits 1, 2 and 3; with the default limit the next map is
    the oracle's."""
    from paper_1904_09409_gb300 import funnel as f
    H = W = 256
    imgs = _images(2, H, W, seed=3)
    with f.Plan(H, W, W, H, interp) as plan:
        assert f.ft_plan_tc_errors(plan) == 0
        f.ft_plan_set_wait_cycles(plan, 0)
        _gpu.forward(plan, imgs)
        with pytest.raises(f.FunnelError) as e:
            f.ft_plan_tc_errors(plan)
        assert e.value.status == f.FT_ERR_TIMEOUT
        assert "bulk copy" in f.ft_last_error()
        assert "flags 0xe" in str(e.value)             # steps 1 and 4's tensor copies, the rows' bulk copies
        f.ft_plan_set_wait_cycles(plan, f.FT_WAIT_CYCLES_DEFAULT)
        got = _gpu.forward(plan, imgs)
        assert f.ft_plan_tc_errors(plan) == 0
    for i in range(2):
        assert _gpu.rel_l2(got[i], oracle.funnel_ref(imgs[i], W, H, interp)) <= 1e-5


def test_loss_backward_tensor_copy_timeout(torch):
    """The first kernel of ft_abs_mse_backward stages its map columns with tensor
    copies (bit 3) and the adjoint of step 1 its Hermitian halves (bit 2); with
    the wait limit at 0 both give up, the blocks drain their copies and write
    nothing, and ft_plan_tc_errors returns FT_ERR_TIMEOUT with flags 0xc; with
    the default limit the loss and the image gradient equal ft_abs_mse_grad
    followed by ft_backward."""
    from paper_1904_09409_gb300 import funnel as f
    H = W = 256
    imgs = _images(2, H, W, seed=5)
    rng = np.random.default_rng(5)
    with f.Plan(H, W, W, H) as plan:
        P = torch.from_numpy(_gpu.forward(plan, imgs)).cuda()
        tgt = torch.from_numpy(rng.uniform(0.0, 1.0, size=(2, H, W)).astype(np.float32)).cuda()
        f.ft_plan_set_wait_cycles(plan, 0)
        f.ft_abs_mse_backward(plan, P, tgt, 2.0 / W)
        with pytest.raises(f.FunnelError) as e:
            f.ft_plan_tc_errors(plan)
        assert e.value.status == f.FT_ERR_TIMEOUT
        assert "flags 0xc" in str(e.value)
        f.ft_plan_set_wait_cycles(plan, f.FT_WAIT_CYCLES_DEFAULT)
        loss, gx = f.ft_abs_mse_backward(plan, P, tgt, 2.0 / W)
        loss_g, gmap = f.ft_abs_mse_grad(plan, P, tgt, 2.0 / W)
        gx_ref = torch.empty_like(gx)
        f.ft_backward(plan, gmap, gx_ref)
        torch.cuda.synchronize()
        assert f.ft_plan_tc_errors(plan) == 0
    assert torch.allclose(loss, loss_g, rtol=1e-5, atol=0.0)
    assert float((gx - gx_ref).norm() / gx_ref.norm()) <= 1e-5
