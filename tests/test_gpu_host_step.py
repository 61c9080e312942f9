"""The host-buffer RK step (state streamed in by chunks that overlap the first
stage) gives bitwise the state, temperature, time and time step of the
device-buffer step, in place and out of place."""
import pytest
import torch

from paper_2202_02319_b300 import synth
from tests.gpu_common import gpu_setup, laser_tuple

pytestmark = pytest.mark.gpu


def _jet():
    c = synth.case_jet(0, 16)
    c.laser.t0 = 2e-8
    return c


@pytest.mark.parametrize("precision", [0, 1], ids=["fp64", "mixed"])
@pytest.mark.parametrize("in_place", [True, False], ids=["in_place", "separate"])
def test_host_step_equals_device_step(precision, in_place):
    from paper_2202_02319_b300 import native as nv
    case = _jet()
    las = laser_tuple(case)
    mech, ctx, U, T = gpu_setup(case, precision=precision)
    Uh = U.cpu().pin_memory()
    Th = T.cpu().pin_memory()
    Uo = Uh if in_place else torch.empty_like(Uh).pin_memory()
    To = Th if in_place else None
    t = torch.zeros(1, dtype=torch.float64, device="cuda")
    th = torch.zeros(1, dtype=torch.float64, device="cuda")
    dt = torch.zeros(1, dtype=torch.float64, device="cuda")
    dth = torch.zeros(1, dtype=torch.float64, device="cuda")
    for _ in range(3):
        nv.rk_step(ctx, U, T, t, 0.0, case.cfl, las, dt)
        nv.rk_step_host(ctx, Uh, Th, Uo, To, th, 0.0, case.cfl, las, dth)
        torch.cuda.synchronize()
        if not in_place:
            Uh.copy_(Uo)                  # next step starts from the host result
            # the temperature stays on the device copy: feed back the device step's T
            Th.copy_(T.cpu())
        assert torch.equal(U.cpu(), Uo)
        assert float(t) == float(th) and float(dt) == float(dth)
    nv.check(ctx)
    if in_place:
        assert torch.equal(T.cpu(), Th)


@pytest.mark.parametrize("precision", [0, 1], ids=["fp64", "mixed"])
def test_back_to_back_host_steps_equal_device_steps(precision):
    """Five in-place host-buffer steps queued without synchronising (each step's
    copies in wait, chunk by chunk, for the previous step's copies out of the same
    buffer) give bitwise the state of five device-buffer steps."""
    from paper_2202_02319_b300 import native as nv
    case = _jet()
    las = laser_tuple(case)
    mech, ctx, U, T = gpu_setup(case, precision=precision)
    Uh = U.cpu().pin_memory()
    Th = T.cpu().pin_memory()
    t = torch.zeros(1, dtype=torch.float64, device="cuda")
    th = torch.zeros(1, dtype=torch.float64, device="cuda")
    for _ in range(5):
        nv.rk_step(ctx, U, T, t, 0.0, case.cfl, las, None)
    for _ in range(5):
        nv.rk_step_host(ctx, Uh, Th, Uh, Th, th, 0.0, case.cfl, las, None)
    torch.cuda.synchronize()
    nv.check(ctx)
    assert torch.equal(U.cpu(), Uh)
    assert torch.equal(T.cpu(), Th)
    assert float(t) == float(th)
