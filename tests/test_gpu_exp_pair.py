"""The FP64 elementary functions of the kernels (the exponential pair of G_s and
1/G_s, the single exponential, the logarithm) against CUDA's functions (through
torch) and numpy's; the mixed path's shorter exponential pair and logarithm
against their stated bounds."""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


def _pair(x):
    from paper_2202_02319_b300 import native as nv
    xd = torch.as_tensor(x, dtype=torch.float64).cuda()
    ep, em = torch.empty_like(xd), torch.empty_like(xd)
    nv.probe_exp_pair(xd, ep, em)
    torch.cuda.synchronize()
    return xd, ep, em


def test_exp_pair_within_a_few_ulp():
    g = np.random.default_rng(11)
    ln2_64 = np.log(2.0) / 64.0
    k = np.arange(-200, 201)
    x = np.concatenate([
        g.uniform(-700.0, 700.0, 400_000), g.uniform(-1.0, 1.0, 200_000), g.uniform(-30.0, 30.0, 200_000),
        k * ln2_64, np.nextafter(k * ln2_64, np.inf), np.nextafter(k * ln2_64, -np.inf),
        [0.0, -0.0, 1e-300, -1e-300, 706.9, -706.9],
    ])
    xd, ep, em = _pair(x)
    ref = np.exp(x)
    for got, want in ((ep.cpu().numpy(), ref), (em.cpu().numpy(), np.exp(-x))):
        assert float(np.max(np.abs(got - want) / want)) < 1e-15
    for got, want in ((ep, torch.exp(xd)), (em, torch.exp(-xd))):
        assert float(((got - want).abs() / want).max()) < 1e-15
    assert float((ep * em - 1.0).abs().max()) < 2e-15


def test_exp_pair_saturates_beyond_707_and_handles_empty():
    xd, ep, em = _pair(np.array([800.0, -800.0, 1e6, -1e6]))
    ep, em = ep.cpu().numpy(), em.cpu().numpy()
    assert np.isfinite(ep).all() and np.isfinite(em).all() and (ep > 0).all() and (em > 0).all()
    big = np.exp(706.0)
    assert ep[0] >= big and em[1] >= big and ep[2] >= big and em[3] >= big
    assert em[0] <= 1.0 / big and ep[1] <= 1.0 / big
    _pair(np.zeros(0))


def test_log64_within_a_few_ulp():
    from paper_2202_02319_b300 import native as nv
    g = np.random.default_rng(12)
    x = np.concatenate([g.uniform(50.0, 1.0e5, 400_000), np.exp(g.uniform(-700.0, 700.0, 200_000)),
                        g.uniform(0.99, 1.01, 100_000), [1.0, 2.0, 0.5, 1.0 + 1.0 / 128.0, 1.0 - 1e-16, 1e-300, 1e300]])
    xd = torch.as_tensor(x, dtype=torch.float64).cuda()
    y = torch.empty_like(xd)
    nv.probe_log(xd, y)
    torch.cuda.synchronize()
    got = y.cpu().numpy()
    ref = np.log(x)
    # absolute error against |ln x| + 1: a few ulp of the result, and of 1 near x = 1
    assert float(np.max(np.abs(got - ref) / (np.abs(ref) + 1.0))) < 1e-15
    assert float(((y - torch.log(xd)).abs() / (torch.log(xd).abs() + 1.0)).max()) < 1e-15
    assert got[x == 1.0][0] == 0.0


def test_single_exp64_within_a_few_ulp():
    from paper_2202_02319_b300 import native as nv
    g = np.random.default_rng(13)
    x = np.concatenate([g.uniform(-700.0, 700.0, 400_000), g.uniform(-1.0, 1.0, 200_000),
                        np.arange(-200, 201) * np.log(2.0) / 128.0, [0.0, -0.0, 706.9, -706.9]])
    xd = torch.as_tensor(x, dtype=torch.float64).cuda()
    y = torch.empty_like(xd)
    nv.probe_exp(xd, y)
    torch.cuda.synchronize()
    assert float(np.max(np.abs(y.cpu().numpy() - np.exp(x)) / np.exp(x))) < 1e-15
    assert float(((y - torch.exp(xd)).abs() / torch.exp(xd)).max()) < 1e-15


def test_mixed_exp_pair_within_2e_13():
    from paper_2202_02319_b300 import native as nv
    g = np.random.default_rng(12)
    x = np.concatenate([g.uniform(-700.0, 700.0, 400_000), g.uniform(-1.0, 1.0, 200_000),
                        g.uniform(-60.0, 60.0, 200_000), np.arange(-2000, 2001) * (np.log(2.0) / 256.0),
                        [0.0, -0.0, 700.0, -700.0]])
    xd = torch.as_tensor(x, dtype=torch.float64).cuda()
    ep, em = torch.empty_like(xd), torch.empty_like(xd)
    nv.probe_exp_pair_mixed(xd, ep, em)
    torch.cuda.synchronize()
    for got, want in ((ep.cpu().numpy(), np.exp(x)), (em.cpu().numpy(), np.exp(-x))):
        assert float(np.max(np.abs(got - want) / want)) < 2e-13


def test_mixed_log_within_5e_14():
    from paper_2202_02319_b300 import native as nv
    g = np.random.default_rng(13)
    x = np.concatenate([g.uniform(50.0, 1.0e5, 400_000), np.exp2(g.uniform(-60.0, 60.0, 200_000)),
                        g.uniform(0.99, 1.01, 100_000), [1.0, 2.0, 0.5, 300.0, 1.0 + 1.0 / 128.0]])
    xd = torch.as_tensor(x, dtype=torch.float64).cuda()
    y = torch.empty_like(xd)
    nv.probe_log_mixed(xd, y)
    torch.cuda.synchronize()
    assert float(np.max(np.abs(y.cpu().numpy() - np.log(x)))) < 5e-14
