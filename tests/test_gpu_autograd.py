"""Differentiation through the apply: IDBFApply's backward is the adjoint butterfly.

For the loss L(x) = ||K x - b||^2 PyTorch's complex autograd returns x.grad = 2 K^* (K x - b).
Checked against (i) central finite differences of L along random complex directions (exact up
to rounding for a quadratic loss), (ii) the dense gradient 2 K^* (K x - b) with the oracle's
dense K (the factorization approximates K to O(eps)), (iii) torch.autograd.gradcheck on a small
case."""
import numpy as np
import pytest
import torch

import paper_1809_10573_gb300 as P
from oracle import kernels
from paper_1809_10573_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__
    __graft_entry__.build()


@pytest.fixture(scope="module")
def fio4096():
    N, n0, eps = 4096, 64, 1e-8
    x, xi = inputs.uniform_grid(N)
    plan = P.Plan.build(x, xi, eps=eps, leaf=n0, kernel="fio", c_profile=0, oversample=2.0, oversample_leaf=4.0)
    plan.set_storage(P.STORE_C128, P.STORE_DF64, P.STORE_C64)
    Kd = kernels.Kernel(kernels.KIND_FIO, c_profile=0).entries(x, xi, np.arange(N), np.arange(N))
    return N, eps, plan, Kd


def _loss(plan, x, b, mode):
    r = P.apply(plan, x, mode) - b
    return (r.abs() ** 2).sum()


@pytest.mark.parametrize("mode,tol", [(P.MODE_FP64, 1e-9), (P.MODE_DF64, 1e-9)])
def test_gradient_matches_finite_differences(fio4096, mode, tol):
    N, eps, plan, Kd = fio4096
    X = torch.from_numpy(inputs.complex_gaussian(N, 3, seed=51)).cuda()
    B = torch.from_numpy(inputs.complex_gaussian(N, 3, seed=52)).cuda()
    x = X.clone().requires_grad_(True)
    _loss(plan, x, B, mode).backward()
    g = x.grad.detach()
    for k in range(3):
        v = torch.from_numpy(inputs.complex_gaussian(N, 3, seed=60 + k)).cuda()
        h = 1e-3
        with torch.no_grad():
            fd = (_loss(plan, X + h * v, B, mode) - _loss(plan, X - h * v, B, mode)) / (2 * h)
        an = torch.real(torch.vdot(g.flatten(), v.flatten()))
        assert abs(float(fd - an)) <= tol * float(abs(an)) + 1e-9 * float(_loss(plan, X, B, mode))


def test_gradient_matches_dense_adjoint(fio4096):
    N, eps, plan, Kd = fio4096
    X = inputs.complex_gaussian(N, 2, seed=53)
    B = inputs.complex_gaussian(N, 2, seed=54)
    x = torch.from_numpy(X).cuda().requires_grad_(True)
    _loss(plan, x, torch.from_numpy(B).cuda(), P.MODE_DF64).backward()
    dense = 2 * Kd.conj().T @ (Kd @ X - B)
    got = x.grad.cpu().numpy()
    assert np.linalg.norm(got - dense) / np.linalg.norm(dense) < 10 * eps


def test_fp32_gradient_of_the_split_precision_path(fio4096):
    N, eps, plan, Kd = fio4096
    X = inputs.complex_gaussian(N, 4, seed=55).astype(np.complex64)
    B = inputs.complex_gaussian(N, 4, seed=56).astype(np.complex64)
    x = torch.from_numpy(X).cuda().requires_grad_(True)
    _loss(plan, x, torch.from_numpy(B).cuda(), P.MODE_FP32).backward()
    dense = 2 * Kd.conj().T @ (Kd @ X.astype(np.complex128) - B)
    got = x.grad.cpu().numpy()
    assert np.linalg.norm(got - dense) / np.linalg.norm(dense) < 1e-5


def test_gradcheck_small():
    N = 256
    x, xi = inputs.uniform_grid(N)
    plan = P.Plan.build(x, xi, eps=1e-12, leaf=16, kernel="fio", c_profile=1)
    z = torch.from_numpy(inputs.complex_gaussian(N, 1, seed=57)[:, 0]).cuda().requires_grad_(True)
    assert torch.autograd.gradcheck(lambda t: P.apply(plan, t, P.MODE_FP64), (z,), eps=1e-6, atol=1e-7, rtol=1e-6,
                                    fast_mode=True)
