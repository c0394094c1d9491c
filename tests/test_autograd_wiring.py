"""CPU checks of the torch.autograd.Function wiring of PrismLoss (no GPU, no library).

A stand-in handle with the Fitter's forward / backward contract (backward is the gradient at
the point of the handle's last forward) evaluates J(theta, g) = sum w theta^2 + sum c g^2 in
plain torch. The checks: groups=None (the handle's current group parameters) gets no
gradient and raises nothing; two nodes on one handle in one graph each get the gradient at
their own point; a step between forward and backward does not leak into the gradient.
"""
import torch

import paper_2604_00250_gb300 as prism


class FakeHandle:
    def __init__(self, V=3, Q=4, GP=5):
        self.n_vox, self.Q, self.n_group_params = V, Q, GP
        self.w = torch.linspace(0.5, 2.0, V * Q, dtype=torch.float32).reshape(V, Q)
        self.c = torch.linspace(1.0, 3.0, GP, dtype=torch.float32)
        self.theta = torch.zeros(V, Q)
        self.groups = torch.ones(GP)
        self._fwd_token = None
        self.forward_calls = 0

    def groups_device(self):
        return self.groups.clone()

    def forward(self, theta=None, groups=None):
        if theta is not None:
            self.theta = theta.clone()
        if groups is not None:
            self.groups = groups.clone()
        self.forward_calls += 1
        self._fwd_token = object()
        J = (self.w * self.theta ** 2).sum() + (self.c * self.groups ** 2).sum()
        return J.to(torch.float64).reshape(1), None

    def backward(self):
        return 2 * self.w * self.theta, 2 * self.c * self.groups

    def step(self):
        self.theta = self.theta - 1.0
        self._fwd_token = None


def test_groups_none_gets_no_gradient():
    f = FakeHandle()
    th = torch.randn(3, 4, requires_grad=True)
    J = prism.PrismLoss.apply(th, None, f)
    J.backward()
    torch.testing.assert_close(th.grad, 2 * f.w * th.detach())


def test_groups_gradient_and_upstream_scale():
    f = FakeHandle()
    th = torch.randn(3, 4, requires_grad=True)
    g = torch.randn(5, requires_grad=True)
    (3.0 * prism.PrismLoss.apply(th, g, f)).backward()
    torch.testing.assert_close(th.grad, 3.0 * 2 * f.w * th.detach())
    torch.testing.assert_close(g.grad, 3.0 * 2 * f.c * g.detach())


def test_two_nodes_on_one_handle():
    f = FakeHandle()
    t1 = torch.randn(3, 4, requires_grad=True)
    t2 = torch.randn(3, 4, requires_grad=True)
    J = prism.PrismLoss.apply(t1, None, f) + 2.0 * prism.PrismLoss.apply(t2, None, f)
    J.backward()
    torch.testing.assert_close(t1.grad, 2 * f.w * t1.detach())
    torch.testing.assert_close(t2.grad, 2.0 * 2 * f.w * t2.detach())


def test_step_between_forward_and_backward():
    f = FakeHandle()
    th = torch.randn(3, 4, requires_grad=True)
    J = prism.PrismLoss.apply(th, None, f)
    f.step()
    J.backward()
    torch.testing.assert_close(th.grad, 2 * f.w * th.detach())
    assert f.forward_calls == 2


def test_same_point_is_not_recomputed():
    f = FakeHandle()
    th = torch.randn(3, 4, requires_grad=True)
    prism.PrismLoss.apply(th, None, f).backward()
    assert f.forward_calls == 1
