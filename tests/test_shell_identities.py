"""The arithmetic of the fused kernel's shell loop (MSE schemes whose b-value shells have even
lengths), written out in float64 on the CPU and checked against the oracle's Eqs. 3-5:

  c' = s c = g' . d with s = sqrt(b D_par log2 e), g' = s g;
  m = c'^2 - log2 f_in, f_in e1 = 2^(-m), (1 - f_in) p = 2^(-rho m + C0 - b D_perp log2 e),
  rho = 1 - D_perp / D_par, C0 = log2(1 - f_in) - rho log2 f_in;
  S = S0 T0 + sum_k S0 f_k (f_in e1 + (1 - f_in) p), T0 the shell's isotropic mixture;
  dS/dd_k = S0 f_k (-2 ln 2) c' (f_in e1 + rho (1 - f_in) p) g' (the same factor for every shell).

The signal must equal the oracle's and the closed-form direction derivative must equal autograd
of the oracle's signal, on a scheme with a b = 0 shell (where f_in e1 = f_in, (1 - f_in) p =
1 - f_in) and shells up to b = 13,192."""
import math

import numpy as np
import torch

from oracle import prism_oracle as O

LOG2E = 1.0 / math.log(2.0)


def _problem(seed=0, V=40, K=3):
    g = torch.Generator().manual_seed(seed)
    bvals = torch.tensor([0.0] * 4 + [5.0] * 2 + [1000.0] * 6 + [3000.0] * 8 + [13192.0] * 4, dtype=torch.float64)
    bvecs = torch.randn(len(bvals), 3, generator=g, dtype=torch.float64)
    bvecs = bvecs / bvecs.norm(dim=1, keepdim=True)
    bvecs[bvals == 0] = 0.0
    s0 = 0.5 + torch.rand(V, generator=g, dtype=torch.float64)
    frac = torch.softmax(torch.randn(V, K + 3, generator=g, dtype=torch.float64), dim=1)
    d = torch.randn(V, K, 3, generator=g, dtype=torch.float64)
    d = d / d.norm(dim=2, keepdim=True)
    fin = 0.05 + 0.9 * torch.rand(V, generator=g, dtype=torch.float64)
    return s0, frac, d, fin, bvals, bvecs


def _shell_form(s0, frac, d, fin, bvals, bvecs):
    K = d.shape[1]
    rho = 1.0 - O.D_PERP / O.D_PAR
    s = torch.sqrt(bvals * O.D_PAR * LOG2E)                     # per measurement (its shell)
    gp = s[:, None] * bvecs                                      # g' = s g
    cp = torch.einsum("vkj,nj->vkn", d, gp)                      # c' = g' . d
    lfin = torch.log2(fin)[:, None, None]
    c0 = (torch.log2(1.0 - fin) - rho * torch.log2(fin))[:, None, None]
    m = cp * cp - lfin
    fe1 = torch.exp2(-m)                                         # f_in e1
    omp = torch.exp2(-rho * m + c0 - bvals * O.D_PERP * LOG2E)   # (1 - f_in) p
    t0 = (frac[:, 0:1] * torch.exp(-bvals * O.D_CSF) + frac[:, 1:2] * torch.exp(-bvals * O.D_GM)
          + frac[:, K + 2:K + 3] * torch.exp(-bvals * O.D_RES))
    S = s0[:, None] * t0 + (s0[:, None, None] * frac[:, 2:K + 2, None] * (fe1 + omp)).sum(1)
    return S, cp, fe1, omp, gp, rho


def test_shell_form_reproduces_the_tissue_signal():
    s0, frac, d, fin, bvals, bvecs = _problem(0)
    S, *_ = _shell_form(s0, frac, d, fin, bvals, bvecs)
    ref = O.tissue_signal(s0, frac, d, fin, bvals, bvecs)
    np.testing.assert_allclose(S.numpy(), ref.numpy(), rtol=1e-12, atol=1e-15)


def test_shell_form_direction_derivative_matches_autograd():
    s0, frac, d, fin, bvals, bvecs = _problem(1)
    K = d.shape[1]
    r = torch.randn(s0.shape[0], len(bvals), generator=torch.Generator().manual_seed(5), dtype=torch.float64)
    dd = d.clone().requires_grad_(True)
    (r * O.tissue_signal(s0, frac, dd, fin, bvals, bvecs)).sum().backward()
    _, cp, fe1, omp, gp, rho = _shell_form(s0, frac, d, fin, bvals, bvecs)
    w = s0[:, None, None] * frac[:, 2:K + 2, None] * (-2.0 * math.log(2.0)) * cp * (fe1 + rho * omp)   # [V,K,N]
    closed = torch.einsum("vn,vkn,nj->vkj", r, w, gp)
    np.testing.assert_allclose(closed.numpy(), dd.grad.numpy(), rtol=1e-10, atol=1e-13)


def test_b0_shell_reduces_to_the_fraction_sum():
    s0, frac, d, fin, bvals, bvecs = _problem(2)
    _, _, fe1, omp, _, _ = _shell_form(s0, frac, d, fin, bvals, bvecs)
    b0 = bvals == 0
    np.testing.assert_allclose(fe1[..., b0].numpy(), fin[:, None, None].expand(-1, d.shape[1], int(b0.sum())).numpy(),
                               rtol=1e-14)
    np.testing.assert_allclose(omp[..., b0].numpy(), (1.0 - fin)[:, None, None].expand(-1, d.shape[1], int(b0.sum())).numpy(),
                               rtol=1e-13)
