"""PRISM FP64 CPU oracle -- TEST INFRASTRUCTURE ONLY.

Only tests, the package's smoke check and the benchmark's CPU-baseline leg may
import this module. The product path (the CUDA library and its binding) never
calls it, and it shares no code with the CUDA sources.

It is the plain, slow definition of one PRISM fit (Abouagour et al., "PRISM:
Differentiable Analysis-by-Synthesis for Fixel Recovery in Diffusion MRI"),
in float64 PyTorch CPU ops, following the paper in order:

  * tissue model, Sec. 2.2 Eqs. 3-5 (S, E_iso, stick-and-zeppelin E_wm),
  * per-voxel parameterisation, Sec. 2.2 "Per-voxel parameters" and Sec. 2.5
    "Constraints and solver" (softplus S0, softmax fractions, sigmoid f_intra,
    l2-normalised directions),
  * calibration chain, Sec. 2.3 Eq. 6 (bias field exp(upsample(b_lr)),
    per-measurement exp(alpha_n) and beta_n, sigma = exp(sigma_log)),
  * data terms, Sec. 2.5 Eq. 8 (MSE) and Eq. 9 (Rician NLL), on b0-normalised
    signals (Sec. 2.5, first paragraph),
  * priors, Sec. 2.4 (Huber-Laplacian Eq. 7, repulsion, L1 sparsity,
    directional continuity, calibration L2 and TV),
  * total objective, Sec. 2.5 (L_data + sum_i lambda_i R_i + R_cal),
  * Adam (the paper's Table 2 comparator; Kingma & Ba 2015, Algorithm 1).

The gradient is torch autograd of that objective (exact up to rounding), so it
is independent of any hand-derived adjoint. Where the paper is silent the
readings used are listed at the bottom of this docstring and in the option
defaults; every one is shared, by documentation only, with the CUDA path.

Readings (paper silent or ambiguous):
  R1  solver: Adam (torch defaults beta=(0.9, 0.999), eps=1e-8, bias-corrected,
      lr 1e-2), one step counter for every parameter.
  R2  MSE: (1/|M|) sum_{x,n}, |M| = masked voxels of the volume (group).
  R3  NLL: plain sum over voxels and measurements of the volume.
  R4  f_intra: one scalar per voxel shared by its K fibers.
  R5  fraction logits ordered [csf, gm, wm_1..wm_K, res].
  R6  S0 = softplus(s) = max(s, 0) + log1p(exp(-|s|)).
  R7  d = v / max(|v|, 1e-12).
  R8  b in s/mm^2, diffusivities in mm^2/s (3.0e-3, 0.9e-3, 0.2e-3, 1.7e-3, 0.4e-3).
  R9  bias upsampling: trilinear, align_corners=False over the whole volume grid:
      u = clamp((i + 0.5) * 8 / n - 0.5, 0, 7).
  R10 calibration (alpha, beta, b_lr) and sigma are per volume.
  R11 calibration regularisers: w_a mean_n alpha^2 + w_b mean_n beta^2 +
      w_blr mean b_lr^2 + w_tv (1/|M|) sum_{x, axis: x, x+e in M} sqrt((B(x+e)-B(x))^2 + eps_tv),
      w_* = 1e-3, eps_tv = 1e-6.
  R12 Huber rho(r) = r^2/2 if |r| <= delta else delta (|r| - delta/2), summed over
      the K+3 fractions.
  R13 neighbourhood: 6-connected, masked and in the same patch; |N(x)| = 0 => 0.
  R14 repulsion: lambda_rep * mean_x sum_{i<j} f_wm,i f_wm,j |d_i . d_j|, d|x|/dx(0) = 0.
  R15 sparsity: lambda_sparse * mean_x sum_k f_wm,k [f_wm,k < tau].
  R16 directional continuity: lambda_dir * (1/|M|) sum_x (1/|N(x)|)
      sum_{x' in N(x)} sum_k (1 - (d_k(x) . d_k(x'))^2).
  R25 orphan-WM suppression (Sec. 2.4, form unstated): lambda_orphan * mean_x
      exp(-S0(x) / s_orphan) sum_k f_wm,k(x), s_orphan = 0.05 (negligible at S0 ~ 1).
  R26 fiber ordering (Sec. 2.4, form unstated): lambda_order * mean_x
      sum_{k<K} max(0, f_wm,k+1 - f_wm,k), a hinge toward descending fractions; its
      derivative at the kink (equal fractions, e.g. the equal-logit start) is 0, as for R14.
  R27 26-connectivity: the 26 voxels of the 3x3x3 cube, masked and in the same patch.
  R18 sigma init: pooled std of the b0-normalised b=0 repeats of the volume
      (clamped to >= 1e-3); sigma_init option when fewer than two b=0 volumes.
  R19 b=0 measurements: b <= 50 s/mm^2; b0 = their per-voxel mean.
  R23 group parameters use the same Adam and step counter.
"""
from dataclasses import dataclass, field
import math

import numpy as np
import torch

F64 = torch.float64

# Fixed diffusivities, Sec. 2.2 (x 1e-3 mm^2/s).
D_CSF, D_GM, D_RES = 3.0e-3, 0.9e-3, 0.2e-3
D_PAR, D_PERP = 1.7e-3, 0.4e-3
B0_MAX = 50.0          # R19
NORM_EPS = 1e-12       # R7
NBR6 = ((1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0), (0, 0, 1), (0, 0, -1))
NBR26 = NBR6 + tuple((i, j, k) for i in (-1, 0, 1) for j in (-1, 0, 1) for k in (-1, 0, 1)
                     if abs(i) + abs(j) + abs(k) > 1)


@dataclass
class Options:
    K: int = 3
    loss: str = "mse"                  # "mse" (Eq. 8) or "nll" (Eq. 9)
    calibration: bool = False          # Sec. 2.3 bias + affine
    lam_rep: float = 0.01              # Sec. 2.4 topology priors
    lam_sparse: float = 0.02
    tau: float = 0.15
    lam_sp: float = 0.0                # Huber-Laplacian (Eq. 7), default 0.01 when on
    huber_delta: float = 0.05
    lam_dir: float = 0.0               # directional continuity, 0.005 when on
    lam_orphan: float = 0.0            # R25, 0.01 when on
    s_orphan: float = 0.05
    lam_order: float = 0.0             # R26, 0.01 when on
    connectivity: int = 6              # R13 / R27
    w_alpha: float = 1e-3              # R11
    w_beta: float = 1e-3
    w_blr: float = 1e-3
    w_tv: float = 1e-3
    tv_eps: float = 1e-6
    patch_dim: int = 16
    sigma_init: float = 0.05           # R18 fallback
    lr: float = 1e-2                   # R1
    beta1: float = 0.9
    beta2: float = 0.999
    eps: float = 1e-8


def n_params(K):
    return 4 * K + 5


# ----------------------------------------------------------------------------
# Preprocessing (Sec. 2.5: b0-normalised signals inside the mask).
# ----------------------------------------------------------------------------
class OracleVolume:
    """One volume (one calibration / sigma group) prepared as the paper states it.

    `patches` optionally restricts the voxels to whole patches (for sampled
    checks at full size); the MSE/prior normaliser |M| stays the full volume's.
    """

    def __init__(self, mask, signal, bvals, bvecs, opts, patches=None):
        self.opts = opts
        self.shape = tuple(int(s) for s in mask.shape)
        mask = np.asarray(mask).astype(bool)
        coords_all = np.argwhere(mask)              # C order == mask order
        self.n_mask = coords_all.shape[0]
        P = opts.patch_dim
        pshape = tuple(-(-s // P) for s in self.shape)
        pid_all = np.ravel_multi_index(tuple((coords_all // P).T), pshape)
        if patches is None:
            sel = np.arange(self.n_mask)
        else:
            sel = np.nonzero(np.isin(pid_all, np.asarray(patches)))[0]
        self.sel = sel
        self.coords = coords_all[sel]
        self.pid = pid_all[sel]
        sig = np.asarray(signal)[sel].astype(np.float64)
        self.bvals = torch.as_tensor(np.asarray(bvals, dtype=np.float64))
        self.bvecs = torch.as_tensor(np.asarray(bvecs, dtype=np.float64))
        b0 = self.bvals.numpy() <= B0_MAX
        if not b0.any():
            raise ValueError("no b=0 measurement to normalise by")
        b0mean = sig[:, b0].mean(axis=1)
        if np.any(b0mean <= 0):
            raise ValueError("non-positive b0 mean")
        self.y = torch.as_tensor(sig / b0mean[:, None])
        # R18: pooled std of normalised b0 repeats (computed on the full volume).
        nb0 = int(b0.sum())
        if nb0 >= 2:
            full_b0 = np.asarray(signal)[:, b0].astype(np.float64)
            fb0 = full_b0 / full_b0.mean(axis=1, keepdims=True)
            var = np.sum((fb0 - 1.0) ** 2) / (full_b0.shape[0] * (nb0 - 1))
            self.sigma0 = max(math.sqrt(var), 1e-3)
        else:
            self.sigma0 = opts.sigma_init
        # Neighbour table (R13): masked, same patch, inside the selection.
        index = -np.ones(self.shape, dtype=np.int64)
        index[tuple(self.coords.T)] = np.arange(len(sel))
        pid_grid = -np.ones(self.shape, dtype=np.int64)
        pid_grid[tuple(coords_all.T)] = pid_all
        offs = NBR6 if opts.connectivity == 6 else NBR26
        nb = -np.ones((len(sel), len(offs)), dtype=np.int64)
        for a, off in enumerate(offs):
            c = self.coords + np.asarray(off)
            ok = np.all((c >= 0) & (c < np.asarray(self.shape)), axis=1)
            cc = c[ok]
            j = index[tuple(cc.T)]
            same = pid_grid[tuple(cc.T)] == self.pid[ok]
            nb[np.nonzero(ok)[0], a] = np.where(same, j, -1)
        self.nbr = torch.as_tensor(nb)
        # TV pairs (R11): forward neighbour x+e inside the mask (any patch).
        up = np.zeros((len(sel), 3), dtype=bool)
        for a in range(3):
            c = self.coords.copy()
            c[:, a] += 1
            ok = c[:, a] < self.shape[a]
            up[ok, a] = mask[tuple(c[ok].T)]
        self.tv_up = torch.as_tensor(up)

    @property
    def n_vox(self):
        return int(self.coords.shape[0])

    @property
    def n_meas(self):
        return int(self.bvals.shape[0])


# ----------------------------------------------------------------------------
# Model pieces.
# ----------------------------------------------------------------------------
def softplus(s):
    """R6: log(1 + e^s) evaluated without overflow."""
    return torch.clamp(s, min=0.0) + torch.log1p(torch.exp(-torch.abs(s)))


def transforms(theta, K):
    """Sec. 2.2 per-voxel parameters -> (S0, fractions [V, K+3], dirs [V, K, 3], f_in)."""
    s0 = softplus(theta[:, 0])
    frac = torch.softmax(theta[:, 1:K + 4], dim=1)
    v = theta[:, K + 4:4 * K + 4].reshape(-1, K, 3)
    nrm = torch.sqrt((v * v).sum(-1, keepdim=True))
    d = v / torch.clamp(nrm, min=NORM_EPS)
    fin = torch.sigmoid(theta[:, 4 * K + 4])
    return s0, frac, d, fin


def tissue_signal(s0, frac, d, fin, bvals, bvecs):
    """Sec. 2.2 Eq. 3: S = S0 (f_csf E_csf + f_gm E_gm + sum_k f_wm,k E_wm,k + f_res E_res)."""
    K = d.shape[1]
    b = bvals[None, :]
    e_csf = torch.exp(-b * D_CSF)                     # Eq. 4
    e_gm = torch.exp(-b * D_GM)
    e_res = torch.exp(-b * D_RES)
    cos = torch.einsum("vkj,nj->vkn", d, bvecs)        # cos(theta) = d_k . g_n
    cos2 = cos * cos
    sin2 = 1.0 - cos2
    bb = bvals[None, None, :]
    f_in = fin[:, None, None]
    e_wm = (f_in * torch.exp(-bb * D_PAR * cos2)
            + (1.0 - f_in) * torch.exp(-bb * (D_PAR * cos2 + D_PERP * sin2)))   # Eq. 5
    mix = frac[:, 0:1] * e_csf + frac[:, 1:2] * e_gm + frac[:, K + 2:K + 3] * e_res
    mix = mix + (frac[:, 2:K + 2, None] * e_wm).sum(1)
    return s0[:, None] * mix


def trilinear_weights(coords, shape, grid=8):
    """R9: 8 corner indices (flattened into the grid^3 array) and weights per voxel."""
    idx = []
    wts = []
    lo = []
    fr = []
    for a in range(3):
        n = shape[a]
        u = (coords[:, a].astype(np.float64) + 0.5) * grid / n - 0.5
        u = np.clip(u, 0.0, grid - 1.0)
        i0 = np.minimum(np.floor(u), grid - 2).astype(np.int64)
        lo.append(i0)
        fr.append(u - i0)
    for cx in (0, 1):
        for cy in (0, 1):
            for cz in (0, 1):
                w = ((fr[0] if cx else 1 - fr[0]) * (fr[1] if cy else 1 - fr[1])
                     * (fr[2] if cz else 1 - fr[2]))
                ii = ((lo[0] + cx) * grid + (lo[1] + cy)) * grid + (lo[2] + cz)
                idx.append(ii)
                wts.append(w)
    return torch.as_tensor(np.stack(idx, 1)), torch.as_tensor(np.stack(wts, 1))


def bias_log(blr, coords, shape):
    """upsample(b_lr) at the given voxel coordinates (Sec. 2.3 item 1)."""
    idx, w = trilinear_weights(coords, shape)
    return (blr.reshape(-1)[idx] * w).sum(1)


def log_i0(z):
    """log I0(z) = |z| + log(i0e(|z|)) (modified Bessel function of the first kind)."""
    a = torch.abs(z)
    return a + torch.log(torch.special.i0e(a))


def huber(r, delta):
    """R12: Huber loss with transition delta."""
    a = torch.abs(r)
    return torch.where(a <= delta, 0.5 * r * r, delta * (a - 0.5 * delta))


# ----------------------------------------------------------------------------
# Objective of one volume (Sec. 2.5: L_data + sum_i lambda_i R_i + R_cal).
# ----------------------------------------------------------------------------
def group_init(ov):
    """Initial calibration / noise parameters (identity calibration, Sec. 2.3)."""
    N = ov.n_meas
    return dict(sigma_log=torch.tensor(math.log(ov.sigma0), dtype=F64),
                alpha=torch.zeros(N, dtype=F64), beta=torch.zeros(N, dtype=F64),
                blr=torch.zeros(8, 8, 8, dtype=F64))


def predict(ov, theta, gp):
    """Calibrated prediction y_hat [V, N] (Sec. 2.3 Eq. 6) and the tissue signal S."""
    K = ov.opts.K
    s0, frac, d, fin = transforms(theta, K)
    S = tissue_signal(s0, frac, d, fin, ov.bvals, ov.bvecs)
    if not ov.opts.calibration:
        return S, S
    B = torch.exp(bias_log(gp["blr"], ov.coords, ov.shape))
    yhat = torch.exp(gp["alpha"])[None, :] * B[:, None] * S + gp["beta"][None, :]
    return yhat, S


def objective(ov, theta, gp, n_norm=None):
    """Total objective of one volume and its named parts.

    n_norm overrides |M| (used when `ov` holds a subset of the volume's patches).
    """
    o = ov.opts
    K = o.K
    M = float(n_norm if n_norm is not None else ov.n_mask)
    yhat, _ = predict(ov, theta, gp)
    y = ov.y
    parts = {}
    if o.loss == "mse":
        parts["data"] = ((yhat - y) ** 2).sum() / M                        # Eq. 8
    elif o.loss == "nll":
        sig2 = torch.exp(2.0 * gp["sigma_log"])
        z = y * yhat / sig2
        parts["data"] = (2.0 * gp["sigma_log"] + (y * y + yhat * yhat) / (2.0 * sig2)
                         - log_i0(z)).sum()                                 # Eq. 9
    else:
        raise ValueError(o.loss)
    s0, frac, d, fin = transforms(theta, K)
    fwm = frac[:, 2:K + 2]
    if o.lam_rep:
        rep = 0.0
        for i in range(K):
            for j in range(i + 1, K):
                rep = rep + fwm[:, i] * fwm[:, j] * torch.abs((d[:, i] * d[:, j]).sum(-1))
        parts["rep"] = o.lam_rep * (rep.sum() / M if K > 1 else torch.zeros((), dtype=F64))
    if o.lam_sparse:
        gate = (fwm < o.tau).to(F64)
        parts["sparse"] = o.lam_sparse * (fwm * gate).sum() / M
    if o.lam_orphan:
        parts["orphan"] = o.lam_orphan * (torch.exp(-s0 / o.s_orphan) * fwm.sum(1)).sum() / M   # R25
    if o.lam_order and K > 1:
        parts["order"] = o.lam_order * torch.relu(fwm[:, 1:] - fwm[:, :-1]).sum() / M  # R26
    nbr = ov.nbr
    valid = nbr >= 0
    cnt = valid.sum(1)
    safe = torch.where(valid, nbr, torch.zeros_like(nbr))
    has = cnt > 0
    if o.lam_sp:
        fn = frac[safe] * valid[..., None]                                   # [V, |N|, K+3]
        mean = fn.sum(1) / torch.clamp(cnt, min=1)[:, None]
        r = frac - mean
        parts["spatial"] = o.lam_sp * (huber(r, o.huber_delta).sum(1) * has).sum() / M  # Eq. 7
    if o.lam_dir:
        dn = d[safe]                                                         # [V, |N|, K, 3]
        dot = (d[:, None] * dn).sum(-1)                                      # [V, |N|, K]
        term = ((1.0 - dot * dot).sum(-1) * valid).sum(1) / torch.clamp(cnt, min=1)
        parts["dir"] = o.lam_dir * term.sum() / M
    if o.calibration:
        parts["cal_alpha"] = o.w_alpha * (gp["alpha"] ** 2).mean()
        parts["cal_beta"] = o.w_beta * (gp["beta"] ** 2).mean()
        parts["cal_blr"] = o.w_blr * (gp["blr"] ** 2).mean()
        if o.w_tv:
            B0 = torch.exp(bias_log(gp["blr"], ov.coords, ov.shape))
            tv = torch.zeros((), dtype=F64)
            for a in range(3):
                up = ov.tv_up[:, a]
                if not bool(up.any()):
                    continue
                c1 = ov.coords[up.numpy()].copy()
                c1[:, a] += 1
                B1 = torch.exp(bias_log(gp["blr"], c1, ov.shape))
                diff = B1 - B0[up]
                tv = tv + torch.sqrt(diff * diff + o.tv_eps).sum()
            parts["cal_tv"] = o.w_tv * tv / M
    total = sum(parts.values())
    return total, parts


def trainable_groups(opts):
    names = []
    if opts.loss == "nll":
        names.append("sigma_log")
    if opts.calibration:
        names += ["alpha", "beta", "blr"]
    return names


def value_and_grad(ov, theta, gp, n_norm=None):
    """J, dJ/dtheta [V, Q] and dJ/d(group params) by autograd."""
    th = theta.detach().clone().requires_grad_(True)
    g = {k: v.detach().clone().requires_grad_(True) for k, v in gp.items()}
    J, parts = objective(ov, th, g, n_norm)
    names = trainable_groups(ov.opts)
    grads = torch.autograd.grad(J, [th] + [g[k] for k in names], allow_unused=True)
    gth = grads[0]
    gg = {}
    for k, gr in zip(names, grads[1:]):
        gg[k] = gr if gr is not None else torch.zeros_like(g[k])
    return J.detach(), {k: v.detach() for k, v in parts.items()}, gth, gg


# ----------------------------------------------------------------------------
# Adam (Kingma & Ba 2015, Algorithm 1; torch.optim.Adam's update).
# ----------------------------------------------------------------------------
class Adam:
    def __init__(self, opts):
        self.o = opts
        self.t = 0
        self.state = {}

    def step(self, name, p, g):
        o = self.o
        m, v = self.state.get(name, (torch.zeros_like(p), torch.zeros_like(p)))
        m = o.beta1 * m + (1.0 - o.beta1) * g
        v = o.beta2 * v + (1.0 - o.beta2) * g * g
        bc1 = 1.0 - o.beta1 ** self.t
        bc2 = 1.0 - o.beta2 ** self.t
        p = p - o.lr * (m / bc1) / (torch.sqrt(v / bc2) + o.eps)
        self.state[name] = (m, v)
        return p


# ----------------------------------------------------------------------------
# Rprop (Riedmiller & Braun 1993), the paper's solver (Sec. 2.5, Table 2): per-parameter
# step sizes grow by eta_plus while the gradient keeps its sign, shrink by eta_minus
# after a sign change (that step is skipped and the stored gradient is zeroed), clamped
# to [step_min, step_max]; the update is -sign(g) * step. Initial step = lr.
# ----------------------------------------------------------------------------
class Rprop:
    def __init__(self, opts, etas=(0.5, 1.2), step_sizes=(1e-6, 50.0)):
        self.o = opts
        self.eta_minus, self.eta_plus = etas
        self.step_min, self.step_max = step_sizes
        self.t = 0
        self.state = {}

    def step(self, name, p, g):
        prev, size = self.state.get(name, (torch.zeros_like(p), torch.full_like(p, self.o.lr)))
        sgn = torch.sign(g * prev)
        size = torch.where(sgn > 0, torch.clamp(size * self.eta_plus, max=self.step_max),
                           torch.where(sgn < 0, torch.clamp(size * self.eta_minus, min=self.step_min), size))
        g = torch.where(sgn < 0, torch.zeros_like(g), g)
        p = p - torch.sign(g) * size
        self.state[name] = (g, size)
        return p


# ----------------------------------------------------------------------------
# The fit: T iterations of (objective, gradient, Adam or Rprop) over all volumes.
# ----------------------------------------------------------------------------
@dataclass
class FitResult:
    theta: list
    groups: list
    loss_history: np.ndarray          # [T, n_volumes] objective before each update
    parts_history: list = field(default_factory=list)


def fit(vols, theta0, T, record_parts=False, optimizer="adam"):
    """Runs T iterations of Adam (default) or Rprop; theta0 is a list of [V_g, Q] float64 tensors."""
    thetas = [t.detach().clone().to(F64) for t in theta0]
    groups = [group_init(ov) for ov in vols]
    adam = Adam(vols[0].opts) if optimizer == "adam" else Rprop(vols[0].opts)
    hist = np.zeros((T, len(vols)))
    parts_hist = []
    for it in range(T):
        adam.t += 1
        prow = []
        for gi, ov in enumerate(vols):
            J, parts, gth, gg = value_and_grad(ov, thetas[gi], groups[gi])
            hist[it, gi] = float(J)
            prow.append({k: float(v) for k, v in parts.items()})
            thetas[gi] = adam.step(("theta", gi), thetas[gi], gth)
            for k, gk in gg.items():
                groups[gi][k] = adam.step((k, gi), groups[gi][k], gk)
        if record_parts:
            parts_hist.append(prow)
    return FitResult(thetas, groups, hist, parts_hist)
