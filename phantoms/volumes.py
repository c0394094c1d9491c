"""Seeded phantoms shaped like the paper's workloads (Sec. 3 "Datasets").

Generators return `Volume` objects (mask, masked signal rows, scheme, ground
truth). The ground-truth simulator is a multi-compartment stick-and-zeppelin
model with *per-voxel* diffusivities (d_par ~ U(1.5, 2.2)e-3, d_perp ~
U(0.2, 0.8)e-3 mm^2/s) and isotropic CSF/GM/restricted pools at the paper's
diffusivities (Sec. 2.2). Magnitude data get Rician noise |s + sigma (n1 + i n2)|
with sigma = S0 / SNR.
"""
from dataclasses import dataclass, field

import numpy as np

from .schemes import scheme_96, scheme_193, scheme_288, scheme_360

D_ISO = (3.0e-3, 0.9e-3, 0.2e-3)  # CSF, GM, restricted (mm^2/s)


def n_params(K):
    """Raw parameters per voxel: S0, K+3 fraction logits, 3K direction comps, f_intra."""
    return 4 * K + 5


@dataclass
class Volume:
    mask: np.ndarray            # uint8 [nx, ny, nz]
    signal: np.ndarray          # float32 [V, N] masked voxels, C order
    bvals: np.ndarray           # float32 [N]
    bvecs: np.ndarray           # float32 [N, 3]
    gt: dict = field(default_factory=dict)

    @property
    def shape(self):
        return tuple(self.mask.shape)

    @property
    def n_vox(self):
        return int(self.signal.shape[0])

    @property
    def n_meas(self):
        return int(self.signal.shape[1])


def _torch():
    import torch
    return torch


def _simulate(bvals, bvecs, dirs, ffib, fiso, dpar, dperp, fin, s0, device="cpu",
              chunk=16384):
    """Noiseless ground-truth signal, float64 numpy [V, N].

    dirs [V, F, 3] unit, ffib [V, F], fiso [V, 3] (csf, gm, res), dpar/dperp/fin/s0 [V].
    """
    torch = _torch()
    V = dirs.shape[0]
    b = torch.as_tensor(bvals, dtype=torch.float64, device=device)
    g = torch.as_tensor(bvecs, dtype=torch.float64, device=device)
    eiso = torch.exp(-b[None, :] * torch.tensor(D_ISO, dtype=torch.float64,
                                               device=device)[:, None])  # [3, N]
    out = np.empty((V, len(bvals)), dtype=np.float64)
    for a in range(0, V, chunk):
        e = min(V, a + chunk)
        dd = torch.as_tensor(dirs[a:e], dtype=torch.float64, device=device)
        ff = torch.as_tensor(ffib[a:e], dtype=torch.float64, device=device)
        fi = torch.as_tensor(fiso[a:e], dtype=torch.float64, device=device)
        dp = torch.as_tensor(dpar[a:e], dtype=torch.float64, device=device)[:, None, None]
        dq = torch.as_tensor(dperp[a:e], dtype=torch.float64, device=device)[:, None, None]
        fn = torch.as_tensor(fin[a:e], dtype=torch.float64, device=device)[:, None, None]
        cos = torch.einsum("vfj,nj->vfn", dd, g)
        cos2 = cos * cos
        stick = torch.exp(-b * dp * cos2)
        zep = torch.exp(-b * (dp * cos2 + dq * (1.0 - cos2)))
        fib = (ff[:, :, None] * (fn * stick + (1.0 - fn) * zep)).sum(1)
        iso = fi @ eiso
        sig = torch.as_tensor(s0[a:e], dtype=torch.float64, device=device)[:, None] * (fib + iso)
        out[a:e] = sig.cpu().numpy()
    return out


def _rician(clean, sigma, rng, chunk=1 << 22):
    """|clean + sigma (n1 + i n2)|, sigma broadcast per voxel or scalar; float32 out."""
    V, N = clean.shape
    out = np.empty((V, N), dtype=np.float32)
    sig = np.broadcast_to(np.asarray(sigma, dtype=np.float64).reshape(-1, 1), (V, 1))
    rows = max(1, chunk // N)
    for a in range(0, V, rows):
        e = min(V, a + rows)
        n1 = rng.standard_normal((e - a, N), dtype=np.float32)
        n2 = rng.standard_normal((e - a, N), dtype=np.float32)
        re = clean[a:e] + sig[a:e] * n1
        im = sig[a:e] * n2
        out[a:e] = np.sqrt(re * re + im * im).astype(np.float32)
    return out


def _unit(v):
    return v / np.linalg.norm(v, axis=-1, keepdims=True)


def _rotate_about(d1, angle, rng):
    """Unit vectors at `angle` (rad) from d1, in a uniformly random azimuth."""
    helper = np.where(np.abs(d1[:, :1]) < 0.9, np.array([[1.0, 0, 0]]), np.array([[0, 1.0, 0]]))
    u = _unit(np.cross(d1, helper))
    w = np.cross(d1, u)
    phi = rng.uniform(0, 2 * np.pi, size=(d1.shape[0], 1))
    perp = np.cos(phi) * u + np.sin(phi) * w
    a = np.asarray(angle).reshape(-1, 1)
    return _unit(np.cos(a) * d1 + np.sin(a) * perp)


def _crossing_voxels(V, angles_deg, rng):
    """Two-fiber crossing ground truth (Dirichlet(2,2,1,1,1) over fib1, fib2, csf, gm, res)."""
    d1 = _unit(rng.standard_normal((V, 3)))
    d2 = _rotate_about(d1, np.deg2rad(angles_deg), rng)
    fr = rng.dirichlet([2, 2, 1, 1, 1], size=V)
    gt = dict(
        dirs=np.stack([d1, d2], axis=1),
        ffib=fr[:, :2].copy(),
        fiso=fr[:, 2:].copy(),
        dpar=rng.uniform(1.5e-3, 2.2e-3, V),
        dperp=rng.uniform(0.2e-3, 0.8e-3, V),
        fin=rng.uniform(0.4, 0.6, V),
        s0=np.ones(V),
        angle=np.broadcast_to(np.asarray(angles_deg, dtype=np.float64), (V,)).copy(),
    )
    return gt


def _finish(mask, scheme, gt, snr, rng, device, cal=None):
    bvals, bvecs = scheme
    clean = _simulate(bvals, bvecs, gt["dirs"], gt["ffib"], gt["fiso"], gt["dpar"],
                      gt["dperp"], gt["fin"], gt["s0"], device=device)
    if cal is not None:
        clean = cal["scale"][None, :] * cal["bias"][:, None] * clean + cal["offset"][None, :]
        gt["cal"] = cal
    sigma = gt["s0"] / float(snr)
    gt["sigma"] = float(1.0 / snr)
    gt["snr"] = float(snr)
    sig = _rician(clean, sigma, rng)
    return Volume(mask=mask, signal=sig, bvals=bvals, bvecs=bvecs, gt=gt)


def crossing_patch(seed=0, edge=8, snr=30.0, device="cpu"):
    """One edge^3 patch of two-fiber crossings at angles U(20, 90) deg, 96 measurements."""
    rng = np.random.default_rng([seed, 1])
    V = edge ** 3
    gt = _crossing_voxels(V, rng.uniform(20.0, 90.0, V), rng)
    mask = np.ones((edge, edge, edge), dtype=np.uint8)
    return _finish(mask, scheme_96(seed), gt, snr, rng, device)


BENCH_ANGLES = tuple(range(15, 91, 5))      # 16 crossing angles, degrees


def crossing_benchmark(snr=30.0, seed=0, n_per_case=200, device="cpu"):
    """The crossing-fiber benchmark's layout (Sec. 3 "Datasets"): 16 crossing angles
    15, 20, ..., 90 deg and single-fiber controls, n_per_case voxels each (3400 at 200),
    N = 193 (1 b=0 + 64 directions x 1000/2000/3000), Rician noise at the given SNR.

    Each fiber is an axially symmetric tensor with eigenvalues (1.7, 0.3, 0.3) x 1e-3 mm^2/s
    (the fit model's 0.4 perpendicular diffusivity is deliberately different, Sec. 4), equal
    fractions for the two fibers of a crossing, no isotropic compartment, S0 = 1. The mask is
    [17, n_per_case, 1]: row 0 holds the single-fiber controls, row i the crossings at
    BENCH_ANGLES[i - 1]. gt["case"] is that row per voxel, gt["angle"] the crossing angle
    (0 for the controls).
    """
    rng = np.random.default_rng([seed, 7])
    n = int(n_per_case)
    cases = np.repeat(np.arange(len(BENCH_ANGLES) + 1), n)
    V = cases.shape[0]
    angles = np.concatenate([np.zeros(n)] + [np.full(n, float(a)) for a in BENCH_ANGLES])
    d1 = _unit(rng.standard_normal((V, 3)))
    d2 = _rotate_about(d1, np.deg2rad(np.maximum(angles, 1.0)), rng)
    ffib = np.where(cases[:, None] == 0, np.array([[1.0, 0.0]]), np.array([[0.5, 0.5]]))
    gt = dict(
        dirs=np.stack([d1, d2], axis=1),
        ffib=ffib,
        fiso=np.zeros((V, 3)),
        dpar=np.full(V, 1.7e-3),
        dperp=np.full(V, 0.3e-3),
        fin=np.zeros(V),
        s0=np.ones(V),
        angle=angles,
        case=cases,
    )
    mask = np.ones((len(BENCH_ANGLES) + 1, n, 1), dtype=np.uint8)
    return _finish(mask, scheme_193(seed), gt, snr, rng, device)


def crossing_sweep(seed=0, edge=10, n_angles=16, snr=30.0, device="cpu"):
    """16 crossing angles 20 + 70 i / 15 deg, one edge^3 volume (one patch) per angle."""
    vols = []
    scheme = scheme_96(seed)
    for i in range(n_angles):
        rng = np.random.default_rng([seed, 2, i])
        ang = 20.0 + 70.0 * i / (n_angles - 1)
        V = edge ** 3
        gt = _crossing_voxels(V, np.full(V, ang), rng)
        mask = np.ones((edge, edge, edge), dtype=np.uint8)
        vols.append(_finish(mask, scheme, gt, snr, rng, device))
    return vols


def _poly_bias(shape, rng, amp=0.2):
    """Smooth multiplicative bias: 1 + amp * p / max|p|, p a random cubic polynomial."""
    axes = [np.linspace(-1, 1, n) for n in shape]
    X, Y, Z = np.meshgrid(*axes, indexing="ij")
    p = np.zeros(shape)
    for i in range(4):
        for j in range(4 - i):
            for k in range(4 - i - j):
                if i + j + k == 0:
                    continue
                p += rng.standard_normal() * X ** i * Y ** j * Z ** k
    return 1.0 + amp * p / np.max(np.abs(p))


def _calibration(mask, N, rng, amp=0.2, scale_sd=0.02, offset_sd=0.01):
    bias = _poly_bias(mask.shape, rng, amp)[mask.astype(bool)]
    return dict(bias=bias, scale=rng.normal(1.0, scale_sd, N), offset=rng.normal(0.0, offset_sd, N))


def _bezier(ctrl, t):
    t = t[:, None]
    return ((1 - t) ** 3 * ctrl[0] + 3 * (1 - t) ** 2 * t * ctrl[1]
            + 3 * (1 - t) * t ** 2 * ctrl[2] + t ** 3 * ctrl[3])


def _bezier_tangent(ctrl, t):
    t = t[:, None]
    return (3 * (1 - t) ** 2 * (ctrl[1] - ctrl[0]) + 6 * (1 - t) * t * (ctrl[2] - ctrl[1])
            + 3 * t ** 2 * (ctrl[3] - ctrl[2]))


def bundle_phantom(seed=0, edge=64, n_bundles=8, snr=20.0, device="cpu", scheme=None):
    """Curved tubular bundles in a CSF/GM background, with bias and per-measurement affine.

    8 cubic-Bezier bundles of radius U(3, 6) voxels; each voxel keeps the tangents of
    the (up to 3) nearest bundles that contain it. Background: a CSF ellipsoid core,
    GM elsewhere. Bias 1 +- 20 % (cubic polynomial), scale N(1, .02), offset N(0, .01).
    """
    rng = np.random.default_rng([seed, 3])
    n = edge
    mask = np.ones((n, n, n), dtype=np.uint8)
    coords = np.stack(np.meshgrid(*([np.arange(n)] * 3), indexing="ij"), -1).reshape(-1, 3).astype(np.float64)
    V = coords.shape[0]
    ts = np.linspace(0, 1, 256)
    dist = np.full((n_bundles, V), np.inf)
    tang = np.zeros((n_bundles, V, 3))
    radius = rng.uniform(3.0, 6.0, n_bundles) * n / 64.0
    for bi in range(n_bundles):
        ctrl = rng.uniform(0.1 * n, 0.9 * n, size=(4, 3))
        # endpoints near opposite faces so bundles traverse the volume
        ax = bi % 3
        ctrl[0, ax] = 0.02 * n
        ctrl[3, ax] = 0.98 * n
        pts = _bezier(ctrl, ts)
        tg = _unit(_bezier_tangent(ctrl, ts))
        best = np.full(V, np.inf)
        bidx = np.zeros(V, dtype=np.int64)
        for c0 in range(0, len(ts), 32):
            d = np.linalg.norm(coords[:, None, :] - pts[None, c0:c0 + 32, :], axis=2)
            j = np.argmin(d, axis=1)
            dm = d[np.arange(V), j]
            upd = dm < best
            best[upd] = dm[upd]
            bidx[upd] = c0 + j[upd]
        dist[bi] = best
        tang[bi] = tg[bidx]
    inside = dist < radius[:, None]
    order = np.argsort(np.where(inside, dist, np.inf), axis=0)[:3]  # nearest 3 bundles
    nfib = np.minimum(inside.sum(0), 3)
    dirs = np.zeros((V, 3, 3))
    ffib = np.zeros((V, 3))
    for s in range(3):
        on = nfib > s
        bsel = order[s]
        dirs[:, s] = tang[bsel, np.arange(V)]
        ffib[on, s] = 0.7 / nfib[on]
    dirs[ffib == 0] = np.array([1.0, 0.0, 0.0])
    c = (n - 1) / 2.0
    core = np.sum(((coords - c) / (0.18 * n)) ** 2, axis=1) <= 1.0
    fiso = np.where(core[:, None], [[0.85, 0.10, 0.05]], [[0.10, 0.75, 0.15]])
    wm = nfib > 0
    fiso[wm] = [0.05, 0.15, 0.10]
    gt = dict(dirs=dirs, ffib=ffib, fiso=fiso, dpar=rng.uniform(1.5e-3, 2.2e-3, V),
              dperp=rng.uniform(0.2e-3, 0.8e-3, V), fin=rng.uniform(0.4, 0.6, V),
              s0=np.ones(V), nfib=nfib)
    sch = scheme if scheme is not None else scheme_360(seed)
    cal = _calibration(mask, len(sch[0]), rng)
    return _finish(mask, sch, gt, snr, rng, device, cal)


def _smooth_field(shape, sigma, rng):
    from scipy.ndimage import gaussian_filter
    f = gaussian_filter(rng.standard_normal(shape), sigma, mode="wrap")
    return (f - f.mean()) / (f.std() + 1e-12)


def _ellipsoid_mask(shape, semi):
    c = [(s - 1) / 2.0 for s in shape]
    g = np.meshgrid(*[np.arange(s, dtype=np.float64) for s in shape], indexing="ij")
    r = sum(((g[i] - c[i]) / semi[i]) ** 2 for i in range(3))
    return (r <= 1.0).astype(np.uint8)


def _tissue_from_fields(mask, rng, smooth):
    """WM fraction, 1-3 fibers with directions from smoothed vector fields, GM/CSF rest."""
    shape = mask.shape
    m = mask.astype(bool)
    w = np.clip(0.5 + 0.35 * _smooth_field(shape, smooth, rng), 0.0, 1.0)[m]
    z2 = _smooth_field(shape, smooth, rng)[m]
    nfib = np.where(w > 0.05, 1 + (z2 > 0.3) + (z2 > 1.0), 0)
    dirs = np.zeros((w.size, 3, 3))
    for s in range(3):
        vec = np.stack([_smooth_field(shape, 1.5 * smooth, rng)[m] for _ in range(3)], -1)
        dirs[:, s] = _unit(vec + 1e-9)
    share = rng.dirichlet([2.0, 2.0, 2.0], size=w.size)
    share = np.where(np.arange(3)[None, :] < nfib[:, None], share, 0.0)
    share /= np.maximum(share.sum(1, keepdims=True), 1e-12)
    ffib = w[:, None] * share
    wm_tot = ffib.sum(1)
    sc = np.clip(0.2 + 0.3 * _smooth_field(shape, smooth, rng), 0.0, 1.0)[m]
    rest = 1.0 - wm_tot
    fiso = np.stack([rest * 0.9 * sc, rest * 0.9 * (1 - sc), rest * 0.1], -1)
    V = w.size
    return dict(dirs=dirs, ffib=ffib, fiso=fiso, dpar=rng.uniform(1.5e-3, 2.2e-3, V),
                dperp=rng.uniform(0.2e-3, 0.8e-3, V), fin=rng.uniform(0.4, 0.6, V),
                s0=np.ones(V), nfib=nfib)


def brain_phantom(seed=0, shape=(145, 174, 145), semi=(52.8, 63.4, 52.8), snr=30.0,
                  device="cpu", scheme=None):
    """HCP-shaped whole brain: ellipsoid mask (~741k voxels), tissue from smoothed fields."""
    rng = np.random.default_rng([seed, 4])
    mask = _ellipsoid_mask(shape, semi)
    gt = _tissue_from_fields(mask, rng, smooth=4.0 * shape[0] / 145.0)
    sch = scheme if scheme is not None else scheme_288(seed)
    return _finish(mask, sch, gt, snr, rng, device)


def multi_volume_batch(seed=0, edges=(32, 40, 48, 56, 64, 72, 80, 88, 96, 104, 112, 128),
                       device="cpu"):
    """Uneven batch of cubic volumes with inscribed ellipsoid masks and mixed schemes.

    Schemes cycle 96/288/360 measurements; SNR ~ U{10..40} per volume; every volume
    carries a bias field and a per-measurement affine perturbation.
    """
    schemes = [scheme_96(seed), scheme_288(seed), scheme_360(seed)]
    vols = []
    for i, e in enumerate(edges):
        rng = np.random.default_rng([seed, 5, i])
        mask = _ellipsoid_mask((e, e, e), (e / 2.0 - 0.5,) * 3)
        gt = _tissue_from_fields(mask, rng, smooth=max(1.5, e / 32.0))
        snr = float(rng.integers(10, 41))
        sch = schemes[i % 3]
        cal = _calibration(mask, len(sch[0]), rng)
        vols.append(_finish(mask, sch, gt, snr, rng, device, cal))
    return vols


def random_volume(shape=(4, 4, 4), scheme=None, seed=0, mask_density=1.0, snr=30.0,
                  calibration=False, device="cpu"):
    """Small generic volume for tests: random crossings, optional sparse mask."""
    rng = np.random.default_rng([seed, 6])
    mask = (rng.uniform(size=shape) < mask_density).astype(np.uint8)
    if mask.sum() == 0:
        mask.flat[0] = 1
    V = int(mask.sum())
    gt = _crossing_voxels(V, rng.uniform(20.0, 90.0, V), rng)
    sch = scheme if scheme is not None else scheme_96(seed)
    cal = _calibration(mask, len(sch[0]), rng) if calibration else None
    return _finish(mask, sch, gt, snr, rng, device, cal)


def default_init(V, K, seed=0):
    """Seeded raw initial parameters [V, 4K+5] (float32), shared by oracle and GPU.

    S0 raw = softplus^-1(1) = log(e - 1); fraction logits 0 (equal fractions);
    directions uniform on the sphere (normalised Gaussians); f_intra raw 0, i.e.
    sigmoid(0) = 0.5 as the paper initialises it (Sec. 2.2).
    """
    rng = np.random.default_rng([seed, 7])
    Q = n_params(K)
    th = np.zeros((V, Q), dtype=np.float64)
    th[:, 0] = np.log(np.e - 1.0)
    d = rng.standard_normal((V, K, 3))
    d /= np.linalg.norm(d, axis=2, keepdims=True)
    th[:, K + 4:4 * K + 4] = d.reshape(V, 3 * K)
    return th.astype(np.float32)
