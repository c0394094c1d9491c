"""GB300 (sm_103a) implementation of the PRISM analysis-by-synthesis fit.

Python binding of the C-ABI library (include/prism.h). Every step of the fit runs
in the library's CUDA kernels; this module only marshals arguments. PyTorch
provides device memory and streams.

    import paper_2604_00250_gb300 as prism
    f = prism.Fitter(volumes, prism.options(K=3, loss="mse"))
    f.step(200)
    theta = f.params()           # [V, 4K+5] raw parameters, mask order

`volumes` are objects with `mask` (uint8 [nx, ny, nz]), `signal` ([V, N] float32,
numpy for host memory or a CUDA tensor), `bvals` [N] and `bvecs` [N, 3].
"""
import ctypes

import numpy as np

from . import _lib
from ._lib import PrismError, MEM_HOST, MEM_DEVICE, LOSS_MSE, LOSS_NLL

__all__ = ["options", "Fitter", "fit", "PrismLoss", "PrismError", "library_path"]


def library_path():
    return _lib.LIB_PATH


def _torch():
    import torch
    return torch


def options(**kw):
    """prism_options with the paper's defaults, overridden by keyword (loss="mse"|"nll",
    optimizer="adam"|"rprop")."""
    lib = _lib.load()
    o = _lib.Options()
    lib.prism_default_options(ctypes.byref(o))
    for k, v in kw.items():
        if k == "loss" and isinstance(v, str):
            v = {"mse": LOSS_MSE, "nll": LOSS_NLL}[v.lower()]
        if k == "optimizer" and isinstance(v, str):
            v = {"adam": _lib.OPT_ADAM, "rprop": _lib.OPT_RPROP}[v.lower()]
        if isinstance(v, bool):
            v = int(v)
        if not hasattr(o, k):
            raise TypeError(f"unknown option {k!r}")
        setattr(o, k, v)
    return o


def _stream_ptr(stream):
    torch = _torch()
    if stream is None:
        if torch.cuda.is_available():
            return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
        return ctypes.c_void_p(0)
    if isinstance(stream, int):
        return ctypes.c_void_p(stream)
    return ctypes.c_void_p(stream.cuda_stream)


def _host_f32(a, shape=None):
    a = np.ascontiguousarray(np.asarray(a, dtype=np.float32))
    if shape is not None and a.shape != tuple(shape):
        raise ValueError(f"expected shape {shape}, got {a.shape}")
    return a


def _volume_struct(vol, keep):
    torch = _torch()
    mask = np.ascontiguousarray(np.asarray(vol.mask).astype(np.uint8))
    if mask.ndim != 3:
        raise ValueError("mask must be 3-D")
    bvals = _host_f32(vol.bvals)
    N = int(bvals.shape[0])
    bvecs = _host_f32(vol.bvecs, (N, 3))
    sig = vol.signal
    init = getattr(vol, "init", None)
    V = int(mask.astype(bool).sum())
    if isinstance(sig, torch.Tensor) and sig.is_cuda:
        mem = MEM_DEVICE
        sig = sig.detach().to(torch.float32).contiguous()
        if tuple(sig.shape) != (V, N):
            raise ValueError(f"signal must be [V={V}, N={N}], got {tuple(sig.shape)}")
        sp = sig.data_ptr()
        ip = None
        if init is not None:
            init = torch.as_tensor(init, device=sig.device, dtype=torch.float32).contiguous()
            ip = init.data_ptr()
    else:
        mem = MEM_HOST
        if isinstance(sig, torch.Tensor):
            sig = sig.detach().cpu().numpy()
        sig = _host_f32(sig, (V, N))
        sp = sig.ctypes.data
        ip = None
        if init is not None:
            if isinstance(init, torch.Tensor):
                init = init.detach().cpu().numpy()
            init = _host_f32(init)
            ip = init.ctypes.data
    keep.extend([mask, bvals, bvecs, sig, init])
    nx, ny, nz = mask.shape
    norm = int(getattr(vol, "norm_count", 0) or 0)
    return _lib.Volume(nx, ny, nz, N, mem, norm, mask.ctypes.data, sp, bvals.ctypes.data, bvecs.ctypes.data, ip)


def _volumes_array(volumes, keep):
    if not isinstance(volumes, (list, tuple)):
        volumes = [volumes]
    arr = (_lib.Volume * len(volumes))()
    for i, v in enumerate(volumes):
        arr[i] = _volume_struct(v, keep)
    return arr, len(volumes)


class Fitter:
    """One PRISM fit (a handle of the C library) over a batch of volumes."""

    def __init__(self, volumes, opts=None, stream=None, slabs=None, **kw):
        """`slabs=(slab, overlap)` fits one whole volume as overlapping slabs along its last
        axis (prism_fit_init_slabs); `stitch()` then returns the whole-volume maps."""
        lib = _lib.load()
        self._lib = lib
        self.opts = opts if opts is not None else options(**kw)
        keep = []
        h = ctypes.c_void_p()
        if slabs is not None:
            vol = volumes[0] if isinstance(volumes, (list, tuple)) else volumes
            vs = _volume_struct(vol, keep)
            _lib.check(lib.prism_fit_init_slabs(ctypes.byref(vs), int(slabs[0]), int(slabs[1]),
                                                ctypes.byref(self.opts), _stream_ptr(stream), ctypes.byref(h)))
        else:
            arr, n = _volumes_array(volumes, keep)
            _lib.check(lib.prism_fit_init(arr, n, ctypes.byref(self.opts), _stream_ptr(stream), ctypes.byref(h)))
        self._h = h
        self._fwd_token = None      # identifies the handle's last prism_forward (PrismLoss)
        V, G, Q, GP, it = (ctypes.c_int64(), ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int64(),
                           ctypes.c_int64())
        _lib.check(lib.prism_info(h, ctypes.byref(V), ctypes.byref(G), ctypes.byref(Q), ctypes.byref(GP),
                                  ctypes.byref(it)))
        self.n_vox, self.n_groups, self.Q, self.n_group_params = V.value, G.value, Q.value, GP.value
        self.K = int(self.opts.K)
        vols = volumes if isinstance(volumes, (list, tuple)) else [volumes]
        if slabs is not None:
            N = int(np.asarray(vols[0].bvals).shape[0])
            self.n_meas = [N] * self.n_groups
            self.yhat_len = self.n_vox * N
            self.n_out = int(np.asarray(vols[0].mask).astype(bool).sum())
        else:
            self.n_meas = [int(np.asarray(v.bvals).shape[0]) for v in vols]
            self.yhat_len = sum(int(np.asarray(v.mask).astype(bool).sum()) * n for v, n in zip(vols, self.n_meas))

    # -- lifecycle -----------------------------------------------------------
    def close(self):
        if getattr(self, "_h", None):
            self._lib.prism_fit_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    # -- iterations ------------------------------------------------------------
    def step(self, n=1, stream=None):
        self._fwd_token = None
        _lib.check(self._lib.prism_step(self._h, int(n), _stream_ptr(stream)))

    def sync(self, stream=None):
        _lib.check(self._lib.prism_sync(self._h, _stream_ptr(stream)))

    def wait_probe(self, max_polls=1000, stream=None):
        """Runs the library's check of its bounded device waits (prism_wait_probe): the next
        sync() raises PrismError E_TIMEOUT, as every later one on this Fitter does."""
        _lib.check(self._lib.prism_wait_probe(self._h, int(max_polls), _stream_ptr(stream)))

    @property
    def iterations(self):
        it = ctypes.c_int64()
        _lib.check(self._lib.prism_info(self._h, None, None, None, None, ctypes.byref(it)))
        return it.value

    # -- parameters --------------------------------------------------------------
    def params(self, stream=None):
        torch = _torch()
        out = torch.empty((self.n_vox, self.Q), dtype=torch.float32, device="cuda")
        _lib.check(self._lib.prism_get_params(self._h, ctypes.c_void_p(out.data_ptr()), MEM_DEVICE,
                                              _stream_ptr(stream)))
        return out

    def params_host(self):
        out = np.empty((self.n_vox, self.Q), dtype=np.float32)
        _lib.check(self._lib.prism_get_params(self._h, out.ctypes.data, MEM_HOST, _stream_ptr(None)))
        return out

    def set_params(self, theta, stream=None):
        torch = _torch()
        t = torch.as_tensor(theta, dtype=torch.float32, device="cuda").contiguous()
        if tuple(t.shape) != (self.n_vox, self.Q):
            raise ValueError("theta must be [V, Q]")
        self._fwd_token = None
        _lib.check(self._lib.prism_set_params(self._h, ctypes.c_void_p(t.data_ptr()), MEM_DEVICE,
                                              _stream_ptr(stream)))
        torch.cuda.current_stream().synchronize()

    def stitch(self, out=None):
        """Whole-volume maps of a slab fit: (S0 [V], fractions [V, K+3], f_intra [V],
        unit directions [V, K, 3]) in the volume's mask order, float32. By default new numpy
        arrays; `out` = four arrays of those shapes to write into instead (numpy arrays, or torch
        tensors all on the host or all on the GPU, C-contiguous float32), for example pinned host
        tensors kept across fits, which spares the first touch of fresh host pages."""
        V, K = self.n_out, self.K
        shapes = ((V,), (V, K + 3), (V,), (V, K, 3))
        if out is None:
            out = tuple(np.empty(s, np.float32) for s in shapes)
        ptrs, mem = _out_pointers(out, shapes)
        _lib.check(self._lib.prism_stitch_slabs(self._h, *ptrs, mem, _stream_ptr(None)))
        return tuple(out)

    def fibers(self, rel_thresh=0.15):
        """(unit directions [V, K, 3], fractions [V, K+3], peak flags [V, K]) as numpy arrays."""
        d = np.empty((self.n_vox, self.K, 3), dtype=np.float32)
        f = np.empty((self.n_vox, self.K + 3), dtype=np.float32)
        p = np.empty((self.n_vox, self.K), dtype=np.uint8)
        _lib.check(self._lib.prism_get_fibers(self._h, d.ctypes.data, f.ctypes.data, p.ctypes.data,
                                              float(rel_thresh), MEM_HOST, _stream_ptr(None)))
        return d, f, p.astype(bool)

    def groups_device(self, stream=None):
        """Packed group parameters as a CUDA float32 tensor (a copy)."""
        torch = _torch()
        out = torch.empty(self.n_group_params, dtype=torch.float32, device="cuda")
        _lib.check(self._lib.prism_get_groups(self._h, ctypes.c_void_p(out.data_ptr()), MEM_DEVICE,
                                              _stream_ptr(stream)))
        return out

    def group_layout(self):
        off = np.zeros(4 * self.n_groups + 1, dtype=np.int64)
        _lib.check(self._lib.prism_group_layout(self._h, off.ctypes.data))
        return off

    def groups(self):
        out = np.empty(self.n_group_params, dtype=np.float32)
        _lib.check(self._lib.prism_get_groups(self._h, out.ctypes.data, MEM_HOST, _stream_ptr(None)))
        return out

    def set_groups(self, packed):
        a = _host_f32(packed, (self.n_group_params,))
        self._fwd_token = None
        _lib.check(self._lib.prism_set_groups(self._h, a.ctypes.data, MEM_HOST, _stream_ptr(None)))

    def group_view(self, packed=None):
        """Per group: sigma_log, alpha [N], beta [N], b_lr [8, 8, 8] from the packed array."""
        p = self.groups() if packed is None else np.asarray(packed)
        off = self.group_layout()
        out = []
        for g in range(self.n_groups):
            a, b, c, d = (int(x) for x in off[4 * g:4 * g + 4])
            N = self.n_meas[g]
            out.append(dict(sigma_log=float(p[a]), alpha=p[b:b + N], beta=p[c:c + N],
                            blr=p[d:d + 512].reshape(8, 8, 8)))
        return out

    # -- objective -----------------------------------------------------------------
    def loss(self):
        out = np.empty(self.n_groups, dtype=np.float64)
        _lib.check(self._lib.prism_get_loss(self._h, out.ctypes.data, None, 0, None))
        return out

    def loss_history(self, max_iters=4096):
        out = np.empty((max_iters, self.n_groups), dtype=np.float64)
        n = ctypes.c_int32()
        _lib.check(self._lib.prism_get_loss(self._h, None, out.ctypes.data, max_iters, ctypes.byref(n)))
        return out[:n.value]

    def forward(self, theta=None, groups=None, want_yhat=False, stream=None):
        """J per group (CUDA float64 [G]) and optionally y_hat (flat, volume-major rows).

        A given `theta` ([V, Q] CUDA) or `groups` (packed, CUDA) becomes the handle's current
        parameters, as with set_params / set_groups; None keeps the current ones."""
        torch = _torch()
        loss = torch.empty(self.n_groups, dtype=torch.float64, device="cuda")
        tp = gp = None
        if theta is not None:
            theta = theta.detach().to(torch.float32).contiguous()
            if not theta.is_cuda or tuple(theta.shape) != (self.n_vox, self.Q):
                raise ValueError(f"theta must be a CUDA tensor [V={self.n_vox}, Q={self.Q}]")
            tp = ctypes.c_void_p(theta.data_ptr())
        if groups is not None:
            groups = groups.detach().to(torch.float32).contiguous()
            if not groups.is_cuda or tuple(groups.shape) != (self.n_group_params,):
                raise ValueError(f"groups must be a CUDA tensor [{self.n_group_params}]")
            gp = ctypes.c_void_p(groups.data_ptr())
        yhat = None
        yp = None
        if want_yhat:
            yhat = torch.empty(self.yhat_len, dtype=torch.float32, device="cuda")
            yp = ctypes.c_void_p(yhat.data_ptr())
        self._fwd_token = None
        _lib.check(self._lib.prism_forward(self._h, tp, gp, yp, ctypes.c_void_p(loss.data_ptr()),
                                           _stream_ptr(stream)))
        self._fwd_token = object()
        return loss, yhat

    def backward(self, stream=None):
        torch = _torch()
        gth = torch.empty((self.n_vox, self.Q), dtype=torch.float32, device="cuda")
        gg = torch.empty(self.n_group_params, dtype=torch.float32, device="cuda")
        _lib.check(self._lib.prism_backward(self._h, ctypes.c_void_p(gth.data_ptr()),
                                            ctypes.c_void_p(gg.data_ptr()), _stream_ptr(stream)))
        return gth, gg

    def shape(self):
        """Launch shape: lanes per voxel, voxels per tile, CTAs of the fused kernel, shell loop."""
        tpv, tv, grid, sh = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
        _lib.check(self._lib.prism_get_shape(self._h, ctypes.byref(tpv), ctypes.byref(tv), ctypes.byref(grid),
                                             ctypes.byref(sh)))
        return dict(threads_per_voxel=tpv.value, tile_voxels=tv.value, fused_grid=grid.value, shell_loop=sh.value)

    def profile(self, n_iters=10, stream=None):
        """Average ms per iteration: fused kernel, prior preparation, group kernels, total."""
        ms = (ctypes.c_float * 4)()
        self._fwd_token = None
        _lib.check(self._lib.prism_profile(self._h, int(n_iters), _stream_ptr(stream), ms))
        return dict(fused_ms=ms[0], prep_ms=ms[1], group_ms=ms[2], iter_ms=ms[3])

    # -- checkpoint ------------------------------------------------------------------
    def state(self):
        n = ctypes.c_int64()
        _lib.check(self._lib.prism_state_size(self._h, ctypes.byref(n)))
        buf = ctypes.create_string_buffer(n.value)
        _lib.check(self._lib.prism_get_state(self._h, buf, n.value, _stream_ptr(None)))
        return buf.raw

    def load_state(self, blob):
        buf = ctypes.create_string_buffer(blob, len(blob))
        self._fwd_token = None
        _lib.check(self._lib.prism_set_state(self._h, buf, len(blob), _stream_ptr(None)))


def fit(volumes, opts=None, n_iters=200, stream=None, **kw):
    """One-call fit (prism_fit): returns (theta [V, Q] numpy float32, J per group numpy float64)."""
    lib = _lib.load()
    o = opts if opts is not None else options(**kw)
    keep = []
    arr, n = _volumes_array(volumes, keep)
    V = sum(int(np.asarray(v.mask).astype(bool).sum()) for v in (volumes if isinstance(volumes, (list, tuple)) else [volumes]))
    theta = np.empty((V, 4 * int(o.K) + 5), dtype=np.float32)
    loss = np.empty(n, dtype=np.float64)
    _lib.check(lib.prism_fit(arr, n, ctypes.byref(o), int(n_iters), theta.ctypes.data, loss.ctypes.data, MEM_HOST,
                             _stream_ptr(stream)))
    return theta, loss


def _out_pointers(arrays, shapes):
    """Data pointers and memory space (MEM_HOST / MEM_DEVICE) of caller-provided output arrays,
    each checked against its shape: numpy arrays, or torch tensors all on the host or all on the
    GPU; C-contiguous float32."""
    if len(arrays) != len(shapes):
        raise ValueError(f"expected {len(shapes)} output arrays, got {len(arrays)}")
    ptrs, spaces = [], set()
    for a, shp in zip(arrays, shapes):
        if isinstance(a, np.ndarray):
            if a.dtype != np.float32 or not a.flags.c_contiguous or a.shape != tuple(shp):
                raise ValueError(f"output array must be C-contiguous float32 of shape {tuple(shp)}")
            ptrs.append(ctypes.c_void_p(a.ctypes.data))
            spaces.add(MEM_HOST)
        else:
            torch = _torch()
            if (not isinstance(a, torch.Tensor) or a.dtype != torch.float32 or not a.is_contiguous()
                    or tuple(a.shape) != tuple(shp)):
                raise ValueError(f"output tensor must be contiguous float32 of shape {tuple(shp)}")
            ptrs.append(ctypes.c_void_p(a.data_ptr()))
            spaces.add(MEM_DEVICE if a.is_cuda else MEM_HOST)
    if len(spaces) != 1:
        raise ValueError("output arrays must all be on the host or all on the GPU")
    return ptrs, spaces.pop()


def microbench(kind):
    """Measured arithmetic rate of one pipe: "ffma", "ffma2" (flops/s), "ex2" (2^x per s), "dfma"."""
    k = {"ffma": 0, "ffma2": 1, "ex2": 2, "dfma": 3}[kind]
    r = ctypes.c_double()
    _lib.check(_lib.load().prism_microbench(k, ctypes.byref(r), _stream_ptr(None)))
    return r.value


def _make_autograd():
    torch = _torch()

    class PrismLoss(torch.autograd.Function):
        """J(theta, groups) = sum_g J_g as a differentiable function of the raw voxel parameters
        theta ([V, Q] CUDA) and the packed group parameters (CUDA, or None for the handle's
        current ones, which then get no gradient). Forward: prism_forward (synthesis,
        calibration, data term, priors). Backward: prism_backward, the hand-written adjoint,
        which recomputes the compartment exponentials instead of storing them (Sec. 2.1: every
        component is differentiable, so tissue and calibration parameters can be updated
        jointly). Each node keeps its own evaluation point; when the handle has evaluated
        another point since (a second node on the same Fitter, a step), backward first repeats
        the forward at this node's point. The handle's current parameters are those of the
        last evaluation."""

        @staticmethod
        def forward(ctx, theta, groups, fitter):
            th = theta.detach().to(torch.float32).contiguous()
            gp = groups.detach().to(torch.float32).contiguous() if groups is not None else fitter.groups_device()
            loss, _ = fitter.forward(th, gp)
            ctx.fitter = fitter
            ctx.token = fitter._fwd_token
            ctx.point = (th, gp)
            ctx.dtypes = (theta.dtype, groups.dtype if groups is not None else None)
            return loss.sum()

        @staticmethod
        def backward(ctx, gout):
            f = ctx.fitter
            if f._fwd_token is None or f._fwd_token is not ctx.token:
                f.forward(*ctx.point)
                ctx.token = f._fwd_token
            gth, gg = f.backward()
            s = gout.to(torch.float32)
            g_theta = (gth * s).to(ctx.dtypes[0]) if ctx.needs_input_grad[0] else None
            g_groups = (gg * s).to(ctx.dtypes[1]) if ctx.needs_input_grad[1] else None
            return g_theta, g_groups, None

    return PrismLoss


class _LazyAutograd:
    _cls = None

    def __getattr__(self, name):
        if _LazyAutograd._cls is None:
            _LazyAutograd._cls = _make_autograd()
        return getattr(_LazyAutograd._cls, name)


PrismLoss = _LazyAutograd()
