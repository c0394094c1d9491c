"""C-ABI checks that need no GPU: the library builds and loads, exports every symbol
include/prism.h declares, its structs have the header's layout, and argument
validation fails before any device work."""
import ctypes
import json
import os
import re
import shutil
import subprocess
import types

import numpy as np
import pytest

import phantoms as P

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "prism.h")


@pytest.fixture(scope="module")
def prism():
    from paper_2604_00250_gb300 import build
    if shutil.which("nvcc") or os.path.exists("/usr/local/cuda/bin/nvcc"):
        build.build()
    import paper_2604_00250_gb300 as p
    p._lib.load()
    return p


def _declared():
    txt = open(HEADER).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(prism_[a-z_]+)\s*\(", txt)))


def test_exports_every_declared_symbol(prism):
    lib = ctypes.CDLL(prism.library_path())
    names = _declared()
    assert len(names) >= 19
    for n in names:
        assert hasattr(lib, n), n
    assert set(names) == set(prism._lib.EXPORTS)


def test_struct_layout_matches_header(prism, tmp_path):
    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("gcc missing")
    src = tmp_path / "layout.c"
    src.write_text(
        '#include <stdio.h>\n#include <stddef.h>\n#include "prism.h"\n'
        "int main(void){\n"
        'printf("%zu %zu %zu %zu %zu %zu %zu %zu\\n", sizeof(prism_volume), sizeof(prism_options),'
        " offsetof(prism_volume, signal), offsetof(prism_volume, init), offsetof(prism_options, lr),"
        " offsetof(prism_options, fused), offsetof(prism_options, seed), offsetof(prism_options, tv_eps));\n"
        "return 0;}\n")
    exe = tmp_path / "layout"
    subprocess.run([gcc, "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = [int(x) for x in subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split()]
    L = prism._lib
    want = [ctypes.sizeof(L.Volume), ctypes.sizeof(L.Options), L.Volume.signal.offset, L.Volume.init.offset,
            L.Options.lr.offset, L.Options.fused.offset, L.Options.seed.offset, L.Options.tv_eps.offset]
    assert got == want


def test_default_options_are_the_papers(prism):
    gold = json.load(open(os.path.join(ROOT, "tests", "golden", "paper_constants.json")))
    o = prism.options()
    assert o.K == 3 and o.loss == 0
    f32 = lambda x: float(np.float32(x))  # options are float32 in the C struct
    assert o.lam_rep == f32(gold["lambda_rep"]["value"])
    assert o.lam_sparse == f32(gold["lambda_sparse"]["value"])
    assert o.tau == f32(gold["tau"]["value"])
    assert o.huber_delta == f32(gold["huber_delta"]["value"])
    assert o.lr == f32(gold["adam_lr"]["value"])


def _vol(mask, bvals=None, bvecs=None):
    N = 4 if bvals is None else len(bvals)
    bvals = np.array([0, 1000, 1000, 2000], np.float32) if bvals is None else np.asarray(bvals, np.float32)
    bvecs = (np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1]], np.float32) if bvecs is None
             else np.asarray(bvecs, np.float32))
    V = int(mask.sum())
    return types.SimpleNamespace(mask=mask, signal=np.ones((V, N), np.float32), bvals=bvals, bvecs=bvecs, init=None)


@pytest.mark.parametrize("case,code", [
    ("k_out_of_range", 1), ("empty_mask", 2), ("no_b0", 2), ("non_unit_bvec", 1), ("negative_b", 1),
    ("bad_patch", 1), ("bad_tpv", 1), ("negative_lambda", 1), ("norm_count_below_mask", 2),
])
def test_validation_errors(prism, case, code):
    m = np.ones((2, 2, 2), np.uint8)
    kw = {}
    vol = _vol(m)
    if case == "k_out_of_range":
        kw = dict(K=7)
    elif case == "empty_mask":
        vol = _vol(np.zeros((2, 2, 2), np.uint8))
    elif case == "no_b0":
        vol = _vol(m, bvals=[500, 1000, 1000, 2000], bvecs=[[1, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1]])
    elif case == "non_unit_bvec":
        vol = _vol(m, bvecs=[[0, 0, 0], [2, 0, 0], [0, 1, 0], [0, 0, 1]])
    elif case == "negative_b":
        vol = _vol(m, bvals=[0, -5, 1000, 2000])
    elif case == "bad_patch":
        kw = dict(patch_dim=0)
    elif case == "bad_tpv":
        kw = dict(threads_per_voxel=3)
    elif case == "negative_lambda":
        kw = dict(lam_rep=-1.0)
    elif case == "norm_count_below_mask":
        vol.norm_count = 7               # the mask holds 8 voxels
    with pytest.raises(prism.PrismError) as e:
        prism.Fitter([vol], prism.options(**kw))
    assert e.value.code == code
    assert prism._lib.load().prism_last_error()


def test_null_arguments(prism):
    lib = prism._lib.load()
    h = ctypes.c_void_p()
    assert lib.prism_fit_init(None, 1, None, None, ctypes.byref(h)) == 1
    assert lib.prism_step(None, 1, None) == 1
    assert lib.prism_backward(None, None, None, None) == 1
    lib.prism_fit_destroy(None)


def test_missing_library_fails_loudly(monkeypatch, tmp_path):
    import paper_2604_00250_gb300._lib as L
    monkeypatch.setattr(L, "_lib", None)
    monkeypatch.setattr(L, "LIB_PATH", str(tmp_path / "absent.so"))
    with pytest.raises(ImportError):
        L.load()


@pytest.mark.parametrize("slab,overlap,code", [(0, 0, 1), (10, -1, 1), (10, 6, 1)])
def test_slab_driver_validation(prism, slab, overlap, code):
    """prism_fit_init_slabs rejects a slab of no slices, a negative overlap and an overlap
    above half a slab before any device work."""
    vol = _vol(np.ones((2, 2, 12), np.uint8))
    with pytest.raises(prism.PrismError) as e:
        prism.Fitter(vol, prism.options(), slabs=(slab, overlap))
    assert e.value.code == code


def test_slab_driver_empty_mask(prism):
    vol = _vol(np.zeros((2, 2, 12), np.uint8))
    with pytest.raises(prism.PrismError) as e:
        prism.Fitter(vol, prism.options(), slabs=(6, 2))
    assert e.value.code == 2


def test_readout_entry_points_reject_null_handles(prism):
    lib = prism._lib.load()
    assert lib.prism_get_fibers(None, None, None, None, ctypes.c_float(0.15), 0, None) == 1
    assert lib.prism_stitch_slabs(None, None, None, None, None, 0, None) == 1
    assert lib.prism_get_shape(None, None, None, None, None) == 1


def test_host_plan_runs_on_a_machine_without_a_gpu(prism):
    """Without a GPU, prism_fit_init still builds the whole host plan (voxel counts, patches,
    tiles, slot tables) for a batch of unlike volumes, and then reports the first failing CUDA
    call as PRISM_E_CUDA instead of crashing."""
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present: the handle would be created")
    rng = np.random.default_rng(5)
    vols = [_vol((rng.random(shape) < dens).astype(np.uint8)) for shape, dens in
            (((37, 23, 41), 0.6), ((8, 8, 8), 1.0), ((1, 1, 1), 1.0), ((50, 3, 17), 0.3))]
    for kw in (dict(patch_dim=16), dict(patch_dim=4, threads_per_voxel=4, calibration=1)):
        with pytest.raises(prism.PrismError) as e:
            prism.Fitter(vols, prism.options(**kw))
        assert e.value.code == 3
