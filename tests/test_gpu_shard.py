"""One volume's patches split across two handles on one GPU, as two ranks would fit them.

Without calibration and with the MSE, patches are independent problems (neighbour priors stay
inside a patch, Sec. 2.4) coupled only through the normaliser |M| of Eq. 8. A part = the
volume's mask restricted to some whole patches, its signal rows, and norm_count = the whole
volume's |M|. The merged parameters of the parts after several iterations must equal the
whole-volume fit bitwise (fused kernel with one and four lanes per voxel, and the plain path),
starting from the library's default start (drawn per grid position), and the parts' objectives
must add up to the whole volume's.
"""
import types

import numpy as np
import pytest
import torch

import phantoms as P
from paper_2604_00250_gb300 import shard

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("fused,tpv", [(1, 1), (1, 4), (0, 1)])
def test_patch_shards_merge_to_the_whole_fit(fused, tpv):
    import paper_2604_00250_gb300 as prism
    vol = P.bundle_phantom(2, edge=24, device="cpu")
    K, PD, iters = 3, 8, 6
    kw = dict(K=K, loss="mse", patch_dim=PD, lam_sp=0.01, lam_dir=0.005, fused=fused, use_graph=fused,
              threads_per_voxel=tpv)
    whole = types.SimpleNamespace(mask=vol.mask, signal=torch.as_tensor(vol.signal).cuda(), bvals=vol.bvals,
                                  bvecs=vol.bvecs, init=None)
    f = prism.Fitter([whole], prism.options(**kw))
    th_start = f.params_host()
    f.step(iters)
    f.sync()
    ref = f.params_host()
    ref_hist = f.loss_history()[:, 0]
    f.close()
    merged = np.full_like(ref, np.nan)
    hist = np.zeros_like(ref_hist)
    for rank in range(2):
        part, sel = shard.shard_volume(whole, PD, rank, 2)
        assert 0 < sel.size < vol.n_vox
        g = prism.Fitter([part], prism.options(**kw))
        assert np.array_equal(g.params_host(), th_start[sel])   # the same default start
        g.step(iters)
        g.sync()
        merged[sel] = g.params_host()
        hist += g.loss_history()[:, 0]
        g.close()
    assert np.array_equal(merged, ref), float(np.nanmax(np.abs(merged - ref)))
    np.testing.assert_allclose(hist, ref_hist, rtol=1e-6)
