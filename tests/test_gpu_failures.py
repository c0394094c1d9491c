"""Run-time failure paths on the GPU, made without a fault: the host injects the failure.

- A NaN written into the parameters (prism_set_params) makes the next iteration's objective
  non-finite; the kernels record it in the handle's status word and prism_sync returns
  PRISM_E_NONFINITE (fused and plain paths, MSE and calibrated NLL).
- A bounded device wait that runs out (prism_wait_probe: a barrier phase that nothing
  completes, no copy in flight) sets the timeout status; prism_sync returns PRISM_E_TIMEOUT,
  and the CUDA context stays usable for other handles.
"""
import numpy as np
import pytest

import phantoms as P
from tests.helpers import gpu_volume, inits_for

pytestmark = pytest.mark.gpu

E_INVALID_ARG, E_NONFINITE, E_TIMEOUT = 1, 5, 6


def _fitter(loss="mse", cal=False, fused=1, seed=0):
    import paper_2604_00250_gb300 as prism
    vol = P.random_volume((6, 5, 4), seed=seed, mask_density=0.8, calibration=cal)
    init = inits_for([vol], 3, seed)[0]
    return prism.Fitter([gpu_volume(vol, init)], prism.options(K=3, loss=loss, calibration=cal, patch_dim=4,
                                                                fused=fused, use_graph=fused)), init


@pytest.mark.parametrize("fused", [1, 0])
@pytest.mark.parametrize("loss,cal", [("mse", False), ("nll", True)])
def test_nan_parameter_is_reported_as_nonfinite(fused, loss, cal):
    import paper_2604_00250_gb300 as prism
    f, init = _fitter(loss, cal, fused)
    f.step(2)
    f.sync()                                   # healthy so far
    th = init.copy()
    th[5, 2] = np.nan
    f.set_params(th)
    f.step(1)
    with pytest.raises(prism.PrismError) as e:
        f.sync()
    assert e.value.code == E_NONFINITE
    f.close()


def test_wait_that_runs_out_is_reported_as_timeout():
    import paper_2604_00250_gb300 as prism
    f, _ = _fitter()
    f.step(1)
    f.sync()
    with pytest.raises(prism.PrismError) as e:
        f.wait_probe(0)
    assert e.value.code == E_INVALID_ARG
    f.wait_probe(1000)
    with pytest.raises(prism.PrismError) as e:
        f.sync()
    assert e.value.code == E_TIMEOUT
    with pytest.raises(prism.PrismError) as e:
        f.sync()                               # the status stays set on this handle
    assert e.value.code == E_TIMEOUT
    f.close()
    g, _ = _fitter(seed=1)                    # the context is still usable
    g.step(3)
    g.sync()
    assert np.isfinite(g.loss_history()).all()
    g.close()
