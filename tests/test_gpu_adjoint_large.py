"""The GPU adjoint at the gradient workload's size: 200 x 200 weld of 10 x 10 grains, 32 sources x 32
receivers, 4 media samples, FP32 and FP64, against the oracle's adjoint gradient element by element.

The observed times are the oracle's FP64 receiver times of a seeded ground-truth medium plus 10 ns noise,
as in the workload; the oracle runs on the host cores, one thread per (sample) job."""
from concurrent.futures import ThreadPoolExecutor

import numpy as np
import pytest

from paper_2302_10988_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def case(oracle):
    wl, truth = W.weld_adjoint(nsamples=4)
    _, _, t_true = oracle.misfit_and_gradient(truth, 0, truth.samples[0].region_theta, np.zeros((32, 32)))
    t_obs = t_true + W.observation_noise(t_true.shape)
    with ThreadPoolExecutor(max_workers=4) as ex:
        ref = list(ex.map(lambda b: oracle.misfit_and_gradient(wl, b, wl.samples[b].region_theta, t_obs)[1],
                          range(4)))
    return wl, t_obs, np.array(ref)


# element-wise bound over the components that are not tiny (>= 1e-2 of the largest), and a bound on the
# largest error relative to the largest component (the workload's "oracle gradient <= 1e-3 relative")
@pytest.mark.parametrize("precision,tol,tol_norm", [("fp64", 1e-5, 1e-6), ("fp32", 5e-3, 1e-3)])
def test_backward_gradient_workload_size(case, precision, tol, tol_norm):
    from paper_2302_10988_gb300 import api, build
    build.build()
    wl, t_obs, g_o = case
    P = api.Plan(wl, precision=precision, keep_records=1)
    th = P.theta_tensor()
    rec = P.new_records()
    times, rt = P.solve(th, records=rec)
    g = P.backward(th, times, rec, 2.0 * (rt.double() - torch.as_tensor(t_obs, device=rt.device)[None]))
    assert P.status() == 0
    g = g.cpu().numpy()
    m = np.abs(g_o) >= 1e-2 * np.abs(g_o).max(axis=1, keepdims=True)
    rel = np.abs(g - g_o)[m] / np.abs(g_o)[m]
    norm = np.abs(g - g_o).max(axis=1) / np.abs(g_o).max(axis=1)
    print(f"{precision}: element-wise rel error max {rel.max():.2e}, median {np.median(rel):.2e} over {m.sum()} "
          f"components; max-norm error {norm.max():.2e}")
    assert rel.max() < tol
    assert norm.max() < tol_norm
