"""The large single medium at full size: 2048 x 2048 nodes at 0.1 mm, a 1300 x 1300 weld of 100 x 100 regions,
64 sources on the bottom edge and 4096 receivers per source (262,144 rays), FP32 with FP64 angle inversion.

Checked at full size, in the launch configuration the library picks:
  * one whole field (the middle source) against the FP64 oracle, node by node (max relative error 1e-4);
  * every node of every field through the FP64 check (relative residual of F64 at the FP32 field);
  * every ray traced to its source, with its integrated time consistent with the field at the receiver,
    and a sample of rays against the oracle's tracer on the oracle's field.
"""
import numpy as np
import pytest

from paper_2302_10988_gb300 import workloads as W
from tests.gpu_helpers import oracle_field, rel_err

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def api():
    from paper_2302_10988_gb300 import build
    build.build()
    from paper_2302_10988_gb300 import api as A
    return A


def test_large_medium_full_size(api, oracle):
    wl = W.weld_large()
    P = api.Plan(wl, precision="fp32", max_ray_points=1024)  # about 2048 / 4 planes per ray
    th = P.theta_tensor()
    rec = P.new_records()
    times, rt = P.solve(th, records=rec)
    assert P.status() == 0
    st = P.stats()
    print(f"2048^2 x 64: sweep {P.options.sweep}, {P.options.cta_threads} threads x {P.options.cta_cluster} CTAs "
          f"per field, evaluations/node {st['evaluations'] / st['nodes']:.2f}, rounds {st['rounds']}")
    nsm = torch.cuda.get_device_properties(0).multi_processor_count
    if nsm >= 128:  # 64 fields of 2^22 nodes: a cluster of 2 SMs on each
        assert P.options.sweep == 3 and P.options.cta_cluster == 2
    mr, fl = P.check64(th, times, rec)
    torch.cuda.synchronize()
    print(f"FP64 check: max residual {mr.max().item():.3e}, record flips {int(fl.sum())} of {P.total_nodes}")
    assert mr.max().item() < 1e-4
    s = 31
    tau, orec, fr, M = oracle_field(oracle, wl, 0, s)
    g = P.field(times, s).cpu().numpy()
    e = rel_err(g, tau)
    print(f"field {s} vs oracle: max rel {e.max():.3e}, mean rel {e.mean():.3e}")
    assert e.max() < 1e-4
    pts, npts, rtime, rst = P.trace_rays(th, times)
    assert P.status() == 0
    assert int((rst != 0).sum()) == 0
    rt_np, rtime_np = rt.cpu().numpy(), rtime.cpu().numpy()
    ratio = rtime_np / rt_np
    print(f"ray time / field time at the receivers: min {ratio.min():.4f}, max {ratio.max():.4f}")
    assert ratio.min() > 0.97 and ratio.max() < 1.05
    # a sample of rays of the compared field against the oracle's tracer on the oracle's field
    src = wl.samples[0].src[s]
    for r in range(0, 4096, 512):
        opts, ost = oracle.trace_ray(M, tau, wl.samples[0].rec[r], src)
        assert ost == 0
        assert float(rtime[0, s, r]) == pytest.approx(oracle.path_time(M, opts), rel=2e-3)
