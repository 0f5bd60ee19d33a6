"""After a solve, the FP64 check, the rays and the adjoint of one plan may run at the same time on three
streams: they give the same results as when they run one after the other."""
import pytest

from paper_2302_10988_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def api():
    from paper_2302_10988_gb300 import build
    build.build()
    from paper_2302_10988_gb300 import api as A
    return A


@pytest.mark.parametrize("sweep", [1, 2])
def test_check_rays_adjoint_on_three_streams(api, sweep):
    wl = W.weld_batch(nsamples=6, nsrc=4, nrec=6, sizes=(64, 96, 128))
    P = api.Plan(wl, precision="fp32", keep_records=1, sweep=sweep)
    th = P.theta_tensor()
    rec = P.new_records()
    times, rt = P.solve(th, records=rec)
    dT = 2.0 * rt
    mr0, fl0 = P.check64(th, times, rec)
    pts0, np0, rtime0, st0 = P.trace_rays(th, times)
    g0 = P.backward(th, times, rec, dT)
    torch.cuda.synchronize()
    main = torch.cuda.current_stream()
    side = [torch.cuda.Stream(), torch.cuda.Stream()]
    done = torch.cuda.Event()
    done.record(main)
    for s in side:
        s.wait_event(done)
    with torch.cuda.stream(side[0]):
        mr1, fl1 = P.check64(th, times, rec)
    with torch.cuda.stream(side[1]):
        pts1, np1, rtime1, st1 = P.trace_rays(th, times)
    g1 = P.backward(th, times, rec, dT)
    for s in side:
        main.wait_stream(s)
    torch.cuda.synchronize()
    assert P.status() == 0
    assert torch.equal(mr0, mr1) and torch.equal(fl0, fl1)
    assert torch.equal(np0, np1) and torch.equal(rtime0, rtime1) and torch.equal(st0, st1)
    # the adjoint adds FP32 contributions with atomics: equal up to their order
    assert torch.allclose(g0, g1, rtol=0, atol=1e-5 * g0.abs().max().item())
