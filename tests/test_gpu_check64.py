"""The FP64 convergence check on the GPU against the oracle's evaluation of the same check, node by node.

Both sides read the SAME solved field (the GPU's FP32 or FP64 field, cast to double for the oracle) and
evaluate, at every node, the update U(S_D) in double precision with S_D = the frozen neighbours and the
neighbours whose key (tau, index) precedes the node's (the known set of the heap FMM when it accepted the
node, Sec. 2).  The values must agree to rounding (1e-12 relative: the two write the stencil time in
different but equivalent forms), the records exactly, and the per-field summaries (largest relative residual,
count of records that differ from the solve's) must be those of the oracle's values.
"""
import numpy as np
import pytest

from paper_2302_10988_gb300 import workloads as W
from tests.gpu_helpers import oracle_medium

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def api():
    from paper_2302_10988_gb300 import build
    build.build()
    from paper_2302_10988_gb300 import api as A
    return A


def _compare(api, oracle, wl, precision, fields, r0=2):
    P = api.Plan(wl, precision=precision, init_radius=r0)
    th = P.theta_tensor()
    rec = P.new_records()
    times, _ = P.solve(th, records=rec)
    ct, cr, mr, fl = P.check64_nodes(th, times, rec)
    assert P.status() == 0
    torch.cuda.synchronize()
    mr, fl = mr.cpu().numpy(), fl.cpu().numpy()
    # the summaries of the plain check are those of the per-node variant
    mr2, fl2 = P.check64(th, times, rec)
    assert np.array_equal(mr, mr2.cpu().numpy()) and np.array_equal(fl, fl2.cpu().numpy())
    worst_v = worst_res = 0.0
    flips = 0
    for f in fields:
        b, s = divmod(f, P.nsrc)
        M = oracle_medium(oracle, wl, b)
        si, sj = (int(v) for v in wl.samples[b].src[s])
        frozen, _ = oracle.init_radius(M, si, sj, r0)
        tau = P.field(times, f).double().cpu().numpy()
        F_o, rec_o = oracle.F_check(M, frozen, tau)
        F_g = P.field(ct, f).cpu().numpy()
        rec_g = P.field(cr, f).cpu().numpy().astype(np.int64)
        rec_o = np.where(rec_o == -2, 254, np.where(rec_o == -1, 255, rec_o))
        assert np.array_equal(rec_g, rec_o), (f, int((rec_g != rec_o).sum()))
        m = np.isfinite(F_o) & (F_o > 0)
        assert np.array_equal(np.isfinite(F_g), np.isfinite(F_o))
        dv = (np.abs(F_g - F_o)[m] / F_o[m]).max()
        worst_v = max(worst_v, dv)
        assert dv < 1e-12, (f, dv)
        # per-field summaries from the oracle's values: residual (its ratio is taken in FP32 on the GPU) and
        # the records that differ from the solve's
        nf = (frozen.reshape(tau.shape) == 0) & np.isfinite(tau) & (tau > 0)
        res_o = (np.abs(F_o - tau)[nf] / tau[nf]).max() if nf.any() else 0.0
        # (the values agree to 1e-12 relative, so the residuals agree to that absolutely; an FP64 field's
        # residual is itself at rounding level)
        assert mr[f] == pytest.approx(res_o, rel=1e-6, abs=1e-12), (f, mr[f], res_o)
        worst_res = max(worst_res, res_o)
        solve_rec = P.field(rec, f).cpu().numpy().astype(np.int64)
        nflip = int(((solve_rec != rec_o) & (frozen.reshape(tau.shape) == 0)).sum())
        assert fl[f] == nflip, (f, fl[f], nflip)
        flips += nflip
    print(f"{precision}: check values vs oracle {worst_v:.2e}, largest residual {worst_res:.2e}, record flips "
          f"{flips} over {len(fields)} fields")
    return worst_res, flips


def test_check64_weld_256_nodewise(api, oracle):
    wl = W.weld_single()
    res32, _ = _compare(api, oracle, wl, "fp32", (0, 5, 11, 16, 21, 26, 31, 13))
    assert res32 < 1e-6  # an FP32 field is at the FP64 fixed point to FP32 rounding
    res64, flips64 = _compare(api, oracle, wl, "fp64", (0, 16, 31))
    assert res64 < 1e-12 and flips64 == 0


def test_check64_uneven_batch_nodewise(api, oracle):
    wl = W.weld_batch(nsamples=5, nsrc=3, nrec=4, sizes=(64, 96, 128, 160))
    _compare(api, oracle, wl, "fp32", range(15))


def test_check64_corner_sources_and_no_box(api, oracle):
    """Sources in corners and on edges, with no frozen box (r0 = 0) and a wide one (r0 = 5)."""
    wl = W.weld_single(n=90, h=0.5e-3, rg=5, seed=8, nsrc=4, nrec=3)
    wl.samples[0].src[:] = [[0, 0], [89, 89], [0, 45], [44, 44]]
    for r0 in (0, 5):
        _compare(api, oracle, wl, "fp32", range(4), r0=r0)


@pytest.mark.parametrize("precision,sweep,threads", [("fp32", 3, 0), ("fp32", 3, 64), ("fp32", 3, 512),
                                                     ("fp32", 1, 0), ("fp32", 2, 0), ("fp64", 3, 0),
                                                     ("fp64", 2, 0)])
def test_solve_check64_equals_solve_then_check(api, precision, sweep, threads):
    """alf_solve_check64 (the check inside the CTA sweep kernel where that kernel runs it, else launched after
    the solve) returns the fields, records and check summaries of alf_solve followed by alf_check64, bit for
    bit, on an uneven batch (several CTA tiles per field, ragged tails), with and without records."""
    wl = W.weld_batch(nsamples=4, nsrc=3, nrec=4, sizes=(64, 96, 160))
    P = api.Plan(wl, precision=precision, sweep=sweep, cta_threads=threads)
    th = P.theta_tensor()
    rec1, rec2 = P.new_records(), P.new_records()
    t1, rt1 = P.solve(th, records=rec1)
    mr1, fl1 = P.check64(th, t1, rec1)
    t2, rt2, mr2, fl2 = P.solve_check64(th, records=rec2)
    _, _, mr3, fl3 = P.solve_check64(th)
    assert P.status() == 0
    assert torch.equal(t1, t2) and torch.equal(rt1, rt2) and torch.equal(rec1, rec2)
    assert torch.equal(mr1, mr2) and torch.equal(fl1, fl2)
    assert torch.equal(mr1, mr3) and int(fl3.abs().sum()) == 0
    assert float(mr1.max()) < (1e-6 if precision == "fp32" else 1e-12)
    if precision == "fp32" and sweep == 3:
        assert int(fl1.sum()) > 0 or float(mr1.max()) > 0.0  # the summaries were written, not left zero
