"""GPU parity: the CUDA path (through the C ABI) against the FP64 CPU oracle on the same seeded inputs.

Tolerances: max relative travel-time error 1e-6 in the library's FP64 mode and 1e-4 in FP32 mode;
nodes whose stencil record differs from the oracle's are counted and reported.
"""
import numpy as np
import pytest

from paper_2302_10988_gb300 import workloads as W
from tests.gpu_helpers import oracle_field, record_mismatch, rel_err

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def api():
    from paper_2302_10988_gb300 import build
    build.build()
    from paper_2302_10988_gb300 import api as A
    return A


def _solve(api, wl, precision, records=True, **opts):
    P = api.Plan(wl, precision=precision, **opts)
    th = P.theta_tensor()
    rec = P.new_records() if records else None
    times, rt = P.solve(th, records=rec)
    assert P.status() == 0
    torch.cuda.synchronize()
    st = P.stats()
    print(f"[{precision} {len(wl.samples)}x{P.nsrc} fields] evaluations/node {st['evaluations'] / st['nodes']:.2f}, "
          f"rounds {st['rounds']}")
    return P, th, times, rt, rec


def test_velocity_model_on_device(api, oracle):
    ang = np.radians(np.linspace(-180, 180, 721))
    for c6, rho in (W.WELD_TI, W.PAPER_CUBIC, W.PARENT_ISO):
        m = oracle.mat_from_voigt(c6, rho)
        v_o = np.array([oracle.phase_velocity(m, a) for a in ang])
        gp_o = np.array([oracle.group_paper(m, a)[1] for a in ang])
        ge_o = np.array([oracle.group_exact(m, a)[1] for a in ang])
        assert np.max(np.abs(api.eval_velocity(c6, rho, ang, "phase", precision="fp64") / v_o - 1)) < 1e-13
        assert np.max(np.abs(api.eval_velocity(c6, rho, ang, "phase", precision="fp32") / v_o - 1)) < 2e-7
        assert np.max(np.abs(api.eval_velocity(c6, rho, ang, "group", "paper", "fp64") / gp_o - 1)) < 1e-12
        assert np.max(np.abs(api.eval_velocity(c6, rho, ang, "group", "paper", "fp32") / gp_o - 1)) < 2e-6
        assert np.max(np.abs(api.eval_velocity(c6, rho, ang, "group", "exact", "fp64") / ge_o - 1)) < 1e-11


@pytest.mark.parametrize("group", ["paper", "exact"])
def test_homogeneous_ti_fp64(api, oracle, group):
    wl = W.homogeneous_ti()
    P, th, times, rt, rec = _solve(api, wl, "fp64", group=group)
    gm = 0 if group == "paper" else 1
    tau, orec, fr, M = oracle_field(oracle, wl, 0, 0, group_model=gm)
    g = P.field(times, 0).cpu().numpy()
    assert np.isfinite(g).all()
    assert rel_err(g, tau).max() < 1e-6
    assert record_mismatch(P.field(rec, 0).cpu().numpy(), orec, fr) == 0
    r = wl.samples[0].rec
    assert np.allclose(rt.cpu().numpy()[0, 0], tau[r[:, 1], r[:, 0]], rtol=1e-12, atol=0)


@pytest.mark.parametrize("sweep", [1, 2, 3, 4])
@pytest.mark.parametrize("precision,tol", [("fp64", 1e-6), ("fp32", 1e-4)])
def test_weld_ragged_parity(api, oracle, precision, tol, sweep):
    wl = W.weld_single(n=100, h=0.5e-3, rg=5, seed=12, nsrc=3, nrec=5)
    wl.samples[0].src[:] = [[0, 0], [57, 0], [99, 0]]
    for band in (2.0, 4.0, 0.0):
        P, th, times, rt, rec = _solve(api, wl, precision, band_cells=band, sweep=sweep)
        flips = 0
        for s in range(3):
            tau, orec, fr, M = oracle_field(oracle, wl, 0, s)
            g = P.field(times, s).cpu().numpy()
            e = rel_err(g, tau)
            flips += record_mismatch(P.field(rec, s).cpu().numpy(), orec, fr)
            assert e.max() < tol, (band, s, e.max(), flips)
        if precision == "fp64":
            assert flips == 0
        print(f"{precision} band={band}: record flips {flips}")


@pytest.mark.parametrize("sweep", [1, 2, 3, 4])
def test_tiny_and_edge_grids(api, oracle, sweep):
    for (nx, ny, si, sj) in [(2, 2, 0, 0), (3, 7, 2, 6), (33, 9, 32, 0), (65, 17, 0, 16), (40, 40, 20, 20)]:
        rm = np.zeros((ny, nx), np.uint16)
        rm[:, nx // 2:] = 1
        s = W.Sample(nx, ny, 1e-3, rm, np.array([0.0, 0.7]), np.array([[si, sj]], np.int32),
                     np.array([[nx - 1 - si, ny - 1 - sj]], np.int32))
        wl = W.Workload("tiny", [W.WELD_TI, W.PARENT_ISO], np.array([0, 1], np.uint16), [s])
        P, th, times, rt, rec = _solve(api, wl, "fp64", sweep=sweep)
        tau, orec, fr, M = oracle_field(oracle, wl, 0, 0)
        assert rel_err(P.field(times, 0).cpu().numpy(), tau).max() < 1e-6
        assert record_mismatch(P.field(rec, 0).cpu().numpy(), orec, fr) == 0


def test_weld_256_fp64_and_fp32(api, oracle):
    """256 x 256 weld medium, 32 sources: FP64 within 1e-6 and FP32 within 1e-4 of the oracle (8 of the
    32 sources compared), FP64 check of the FP32 fields."""
    wl = W.weld_single()
    P64, th, t64, r64, rec64 = _solve(api, wl, "fp64")
    P32, _, t32, r32, rec32 = _solve(api, wl, "fp32")
    worst64 = worst32 = 0.0
    flips32 = 0
    for s in (0, 5, 11, 16, 21, 26, 31, 13):
        tau, orec, fr, M = oracle_field(oracle, wl, 0, s)
        worst64 = max(worst64, rel_err(P64.field(t64, s).cpu().numpy(), tau).max())
        worst32 = max(worst32, rel_err(P32.field(t32, s).cpu().numpy(), tau).max())
        flips32 += record_mismatch(P32.field(rec32, s).cpu().numpy(), orec, fr)
        assert record_mismatch(P64.field(rec64, s).cpu().numpy(), orec, fr) == 0
    print(f"weld 256: fp64 max rel {worst64:.3e}, fp32 max rel {worst32:.3e}, fp32 record flips {flips32}")
    assert worst64 < 1e-6
    assert worst32 < 1e-4
    mr, fl = P32.check64(th, t32, rec32)
    torch.cuda.synchronize()
    print(f"FP64 check of FP32 fields: max residual {mr.max().item():.3e}, flips {int(fl.sum())}")
    # an FP32 field sits at the FP64 fixed point to FP32 rounding (a few ulp of the stencil arithmetic)
    assert mr.max().item() < 1e-6
    mr64, fl64 = P64.check64(th, t64, rec64)
    torch.cuda.synchronize()
    assert mr64.max().item() < 1e-12 and int(fl64.sum()) == 0


@pytest.mark.parametrize("sweep", [1, 2, 3])
def test_uneven_batch_fp32(api, oracle, sweep):
    wl = W.weld_batch(nsamples=5, nsrc=3, nrec=4, sizes=(64, 96, 128, 160))
    P, th, times, rt, rec = _solve(api, wl, "fp32", sweep=sweep)
    worst = 0.0
    for b in range(5):
        for s in range(3):
            tau, orec, fr, M = oracle_field(oracle, wl, b, s)
            worst = max(worst, rel_err(P.field(times, b * 3 + s).cpu().numpy(), tau).max())
            r = wl.samples[b].rec
            assert np.allclose(rt[b, s].cpu().numpy(), tau[r[:, 1], r[:, 0]], rtol=1e-4)
    assert worst < 1e-4


def test_host_validation_errors(api):
    from paper_2302_10988_gb300 import binding as B
    wl = W.homogeneous_ti()
    wl.samples[0].src[0] = [64, 0]
    with pytest.raises(B.AlfError) as e:
        api.Plan(wl, precision="fp64")
    assert e.value.code == 3
    wl = W.homogeneous_ti()
    bad = (wl.materials[0][0], -1.0)
    wl.materials[0] = bad
    with pytest.raises(B.AlfError) as e:
        api.Plan(wl, precision="fp64")
    assert e.value.code == 2
    wl = W.homogeneous_ti()
    with pytest.raises(B.AlfError) as e:
        api.Plan(wl, precision="fp64", sweep=5)
    assert e.value.code == 1
    with pytest.raises(B.AlfError) as e:
        api.Plan(wl, precision="fp64", sweep=3, cta_threads=96)
    assert e.value.code == 1
    for bad in ({"cta_cluster": 3}, {"cta_cluster": 2, "cta_threads": 256}):
        with pytest.raises(B.AlfError) as e:
            api.Plan(wl, precision="fp64", sweep=3, **bad)
        assert e.value.code == 1


def test_graph_stream_and_timing(api, oracle):
    """The sweep gives the same fields when replayed from a CUDA graph on a side stream, and with event timing."""
    wl = W.weld_batch(nsamples=3, nsrc=2, nrec=3, sizes=(64, 96))
    P = api.Plan(wl, precision="fp32")
    th = P.theta_tensor()
    ref, _ = P.solve(th)
    torch.cuda.synchronize()
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        t1, _ = P.solve(th)
        t2, _ = P.solve(th)
    s.synchronize()
    assert torch.equal(torch.isfinite(ref), torch.isfinite(t1))
    assert (t1 - ref).abs().max().item() <= 1e-4 * ref[torch.isfinite(ref)].max().item()
    assert torch.equal(t1, t2)
    Pt = api.Plan(wl, precision="fp32", time_kernels=1)
    t3, _ = Pt.solve(th)
    st = Pt.stats()
    assert st["eval_launches"] > 0 and st["eval_ms"] > 0 and st["kernel_launches"] > 0
    assert (t3 - ref).abs().max().item() <= 1e-4 * ref[torch.isfinite(ref)].max().item()
    opt = Pt.autotune(th)
    assert opt.band_cells in (1.0, 1.5, 2.0, 2.5, 3.0, 4.0, 6.0) and opt.sweep in (1, 2, 3)
    assert opt.cta_threads in (64, 128, 256, 512)
    t4, _ = Pt.solve(th)
    assert (t4 - ref).abs().max().item() <= 1e-4 * ref[torch.isfinite(ref)].max().item()


def test_sweep_schedules_agree(api, oracle):
    """Every sweep schedule (lockstep rounds, warp per field, CTA per field, active tiles) reaches the unique
    fixed point of F: in FP64 their fields and records are identical bit for bit, on a batch of uneven
    fields, and they match the oracle."""
    wl = W.weld_batch(nsamples=6, nsrc=4, nrec=4, sizes=(32, 64, 96, 128))
    P1, th, t1, _, rec1 = _solve(api, wl, "fp64", sweep=1)
    P2, _, t2, _, rec2 = _solve(api, wl, "fp64", sweep=2)
    P3, _, t3, _, rec3 = _solve(api, wl, "fp64", sweep=3)
    P4, _, t4, _, rec4 = _solve(api, wl, "fp64", sweep=4)
    assert torch.equal(t1, t2) and torch.equal(t1, t3) and torch.equal(t1, t4)
    assert torch.equal(rec1, rec2) and torch.equal(rec1, rec3) and torch.equal(rec1, rec4)
    for nt in (64, 128, 512):  # other numbers of warps on each field's CTA
        Pn, _, tn, _, recn = _solve(api, wl, "fp64", sweep=3, cta_threads=nt, cta_cluster=1)
        assert Pn.options.cta_threads == nt
        assert torch.equal(t1, tn) and torch.equal(rec1, recn)
    for cs in (2, 4, 8):  # one field shared by a cluster of CTAs on as many SMs
        Pn, _, tn, _, recn = _solve(api, wl, "fp64", sweep=3, cta_cluster=cs)
        assert Pn.options.cta_cluster == cs and Pn.options.cta_threads == 512
        assert torch.equal(t1, tn) and torch.equal(rec1, recn)
    for b, s in ((0, 0), (3, 2), (5, 3)):
        tau, orec, fr, M = oracle_field(oracle, wl, b, s)
        assert rel_err(P2.field(t2, b * 4 + s).cpu().numpy(), tau).max() < 1e-6
        assert record_mismatch(P2.field(rec2, b * 4 + s).cpu().numpy(), orec, fr) == 0


def test_tile_sweep_fp32_matches_cta_sweep(api):
    """The active-tile schedule (8 x 8 tiles iterated in shared memory, no front band) reaches the fixed point
    the CTA sweep reaches, in FP32 too: fields and records identical bit for bit on uneven fields with the
    sources on the edges and inside, and the same travel times at the receivers."""
    wl = W.weld_batch(nsamples=4, nsrc=3, nrec=4, sizes=(40, 96, 130))
    wl.samples[1].src[1] = [wl.samples[1].nx // 2, wl.samples[1].ny // 2]
    P3, th, t3, rt3, rec3 = _solve(api, wl, "fp32", sweep=3)
    P4, _, t4, rt4, rec4 = _solve(api, wl, "fp32", sweep=4)
    assert P4.options.sweep == 4
    assert torch.equal(t3, t4) and torch.equal(rec3, rec4) and torch.equal(rt3, rt4)


@pytest.mark.parametrize("cs", [2, 4])
def test_cluster_sweep_fp32(api, oracle, cs):
    """FP32 fields solved by clusters of CTAs (one field on several SMs) match the FP64 oracle within 1e-4,
    on a batch of ragged fields; for these few small fields the plan's default is one 512-thread CTA each."""
    wl = W.weld_batch(nsamples=3, nsrc=3, nrec=4, sizes=(96, 160, 224))
    P, th, times, rt, rec = _solve(api, wl, "fp32", sweep=3, cta_cluster=cs)
    assert P.options.cta_cluster == cs
    worst = 0.0
    for b in range(3):
        for s in range(3):
            tau, orec, fr, M = oracle_field(oracle, wl, b, s)
            worst = max(worst, rel_err(P.field(times, b * 3 + s).cpu().numpy(), tau).max())
    assert worst < 1e-4
    Pd = api.Plan(wl, precision="fp32", sweep=3)
    assert Pd.options.cta_threads == 512 and Pd.options.cta_cluster == 1
    td, _ = Pd.solve(th)
    assert (td - times).abs().max().item() <= 1e-4 * times[torch.isfinite(times)].max().item()
