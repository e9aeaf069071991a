"""GPU parity of the drop diagnostics beyond the pair statistics, through
the C ABI: the inertia tensor and aspect ratio of every drop (Appendix A),
their running mean in vof_stats, statistics sampled every n steps inside
vof_step (Section 3 samples events every 10 steps), and the tracer count
N(t) that the step reports (Section 2.3)."""
import numpy as np
import pytest

import oracle as O
from paper_2407_07463_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

DEV = "cuda:0"


@pytest.fixture(scope="module")
def vof():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2407_07463_gb300 import build, vof

    build.build()
    vof.lib()
    return vof


@pytest.fixture(scope="module")
def case():
    return synth.make_workload("shape parity", shape=(48, 56, 64), phi=0.15, radius=6.0, n_modes=8,
                               amplitude=0.5, drift=1.0, cfl=0.3, seed=21)


def context(vof, wl, precision=0, **kw):
    nz, ny, nx = wl.shape
    dt = torch.float64 if precision == 0 else torch.float32
    cfg = vof.make_config(nx, ny, nz, k_capacity=wl.k_capacity, k_active=wl.k_active, precision=precision,
                          stats_rbins=400, stats_dr=0.25, **kw)
    c = torch.from_numpy(wl.c).to(DEV, dt).contiguous()
    u = torch.from_numpy(wl.u).to(DEV, dt).contiguous()
    return vof.Context(cfg, c, u), c, u


def tensors(I):
    I = np.asarray(I)
    return np.stack([np.stack([I[:, 0], I[:, 3], I[:, 4]], -1), np.stack([I[:, 3], I[:, 1], I[:, 5]], -1),
                     np.stack([I[:, 4], I[:, 5], I[:, 2]], -1)], -2)


@pytest.mark.parametrize("precision", [0, 1])
def test_drop_shape_matches_oracle(vof, case, precision):
    """After a few steps (the drops deform), every drop's tensor within 1e-10
    of the largest entry of the oracle's, chi within 1e-10 relative."""
    ctx, c_d, _ = context(vof, case, precision)
    ctx.vof_step(case.dt, 4)
    got = c_d.cpu().numpy().astype(np.float64)
    nd = 0
    for f in range(case.k_active):
        lab, n = ctx.vof_label(f)
        vol, cen = ctx.vof_drop_table(f, lab, n)
        I, chi = ctx.vof_drop_shape(f, lab, n, cen)
        torch.cuda.synchronize()
        lab_h = lab.cpu().numpy()
        Io, chio = O.drop_inertia(got[f], lab_h, n, cen=cen.cpu().numpy())
        Ig = I.cpu().numpy()
        assert np.abs(Ig - Io).max() <= 1e-10 * np.abs(Io).max()
        np.testing.assert_allclose(chi.cpu().numpy(), chio, rtol=1e-10)
        # the oracle's own centroids give the same tensors
        _, ceno = O.drop_table(got[f], lab_h, n)
        Io2, _ = O.drop_inertia(got[f], lab_h, n, cen=ceno)
        assert np.abs(Io2 - Io).max() <= 1e-9 * np.abs(Io).max()
        nd += n
    assert nd > 10
    ctx.close()


def test_stats_chi_mean_and_sampling_cadence(vof, case):
    """vof_stats's running chi mean is the mean over the drops of all fields;
    a context sampling every 3 steps inside vof_step accumulates the same
    events as explicit vof_stats calls after steps 3 and 6 of a twin."""
    a, ca, _ = context(vof, case, 0, stats_every=3)
    b, cb, _ = context(vof, case, 0)
    a.vof_step(case.dt, 7)
    for s in range(7):
        b.vof_step(case.dt, 1)
        if s in (2, 5):
            b.vof_stats(reset=False, histograms=False)
    sa = a.vof_stats(reset=False)  # a third event for both, after step 7
    sb = b.vof_stats(reset=False)
    assert sa["events"] == sb["events"] > 0
    np.testing.assert_allclose(sa["hist_r"], sb["hist_r"], rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(sa["R"], sb["R"], rtol=1e-10, atol=1e-12)
    assert sa["chi_drops"] == sb["chi_drops"] and sa["chi_mean"] == pytest.approx(sb["chi_mean"], rel=1e-12)
    # the chi statistics of one event against the oracle on the GPU's field
    r = b.vof_stats(reset=True, histograms=False)
    got = cb.cpu().numpy()
    chis = []
    for f in range(case.k_active):
        lab, n = O.label(got[f], tau=b.cfg.tag_tau)
        if n:
            chis.append(O.drop_inertia(got[f], lab, n)[1])
    chis = np.concatenate(chis)
    assert r["chi_drops"] == len(chis)
    assert r["chi_mean"] == pytest.approx(chis.mean(), rel=1e-10)
    assert r["chi_max"] == pytest.approx(chis.max(), rel=1e-10)
    assert 1.0 <= r["chi_mean"] < 1.5
    a.close()
    b.close()


def test_tracer_count_reported_by_the_step(vof, case):
    """N(t): the fields that hold an occupied cell when Step 1 runs, i.e.
    after the step's transport, counted on the field the step produced."""
    a, ca, _ = context(vof, case, 0, recolour=1)
    b, cb, _ = context(vof, case, 0)
    ra = a.vof_step(case.dt, 1)
    b.vof_step(case.dt, 1)
    got = cb.cpu().numpy()
    want = int(sum((got[f] > b.cfg.tag_tau).any() for f in range(case.k_active)))
    assert ra["n_in_use"] == want == ra["n_in_use_max"]
    assert b.vof_step(case.dt, 1)["n_in_use"] == -1
    a.close()
    b.close()
