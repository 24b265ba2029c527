"""ERS_OPT_SHARP: targets on the surface evaluated with the modified smoothing functions s#_p of
Sec. 2.1 (one delta, no extrapolation), against the oracle's on-surface path."""
import numpy as np
import pytest

from parity import GpuProblem, oracle_eval_sharp, rel_err

pytestmark = pytest.mark.gpu
FP64_TOL = 1e-11
MIXED_TOL = 1e-6


@pytest.fixture(scope="module")
def ers():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2507_00156_gb300
    return paper_2507_00156_gb300


_cache = {}


def gpu(name):
    if name not in _cache:
        _cache[name] = GpuProblem(name)
    return _cache[name]


@pytest.mark.parametrize("name", ["sphere16", "sphere32"])
@pytest.mark.parametrize("precision,tol", [(0, FP64_TOL), (1, MIXED_TOL)])
def test_sharp_matches_oracle(ers, name, precision, tol):
    """Node targets (b = 0) take the s# path, band targets the extrapolated one."""
    y, uo, vo, bo = oracle_eval_sharp(name, rho_sharp=3.0)
    g = gpu(name)
    u, v, b = g.eval(g.targets(), precision=precision, sharp=True, rho_sharp=3.0)
    assert (b == 0).sum() == (bo == 0).sum() > 0
    eu, ev = rel_err(u, uo), rel_err(v, vo)
    assert eu <= tol and ev <= tol, (eu, ev)


@pytest.mark.parametrize("rho_sharp,tc", [(0.0, 6.0), (4.0, 6.0), (2.5, 7.5), (3.0, 5.3)])
def test_sharp_other_delta_and_cutoff(ers, rho_sharp, tc):
    """rho_sharp = 0 selects rho[1]; larger cutoffs need the table up to tau = 64."""
    sel = np.arange(0, 17070 + 2000, 5)
    y, uo, vo, _ = oracle_eval_sharp("sphere32", sel=sel, rho_sharp=rho_sharp or 3.0, tc=tc)
    g = gpu("sphere32")
    u, v, _ = g.eval(g.targets(sel), precision=0, sharp=True, rho_sharp=rho_sharp, tc=tc)
    assert rel_err(u, uo) <= FP64_TOL and rel_err(v, vo) <= FP64_TOL, (rel_err(u, uo), rel_err(v, vo))


def test_sharp_counts_and_off_surface_targets(ers):
    g = gpu("sphere32")
    y = g.targets()
    u3, v3, b = g.eval(y, precision=1)
    us, vs, _ = g.eval(y, precision=1, sharp=True)
    on = b == 0
    # off the surface nothing changes; on it the two O(h^5) methods agree to their accuracy at
    # h = 1/32 (the oracle gives differences of 3.5e-6 and 2.4e-4 for these densities)
    assert np.array_equal(us[~on], u3[~on]) and np.array_equal(vs[~on], v3[~on])
    assert rel_err(us[on], u3[on]) < 2e-5 and rel_err(vs[on], v3[on]) < 5e-4
    assert not np.array_equal(us[on], u3[on])
    _, npairs, _ = g.s.last_counts()
    nsh = g.s.last_sharp_pairs()
    assert 0 < nsh < npairs
    assert sum(g.s.last_class_counts()) + nsh == npairs


def test_sharp_rejected_where_unsupported(ers):
    import torch
    g = gpu("sphere16")
    y = g.targets()[:64]
    yd, x0, n0, b, f0, q0 = g.prepare(y)
    u = torch.empty((64, 3), dtype=torch.float64, device="cuda")
    v = torch.empty((64, 3), dtype=torch.float64, device="cuda")
    with pytest.raises(ers.ErsError) as ex:
        g.s.eval_noalloc(yd, x0, n0, b, f0, q0, u, v, rho=g.wl.rho, sharp=True)
    assert ex.value.code == -5
    with pytest.raises(ers.ErsError):
        g.s.eval(yd, f0, q0, rho=g.wl.rho, sharp=True, rho_sharp=-1.0)


def test_sharp_full_size_bench_workload_sampled(ers):
    """The bench workload with the on-surface option as the bench's leg runs it (mixed precision,
    delta# = rho_1 h, all 392,718 targets); a seeded sample against the oracle."""
    import workloads
    g = gpu("sphere128")
    y_all = g.targets()
    u, v, _ = g.eval(y_all, precision=1, sharp=True)
    sel = workloads.subsample(300, len(y_all), 7373)
    y, uo, vo, bo = oracle_eval_sharp("sphere128", sel=sel, rho_sharp=3.0)
    assert np.array_equal(y, y_all[sel]) and (bo == 0).sum() > 50
    assert rel_err(u[sel], uo) <= MIXED_TOL and rel_err(v[sel], vo) <= MIXED_TOL


@pytest.mark.parametrize("precision,tol", [(0, FP64_TOL), (1, MIXED_TOL)])
def test_sharp_ellipsoid_with_far_points(ers, precision, tol):
    """Ellipsoid (1, 0.8, 0.6) at h = 1/32 (curvature varying over the surface): every 11th node
    (the s# path) and the band and box targets (extrapolated or far), against the oracle."""
    import oracle
    import workloads
    shape = workloads.Shape((0.0, 0.0, 0.0), (1.0, 0.8, 0.6))
    wl = workloads.make_workload("ell32", shape, 1 / 32, (2, 3, 4), 77, 1500, 16 / 32 * 0.7, n_far=700)
    g = GpuProblem("ell32", wl)
    x, n, w = oracle.quadrature(shape, wl.h)
    sel = np.concatenate([np.arange(0, len(w), 11), len(w) + np.arange(len(wl.extra_targets))])
    y = np.concatenate([x, wl.extra_targets])[sel]
    x0, n0, b = oracle.closest_point(shape, y)
    f0, q0 = workloads.poly_eval(wl.f_coef, x0), workloads.poly_eval(wl.q_coef, x0)
    uo, vo, _ = oracle.evaluate_sharp(x, n, w, workloads.poly_eval(wl.f_coef, x), workloads.poly_eval(wl.q_coef, x),
                                      y, x0, n0, b, f0, q0, wl.h, wl.rho, 6.0, 3.0)
    u, v, bg = g.eval(g.targets(sel), precision=precision, sharp=True, rho_sharp=3.0)
    assert (bg == 0).sum() == (b == 0).sum() > 0
    eu, ev = rel_err(u, uo), rel_err(v, vo)
    assert eu <= tol and ev <= tol, (eu, ev)
