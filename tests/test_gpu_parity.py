"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Bars: FP64 path within 1e-11 relative (max-norm over targets, per layer); mixed-precision far
field within 1e-6.  Per target, each target's error against its own magnitude (floored at 1e-3 of
the largest; parity.per_target_rel_err): FP64 within 1e-11, mixed within 1e-5.  Sizes span several far-field tiles and ragged tails; the full-size bench
workload is checked on a seeded sample of targets.
"""
import numpy as np
import pytest

import oracle
import workloads
from parity import GpuProblem, oracle_eval, oracle_problem, per_target_rel_err, rel_err

pytestmark = pytest.mark.gpu
FP64_TOL = 1e-11
MIXED_TOL = 1e-6
# Per target the mixed path is held to 1e-5: its error is absolute (FP32 rounding of the far-field
# terms, about 1e-7 of the largest values), so a target whose value is 10-50 times smaller than the
# largest sees a relative error that much larger (measured up to 6.3e-6 on the ellipsoid's box points).
PER_TARGET_TOL = {0: FP64_TOL, 1: 1e-5}


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
def test_nodes_match_oracle(ers, name):
    g = gpu(name)
    _, x, n, w, _, _ = oracle_problem(name)
    xd, nd, wd = (t.cpu().numpy() for t in g.s.nodes())
    assert xd.shape == x.shape
    assert np.abs(xd - x).max() <= 1e-15 and np.abs(nd - n).max() <= 1e-15
    assert np.abs(wd - w).max() <= 1e-15 * w.max()


@pytest.mark.parametrize("shape", [workloads.unit_sphere((0.1, 0.0, -0.2)), workloads.Shape((0.0, 0.0, 0.0), (1.0, 0.8, 0.6))])
def test_closest_point_matches_oracle(ers, shape):
    import torch
    s = ers.Surface(shape.center, shape.axes, 1 / 16)
    rng = np.random.default_rng(9)
    yb, _, _, _ = workloads.near_band_targets(shape, 3000, 0.3, rng)
    yf = rng.uniform(-2, 2, (3000, 3))
    xs, _, _ = oracle.quadrature(shape, 1 / 16)
    y = np.concatenate([yb, yf, xs[:500]])
    x0, n0, b = (t.cpu().numpy() for t in s.closest_point(torch.from_numpy(y).cuda()))
    x0o, n0o, bo = oracle.closest_point(shape, y)
    assert np.abs(b - bo).max() < 1e-13
    assert (b[-500:] == 0).all()  # node targets are on the surface
    ok = np.abs(bo) < 0.35  # unique closest point inside the reach of the ellipsoid
    assert np.abs(x0 - x0o)[ok].max() < 1e-12
    assert np.abs(n0 - n0o)[ok].max() < 1e-11


@pytest.mark.parametrize("name", ["sphere16", "sphere32"])
@pytest.mark.parametrize("precision,tol", [(0, FP64_TOL), (1, MIXED_TOL)])
def test_eval_all_targets(ers, name, precision, tol):
    y, uo, vo, bo = oracle_eval(name)
    g = gpu(name)
    u, v, b = g.eval(g.targets(), precision=precision)
    assert np.abs(b - bo).max() < 1e-13
    eu, ev = rel_err(u, uo), rel_err(v, vo)
    assert eu <= tol and ev <= tol, (eu, ev)
    pu, pv = per_target_rel_err(u, uo), per_target_rel_err(v, vo)
    assert pu <= PER_TARGET_TOL[precision] and pv <= PER_TARGET_TOL[precision], (pu, pv)


def test_eval_ellipsoid_with_far_points(ers):
    """Ellipsoid (1, 0.8, 0.6) at h = 1/32: node, band and box targets (inside, outside, far)."""
    shape = workloads.Shape((0.0, 0.0, 0.0), (1.0, 0.8, 0.6))
    wl = workloads.make_workload("ell32", shape, 1 / 32, (2, 3, 4), 77, 1500, 16 / 32 * 0.7, n_far=700)
    g = GpuProblem("ell32", wl)
    x, n, w = oracle.quadrature(shape, wl.h)
    sel = np.concatenate([np.arange(0, len(w), 11), len(w) + np.arange(len(wl.extra_targets))])
    y = np.concatenate([x, wl.extra_targets])[sel]
    x0, n0, b = oracle.closest_point(shape, y)
    f0, q0 = workloads.poly_eval(wl.f_coef, x0), workloads.poly_eval(wl.q_coef, x0)
    uo, vo, _ = oracle.evaluate(x, n, w, workloads.poly_eval(wl.f_coef, x), workloads.poly_eval(wl.q_coef, x),
                                y, x0, n0, b, f0, q0, wl.h, wl.rho)
    for prec, tol in ((0, FP64_TOL), (1, MIXED_TOL)):
        u, v, bg = g.eval(g.targets(sel), precision=prec)
        assert rel_err(u, uo) <= tol and rel_err(v, vo) <= tol, (prec, rel_err(u, uo), rel_err(v, vo))
        pu, pv = per_target_rel_err(u, uo), per_target_rel_err(v, vo)
        assert pu <= PER_TARGET_TOL[prec] and pv <= PER_TARGET_TOL[prec], (prec, pu, pv)


def test_eval_far_from_the_origin_and_scaled(ers):
    """Ellipsoid (4, 3.2, 2.4) centred at (40, -25, 12), h = 1/8 (a unit-size case moved and scaled
    by 4): the tile-relative FP32 far field, the FP32 prefilter at absolute coordinates ~50 and the
    near field at kernel factors 4^p times smaller, on node, band and box targets; densities are
    polynomials of the coordinates relative to the centre, divided by 4."""
    import torch
    shape = workloads.Shape((40.0, -25.0, 12.0), (4.0, 3.2, 2.4))
    h, rho = 1 / 8, (2, 3, 4)
    c = np.asarray(shape.center)
    rng = np.random.default_rng(404)
    fc, qc = workloads.density_coeffs(rng), workloads.density_coeffs(rng)
    dens = lambda coef, pts: workloads.poly_eval(coef, (pts - c) / 4.0)
    x, n, w = oracle.quadrature(shape, h)
    yb = workloads.near_band_targets(shape, 1500, 6 * rho[2] * h * 0.7, rng)[0]
    yf = c + rng.uniform(-8.0, 8.0, (300, 3))
    y = np.concatenate([x[::5], yb, yf])
    x0, n0, b = oracle.closest_point(shape, y)
    uo, vo, _ = oracle.evaluate(x, n, w, dens(fc, x), dens(qc, x), y, x0, n0, b, dens(fc, x0), dens(qc, x0), h, rho)
    s = ers.Surface(shape.center, shape.axes, h)
    xd = s.nodes()[0].cpu().numpy()
    assert np.abs(xd - x).max() <= 1e-13
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    s.set_density(t(dens(fc, xd)), t(dens(qc, xd)))
    yd = t(y)
    x0d, n0d, bd = s.closest_point(yd)
    assert np.abs(bd.cpu().numpy() - b).max() < 1e-12
    x0h = x0d.cpu().numpy()
    for prec, tol in ((0, FP64_TOL), (1, MIXED_TOL)):
        u, v = s.eval(yd, t(dens(fc, x0h)), t(dens(qc, x0h)), rho=rho, precision=prec, x0=x0d, n0=n0d, b=bd)
        u, v = u.cpu().numpy(), v.cpu().numpy()
        assert rel_err(u, uo) <= tol and rel_err(v, vo) <= tol, (prec, rel_err(u, uo), rel_err(v, vo))
        pu, pv = per_target_rel_err(u, uo), per_target_rel_err(v, vo)
        assert pu <= PER_TARGET_TOL[prec] and pv <= PER_TARGET_TOL[prec], (prec, pu, pv)


# Below 6 the cutoff is a non-tie value: the lattice rule has many node pairs at exact multiples
# of h (t = i at delta = 2h), and where t = cutoff_t exactly, s_p jumps by eps_p(cutoff_t)
# (6e-6 at 4, 4e-14 at 6), so ulp-level differences between two sets of nodes decide the result.
@pytest.mark.parametrize("rho,tc", [((3, 4, 5), 6.0), ((2, 3, 4), 5.3), ((1.5, 2.5, 3.5), 7.5), ((2, 3, 4), 4.3)])
def test_other_rho_and_cutoff(ers, rho, tc):
    sel = np.arange(0, 17070 + 2000, 7)
    y, uo, vo, _ = oracle_eval("sphere32", sel=sel, rho=rho, tc=tc)
    g = gpu("sphere32")
    u, v, _ = g.eval(g.targets(sel), precision=0, rho=rho, tc=tc)
    assert rel_err(u, uo) <= FP64_TOL and rel_err(v, vo) <= FP64_TOL


def test_layers_and_given_closest_point(ers):
    g = gpu("sphere16")
    y = g.targets()
    u, v, _ = g.eval(y)
    us, _, _ = g.eval(y, layers=1)
    _, vd, _ = g.eval(y, layers=2)
    ug, vg, _ = g.eval(y, given_cp=True)
    assert np.abs(us - u).max() <= 1e-14 * np.abs(u).max()
    assert np.abs(vd - v).max() <= 1e-14 * np.abs(v).max()
    assert np.array_equal(ug, u) and np.array_equal(vg, v)


@pytest.mark.parametrize("name", ["sphere16", "sphere32"])
def test_concurrent_and_serial_mixed_paths_agree(ers, name):
    """ERS_OPT_CONCURRENT runs the far field on a second stream, concurrently with the near field,
    and adds it afterwards; the serial order gives the same sums up to the order of two adds."""
    g = gpu(name)
    y = g.targets()
    yd, x0, n0, b, f0, q0 = g.prepare(y)
    uc, vc = g.s.eval(yd, f0, q0, rho=g.wl.rho, precision=1, x0=x0, n0=n0, b=b, concurrent=True)
    uc, vc = uc.cpu().numpy(), vc.cpu().numpy()
    us, vs = g.s.eval(yd, f0, q0, rho=g.wl.rho, precision=1, x0=x0, n0=n0, b=b)
    us, vs = us.cpu().numpy(), vs.cpu().numpy()
    assert np.abs(uc - us).max() <= 1e-14 * np.abs(us).max()
    assert np.abs(vc - vs).max() <= 1e-14 * np.abs(vs).max()
    # a second concurrent call gives bit-identical results (no order-dependent reduction)
    u2, v2 = g.s.eval(yd, f0, q0, rho=g.wl.rho, precision=1, x0=x0, n0=n0, b=b, concurrent=True)
    assert np.array_equal(u2.cpu().numpy(), uc) and np.array_equal(v2.cpu().numpy(), vc)


def test_profile_reports_both_orders(ers):
    g = gpu("sphere32")
    y = g.targets()
    yd, x0, n0, b, f0, q0 = g.prepare(y)
    g.s.profile(True)
    try:
        for conc in (False, True):
            g.s.eval(yd, f0, q0, rho=g.wl.rho, precision=1, x0=x0, n0=n0, b=b, concurrent=conc)
            tc, tf, tn = g.s.last_profile()
            assert tc == 0.0 and tf > 0.0 and tn > 0.0
    finally:
        g.s.profile(False)


def test_pair_counts_are_consistent(ers):
    """Near pairs by regularized deltas (cutoff) and by defect-path deltas both add up to the
    near-pair count; near + far pairs cover every (target, node) pair."""
    g = gpu("sphere32")
    y = g.targets()
    g.eval(y, precision=1)
    nt, npairs, nfar = g.s.last_counts()
    assert npairs + nfar == len(y) * g.s.nodes()[0].shape[0]
    cut, dfx = g.s.last_class_counts(), g.s.last_defect_class_counts()
    assert sum(cut) == npairs and sum(dfx) == npairs and len(dfx) == 4
    # on a surface the pair count grows with the area of the disc r < t delta: every class is populated
    assert min(cut) > 0 and min(dfx) > 0


def test_eval_host_matches_device(ers):
    g = gpu("sphere16")
    y = g.targets()
    u, v, _ = g.eval(y, precision=1)
    yd, x0, n0, b, f0, q0 = g.prepare(y)
    uh, vh = g.s.eval_host(y, f0.cpu().numpy(), q0.cpu().numpy(), rho=g.wl.rho, precision=1)
    assert np.array_equal(uh, u) and np.array_equal(vh, v)


@pytest.mark.parametrize("count", [1, 31, 257, 1001])
def test_ragged_target_counts(ers, count):
    rng = np.random.default_rng(count)
    g = gpu("sphere16")
    sel = np.sort(rng.choice(4302 + 2000, count, replace=False))
    y, uo, vo, _ = oracle_eval("sphere16", sel=sel)
    u, v, _ = g.eval(g.targets(sel))
    assert rel_err(u, uo) <= FP64_TOL and rel_err(v, vo) <= FP64_TOL


def test_tiny_surface_fewer_nodes_than_a_tile(ers):
    shape = workloads.unit_sphere((0.05, 0.0, 0.0))
    wl = workloads.make_workload("tiny", shape, 0.3, (2, 3, 4), 5, 40, 1.0, n_far=10)
    g = GpuProblem("tiny", wl)
    assert g.s.N < 256
    x, n, w = oracle.quadrature(shape, wl.h)
    y = np.concatenate([x, wl.extra_targets])
    x0, n0, b = oracle.closest_point(shape, y)
    uo, vo, _ = oracle.evaluate(x, n, w, workloads.poly_eval(wl.f_coef, x), workloads.poly_eval(wl.q_coef, x),
                                y, x0, n0, b, workloads.poly_eval(wl.f_coef, x0), workloads.poly_eval(wl.q_coef, x0),
                                wl.h, wl.rho)
    u, v, _ = g.eval(g.targets())
    assert rel_err(u, uo) <= FP64_TOL and rel_err(v, vo) <= FP64_TOL


def test_empty_and_errors(ers):
    import torch
    g = gpu("sphere16")
    empty = torch.zeros((0, 3), dtype=torch.float64, device="cuda")
    u, v = g.s.eval(empty, empty, empty, rho=(2, 3, 4))
    assert u.shape == (0, 3)
    y = torch.zeros((4, 3), dtype=torch.float64, device="cuda")
    with pytest.raises(ers.ErsError) as e:
        g.s.eval(y, y, y, rho=(3, 2, 4))
    assert e.value.code == ers.ERS_E_INVAL
    with pytest.raises(ers.ErsError) as e:
        g.s.eval(y, y, y, cutoff_t=9.0)
    assert e.value.code == ers.ERS_E_UNSUPPORTED
    s2 = ers.Surface((0, 0, 0), (1, 1, 1), 1 / 8)
    with pytest.raises(ers.ErsError) as e:
        s2.eval(y, y, y)
    assert e.value.code == ers.ERS_E_STATE
    s2.set_density(f=torch.zeros((s2.N, 3), dtype=torch.float64, device="cuda"))
    s2.set_density(q=torch.zeros((s2.N, 3), dtype=torch.float64, device="cuda"))
    _, _ = s2.eval(y, y, y, cutoff_t=5.0)
    assert s2.last_rc == ers.ERS_W_CUTOFF


@pytest.mark.parametrize("precision,tol", [(1, MIXED_TOL), (0, FP64_TOL)])
def test_full_size_bench_workload_sampled(ers, precision, tol):
    """Unit sphere h = 1/128 (N = 272,718), all 392,718 targets in one launch as in bench.py;
    a seeded sample of 400 targets (nodes, band, far) is checked against the oracle."""
    g = gpu("sphere128")
    y_all = g.targets()
    u, v, b = g.eval(y_all, precision=precision)
    M = len(y_all)
    sel = workloads.subsample(400, M, 4242)
    y, uo, vo, bo = oracle_eval("sphere128", sel=sel)
    assert np.array_equal(y, y_all[sel])
    assert rel_err(u[sel], uo) <= tol and rel_err(v[sel], vo) <= tol, (rel_err(u[sel], uo), rel_err(v[sel], vo))
    pu, pv = per_target_rel_err(u[sel], uo), per_target_rel_err(v[sel], vo)
    assert pu <= PER_TARGET_TOL[precision] and pv <= PER_TARGET_TOL[precision], (pu, pv)
    assert np.isfinite(u).all() and np.isfinite(v).all()


@pytest.mark.parametrize("precision,tol", [(0, FP64_TOL), (1, MIXED_TOL)])
def test_full_size_ellipsoid_workload_sampled(ers, precision, tol):
    """The plain-FP64-at-scale workload: ellipsoid (1, 0.8, 0.6) at h = 1/64, nodes + 60,000 band
    points |b| <= 4 delta_3 + 20,000 box points, all targets in one launch; a seeded sample of
    400 targets against the oracle."""
    g = gpu("ellipsoid64")
    y_all = g.targets()
    u, v, b = g.eval(y_all, precision=precision)
    sel = workloads.subsample(400, len(y_all), 6464)
    y, uo, vo, bo = oracle_eval("ellipsoid64", sel=sel)
    assert np.array_equal(y, y_all[sel])
    assert np.array_equal(b[sel] == 0, bo == 0) and (bo == 0).sum() > 50
    assert rel_err(u[sel], uo) <= tol and rel_err(v[sel], vo) <= tol, (rel_err(u[sel], uo), rel_err(v[sel], vo))
    pu, pv = per_target_rel_err(u[sel], uo), per_target_rel_err(v[sel], vo)
    assert pu <= PER_TARGET_TOL[precision] and pv <= PER_TARGET_TOL[precision], (pu, pv)
    assert np.isfinite(u).all() and np.isfinite(v).all()
