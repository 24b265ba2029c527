"""ERS_OPT_FOUR_DELTA: the O(delta^7) variant of the extrapolation (Sec. 1) with four deltas and the
I4 column, against the oracle's four-delta path (ers_oracle.c:ora_eval_k with K = 4)."""
import numpy as np
import pytest

from parity import GpuProblem, oracle_eval, oracle_eval_sharp, rel_err

pytestmark = pytest.mark.gpu
FP64_TOL = 1e-11
MIXED_TOL = 1e-6
RHO4 = (3.0, 4.0, 5.0, 6.0)


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


@pytest.mark.parametrize("precision,tol", [(0, FP64_TOL), (1, MIXED_TOL)])
@pytest.mark.parametrize("rho", [RHO4, (2.0, 3.0, 4.0, 5.0)])
def test_four_delta_matches_oracle_sphere16(ers, precision, tol, rho):
    """Every node and band target of the h = 1/16 sphere (near radius 6 rho_3 h reaches around the sphere)."""
    y, uo, vo, _ = oracle_eval("sphere16", rho=rho)
    g = gpu("sphere16")
    u, v, _ = g.eval(g.targets(), precision=precision, rho=rho)
    eu, ev = rel_err(u, uo), rel_err(v, vo)
    assert eu <= tol and ev <= tol, (eu, ev)


@pytest.mark.parametrize("precision,tol", [(0, FP64_TOL), (1, MIXED_TOL)])
def test_four_delta_matches_oracle_sphere32(ers, precision, tol):
    """Every third target of the h = 1/32 sphere: nodes (b = 0) and the band |b| <= 0.25."""
    sel = np.arange(0, 17070 + 2000, 3)
    y, uo, vo, b = oracle_eval("sphere32", sel=sel, rho=RHO4)
    g = gpu("sphere32")
    u, v, bg = g.eval(g.targets(sel), precision=precision, rho=RHO4)
    assert np.array_equal(bg == 0, b == 0)
    eu, ev = rel_err(u, uo), rel_err(v, vo)
    assert eu <= tol and ev <= tol, (eu, ev)
    # the variant differs from the three-delta method by its O(h^5) error
    u3, v3, _ = g.eval(g.targets(sel), precision=precision, rho=RHO4[:3])
    assert 1e-9 < rel_err(u3, u) < 1e-4 and 1e-9 < rel_err(v3, v) < 1e-2


@pytest.mark.parametrize("tc", [4.3, 5.3, 7.5])
@pytest.mark.parametrize("precision,tol", [(0, FP64_TOL), (1, MIXED_TOL)])
def test_four_delta_other_cutoffs(ers, tc, precision, tol):
    """Cutoffs below DEFECT_T = 4.7 (the table path meets the cutoff) and above 6."""
    sel = np.arange(1, 17070 + 2000, 7)
    y, uo, vo, _ = oracle_eval("sphere32", sel=sel, rho=RHO4, tc=tc)
    g = gpu("sphere32")
    u, v, _ = g.eval(g.targets(sel), precision=precision, rho=RHO4, tc=tc)
    eu, ev = rel_err(u, uo), rel_err(v, vo)
    assert eu <= tol and ev <= tol, (eu, ev)


@pytest.mark.parametrize("layers", [1, 2])
def test_four_delta_single_layer_only(ers, layers):
    sel = np.arange(2, 17070 + 2000, 11)
    y, uo, vo, _ = oracle_eval("sphere32", sel=sel, rho=RHO4)
    g = gpu("sphere32")
    u, v, _ = g.eval(g.targets(sel), precision=0, rho=RHO4, layers=layers)
    if layers == 1:
        assert v is None and rel_err(u, uo) <= FP64_TOL
    else:
        assert u is None and rel_err(v, vo) <= FP64_TOL


def test_four_delta_with_sharp(ers):
    """ERS_OPT_SHARP with four deltas: on-surface targets take the s# path (independent of rho),
    the others the four-delta extrapolation."""
    sel = np.arange(0, 17070 + 2000, 5)
    _, us, vs, bs = oracle_eval_sharp("sphere32", sel=sel, rho_sharp=3.0)
    _, u4, v4, _ = oracle_eval("sphere32", sel=sel, rho=RHO4)
    on = bs == 0
    assert 0 < on.sum() < len(sel)
    uo = np.where(on[:, None], us, u4)
    vo = np.where(on[:, None], vs, v4)
    g = gpu("sphere32")
    for precision, tol in ((0, FP64_TOL), (1, MIXED_TOL)):
        u, v, _ = g.eval(g.targets(sel), precision=precision, rho=RHO4, sharp=True, rho_sharp=3.0)
        assert rel_err(u, uo) <= tol and rel_err(v, vo) <= tol, (precision, rel_err(u, uo), rel_err(v, vo))


def test_four_delta_counts(ers):
    """Pair counts: every near pair in one class of each count; the near radius is 6 rho_3 h."""
    g = gpu("sphere32")
    y = g.targets()
    g.eval(y, precision=1, rho=RHO4[:3])
    nt3, np3, _ = g.s.last_counts()
    assert len(g.s.last_class_counts()) == 3
    g.eval(y, precision=1, rho=RHO4)
    nt4, np4, nf4 = g.s.last_counts()
    cut, dfx = g.s.last_class_counts(), g.s.last_defect_class_counts()
    assert len(cut) == 4 and len(dfx) == 5
    assert sum(cut) == np4 and sum(dfx) == np4
    assert min(cut) > 0 and min(dfx) > 0
    assert np4 + nf4 == len(y) * g.s.N
    # (6/5)^2-ish more near area per target, more near targets
    assert nt4 >= nt3 and np4 > 1.3 * np3


def test_four_delta_rejected_where_unsupported(ers):
    import torch
    g = gpu("sphere16")
    y = g.targets()[:64]
    yd, x0, n0, b, f0, q0 = g.prepare(y)
    u = torch.empty((64, 3), dtype=torch.float64, device="cuda")
    v = torch.empty((64, 3), dtype=torch.float64, device="cuda")
    with pytest.raises(ers.ErsError) as ex:
        g.s.eval_noalloc(yd, x0, n0, b, f0, q0, u, v, rho=RHO4)
    assert ex.value.code == -5
    for bad in ((3.0, 4.0, 5.0, 5.0), (3.0, 4.0, 5.0, -1.0), (3.0, 4.0, 5.0, float("nan"))):
        with pytest.raises(ers.ErsError) as ex:
            g.s.eval(yd, f0, q0, rho=bad)
        assert ex.value.code == -1
    # rho4 = 0: the next of the evenly spaced set, 2 rho_2 - rho_1
    ua, va = (t.cpu().numpy() for t in g.s.eval(yd, f0, q0, rho=(3.0, 4.0, 5.0, 0.0)))
    ub, vb = (t.cpu().numpy() for t in g.s.eval(yd, f0, q0, rho=RHO4))
    assert np.array_equal(ua, ub) and np.array_equal(va, vb)


def test_four_delta_full_size_bench_workload_sampled(ers):
    """The bench workload with the four-delta option as the bench's leg runs it (rho = (2, 3, 4, 5),
    mixed precision, all 392,718 targets); a seeded sample against the oracle."""
    import workloads
    g = gpu("sphere128")
    y_all = g.targets()
    rho = (2.0, 3.0, 4.0, 5.0)
    u, v, _ = g.eval(y_all, precision=1, rho=rho)
    sel = workloads.subsample(300, len(y_all), 6262)
    y, uo, vo, _ = oracle_eval("sphere128", sel=sel, rho=rho)
    assert np.array_equal(y, y_all[sel])
    assert rel_err(u[sel], uo) <= MIXED_TOL and rel_err(v[sel], vo) <= MIXED_TOL


@pytest.mark.parametrize("precision,tol", [(0, FP64_TOL), (1, MIXED_TOL)])
def test_four_delta_ellipsoid_with_far_points(ers, precision, tol):
    """Ellipsoid (1, 0.8, 0.6) at h = 1/32 with rho = (2, 3, 4, 5): every 11th node and the band
    and box targets, against the oracle's four-delta path."""
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
    rho = (2.0, 3.0, 4.0, 5.0)
    uo, vo, _ = oracle.evaluate(x, n, w, workloads.poly_eval(wl.f_coef, x), workloads.poly_eval(wl.q_coef, x),
                                y, x0, n0, b, f0, q0, wl.h, rho)
    u, v, _ = g.eval(g.targets(sel), precision=precision, rho=rho)
    eu, ev = rel_err(u, uo), rel_err(v, vo)
    assert eu <= tol and ev <= tol, (eu, ev)
