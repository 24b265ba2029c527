"""Pins of the oracle's treecode far field (Sec. 3.4, Eqs. (MAC), (particle-cluster-KITC),
(mod_weights)) against properties that fix it independently of its own code: the octree's
invariants, the defining properties of the Lagrange basis, the moments of the modified weights,
the direct evaluation it must reduce to, and its convergence."""
import numpy as np
import pytest

import oracle
import workloads
from parity import oracle_problem, oracle_targets
from sphere_exact import dl_exact, rigid, sl_exact

SPHERE = workloads.unit_sphere()
ELL = workloads.Shape((0.1, -0.2, 0.05), (1.0, 0.8, 0.6))


@pytest.fixture(scope="module")
def ell32():
    x, n, w = oracle.quadrature(ELL, 1 / 32)
    return x, n, w


@pytest.mark.parametrize("n0", [1, 37, 500, 4000])
def test_octree_invariants(ell32, n0):
    """Leaves hold at most N0 nodes and partition the nodes; every cluster is the union of its
    children, which lie in distinct octants of its box; boxes are the nodes' bounding boxes."""
    x = ell32[0]
    N = len(x)
    t = oracle.tree_info(x, n0)
    perm = t["perm"]
    assert np.array_equal(np.sort(perm), np.arange(N))
    C = len(t["rc"])
    leaves = np.where(t["nchild"] == 0)[0]
    assert t["count"][leaves].max() <= n0 or n0 == 1
    assert t["count"][leaves].sum() == N
    # leaf ranges tile [0, N)
    order = np.argsort(t["start"][leaves])
    st, ct = t["start"][leaves][order], t["count"][leaves][order]
    assert st[0] == 0 and np.array_equal(st[1:], (st + ct)[:-1]) and st[-1] + ct[-1] == N
    assert t["parent"][0] == -1 and (t["parent"][1:] >= 0).all()
    for c in range(C):
        pts = x[perm[t["start"][c]:t["start"][c] + t["count"][c]]]
        assert np.array_equal(pts.min(0), t["lo"][c]) and np.array_equal(pts.max(0), t["hi"][c])
        ext = t["hi"][c] - t["lo"][c]
        assert t["rc"][c] == pytest.approx(0.5 * np.sqrt((ext ** 2).sum()), rel=1e-15)
        kids = np.where(t["parent"] == c)[0]
        assert len(kids) == t["nchild"][c]
        if len(kids) == 0:
            assert t["count"][c] <= n0 or not (ext > 0).any()
            continue
        assert t["count"][kids].sum() == t["count"][c]
        assert (t["level"][kids] == t["level"][c] + 1).all()
        mid = 0.5 * (t["lo"][c] + t["hi"][c])
        octs = set()
        for k in kids:
            kp = x[perm[t["start"][k]:t["start"][k] + t["count"][k]]]
            upper = kp > mid
            assert (upper == upper[0]).all()  # one octant per child
            octs.add(tuple(upper[0]))
            assert t["start"][c] <= t["start"][k] and t["start"][k] + t["count"][k] <= t["start"][c] + t["count"][c]
        assert len(octs) == len(kids)


def test_octree_matches_brute_force_partition():
    """A small random point set partitioned by direct recursion on sets of indices."""
    rng = np.random.default_rng(3)
    x = rng.normal(size=(700, 3))
    n0 = 20

    def leaves(idx):
        pts = x[idx]
        lo, hi = pts.min(0), pts.max(0)
        if len(idx) <= n0 or not (hi > lo).any():
            return [frozenset(idx)]
        mid = 0.5 * (lo + hi)
        out = []
        code = (pts[:, 0] > mid[0]) * 1 + (pts[:, 1] > mid[1]) * 2 + (pts[:, 2] > mid[2]) * 4
        for o in range(8):
            sub = idx[code == o]
            if len(sub):
                out += leaves(sub)
        return out

    ref = leaves(np.arange(len(x)))
    t = oracle.tree_info(x, n0)
    got = [frozenset(t["perm"][s:s + c]) for s, c, k in zip(t["start"], t["count"], t["nchild"]) if k == 0]
    assert got == ref  # same leaves in the same (octant) order


@pytest.mark.parametrize("p", [1, 2, 5, 8, 12])
def test_lagrange_basis(p):
    """L_k(s_j) = delta_kj at the Chebyshev points of the second kind, and sum_k s_k^m L_k(x) = x^m
    for m <= p (this fixes the basis uniquely)."""
    c, hw = 0.37, 0.81
    s = c + hw * oracle.cheb_points(p)
    assert oracle.cheb_points(p)[0] == 1.0 and oracle.cheb_points(p)[p] == -1.0
    assert np.allclose(oracle.lagrange(p, c, hw, s), np.eye(p + 1), atol=1e-14)
    xs = np.concatenate([np.linspace(c - hw, c + hw, 23), [c - 1.3 * hw, c + 1.7 * hw]])
    L = oracle.lagrange(p, c, hw, xs)
    scale = np.abs(L).sum(1)  # Lebesgue function: O(log p) inside, large outside the interval
    for m in range(p + 1):
        z = (s - c) / hw
        assert (np.abs(L @ z ** m - ((xs - c) / hw) ** m) <= 1e-14 * scale + 1e-14).all(), m
    if p >= 1:  # and not for degree p + 1
        z = (s - c) / hw
        assert not np.allclose(L @ z ** (p + 1), ((xs - c) / hw) ** (p + 1), atol=1e-6)


def test_lagrange_degenerate_interval():
    """An interval of zero width: the node equals every point, L = e_0."""
    L = oracle.lagrange(6, 0.25, 0.0, [0.25])
    assert np.array_equal(L[0], np.eye(7)[0])


@pytest.mark.parametrize("p", [3, 5])
def test_modified_weights_moments(ell32, p):
    """Eq. (mod_weights): for every cluster, the weights reproduce all tensor moments of degree
    <= p in each coordinate of the 15 densities (f w, n w, q_j n_k w), which determine them
    uniquely; the moments are formed from the nodes directly."""
    x, n, w = ell32
    rng = np.random.default_rng(11)
    f, q = rng.normal(size=x.shape), rng.normal(size=x.shape)
    n0 = 2500
    W = oracle.tree_weights(x, n, w, f, q, n0, p)
    t = oracle.tree_info(x, n0)
    assert W.shape == (len(t["rc"]), (p + 1) ** 3, 15)
    g = np.concatenate([f * w[:, None], n * w[:, None], (q[:, :, None] * n[:, None, :]).reshape(-1, 9) * w[:, None]],
                       axis=1)
    z = oracle.cheb_points(p)
    K = np.array([(a, b, c) for a in range(p + 1) for b in range(p + 1) for c in range(p + 1)])
    for cl in range(len(t["rc"])):
        idx = t["perm"][t["start"][cl]:t["start"][cl] + t["count"][cl]]
        cen = 0.5 * (t["lo"][cl] + t["hi"][cl])
        hw = 0.5 * (t["hi"][cl] - t["lo"][cl])
        xr = (x[idx] - cen) / np.where(hw > 0, hw, 1.0)
        sk = z[K]  # (NK, 3) normalized Chebyshev points
        for al in [(0, 0, 0), (1, 0, 0), (0, 1, 0), (0, 0, 1), (p, 0, 0), (0, p, 1), (2, 1, p), (p, p, p)]:
            mom_nodes = (np.prod(xr ** np.array(al), axis=1)[:, None] * g[idx]).sum(0)
            mom_w = (np.prod(sk ** np.array(al), axis=1)[:, None] * W[cl]).sum(0)
            scale = np.abs(g[idx]).sum(0)
            assert np.allclose(mom_w, mom_nodes, rtol=0, atol=1e-12 * scale.max()), (cl, al)


def _problem(name, step):
    wl, x, n, w, f, q = oracle_problem(name)
    y = oracle_targets(wl, x)[::step]
    x0, n0, b = oracle.closest_point(wl.shape, y)
    f0 = workloads.poly_eval(wl.f_coef, x0)
    q0 = workloads.poly_eval(wl.q_coef, x0)
    return wl, (x, n, w, f, q, y, x0, n0, b, f0, q0)


def test_theta_zero_is_the_direct_evaluation():
    """With theta -> 0 no cluster meets the MAC: every pair is summed directly in the leaves, and
    the result is the localized evaluation of ora_eval_k up to the order of summation."""
    wl, a = _problem("sphere16", 3)
    ud, vd, _ = oracle.evaluate(*a, wl.h, wl.rho)
    ut, vt, nf, st = oracle.evaluate_tree(*a, wl.h, wl.rho, theta=1e-9, n0_leaf=300, p=4, stats=True)
    assert nf == 0 and (st[:, 0] == 0).all()
    assert np.abs(ut - ud).max() <= 1e-13 * np.abs(ud).max()
    assert np.abs(vt - vd).max() <= 1e-13 * np.abs(vd).max()


@pytest.mark.parametrize("rho", [(2.0, 3.0, 4.0), (3.0, 4.0, 5.0, 6.0)])
def test_every_node_counted_once(rho):
    """Per target: nodes in approximated clusters + far pairs summed directly + near pairs = N, and
    the near pairs are exactly the nodes within Rc = 6 delta_K."""
    wl, a = _problem("sphere32", 29)
    x, y, b = a[0], a[5], a[8]
    _, _, nf, st = oracle.evaluate_tree(*a, wl.h, rho, theta=0.6, n0_leaf=1000, p=4, stats=True)
    assert nf == 0
    assert np.array_equal(st[:, 1] + st[:, 2] + st[:, 3], np.full(len(y), len(x)))
    Rc = 6.0 * rho[-1] * wl.h
    r = np.sqrt(((y[:, None, :] - x[None, :, :]) ** 2).sum(-1))
    near = (r <= Rc).sum(1)
    sub = np.abs(b) <= Rc
    assert np.array_equal(st[sub, 3], near[sub]) and (st[~sub, 3] == 0).all()
    assert st[:, 0].mean() > 5  # the MAC is met for many clusters


def test_error_decays_spectrally_with_degree():
    """The treecode error against the direct sums falls by orders of magnitude as p grows
    (barycentric interpolation at Chebyshev points), and a smaller theta gives a smaller error."""
    wl, a = _problem("sphere32", 7)
    ud, vd, _ = oracle.evaluate(*a, wl.h, wl.rho)
    err = {}
    for theta, p in [(0.6, 2), (0.6, 4), (0.6, 6), (0.6, 8), (0.4, 4)]:
        ut, vt, nf = oracle.evaluate_tree(*a, wl.h, wl.rho, theta=theta, n0_leaf=1000, p=p)
        assert nf == 0
        err[theta, p] = max(np.abs(ut - ud).max() / np.abs(ud).max(), np.abs(vt - vd).max() / np.abs(vd).max())
    e = [err[0.6, p] for p in (2, 4, 6, 8)]
    assert all(e[i + 1] < e[i] / 5 for i in range(3)), e
    assert e[3] < 1e-6 and e[0] > 1e-4, e
    assert err[0.4, 4] < err[0.6, 4] / 3, err


def test_treecode_keeps_the_method_accurate():
    """Near-band targets on the unit sphere with the rigid-body densities (closed forms), h = 1/64,
    theta = 0.6, N0 = 2000: the treecode's difference from the direct sums falls spectrally with p
    (about 20x per step of 2), and at p = 10 (the degree Table 2 uses one level finer) the error
    of the method against the exact values is the direct method's."""
    h = 1 / 64
    x, n, w = oracle.quadrature(SPHERE, h)
    y, _, _, _ = workloads.near_band_targets(SPHERE, 200, 4 * h, np.random.default_rng(5))
    x0, n0, b = oracle.closest_point(SPHERE, y)
    args = (x, n, w, rigid(x), rigid(x), y, x0, n0, b, rigid(x0), rigid(x0))
    ud, vd, _ = oracle.evaluate(*args, h, (3.0, 4.0, 5.0))
    eu_d, ev_d = np.abs(ud - sl_exact(y)).max(), np.abs(vd - dl_exact(y, b)).max()
    diffs = []
    for p in (6, 8, 10):
        ut, vt, nf = oracle.evaluate_tree(*args, h, (3.0, 4.0, 5.0), theta=0.6, n0_leaf=2000, p=p)
        assert nf == 0
        diffs.append((np.abs(ut - ud).max(), np.abs(vt - vd).max()))
    assert all(diffs[i + 1][0] < diffs[i][0] / 8 and diffs[i + 1][1] < diffs[i][1] / 8 for i in range(2)), diffs
    eu_t, ev_t = np.abs(ut - sl_exact(y)).max(), np.abs(vt - dl_exact(y, b)).max()
    assert eu_t < 1.5 * eu_d + 2e-10 and ev_t < 1.05 * ev_d, (eu_d, eu_t, ev_d, ev_t)
