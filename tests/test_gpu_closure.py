"""The learned near-field closure: tensor-core inference, training kernels, gradients against the
FP64 reference network, and what the trained network gains over the two-delta sums alone."""
import numpy as np
import pytest

import workloads
from oracle import mlp as ref

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ers():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2507_00156_gb300
    return paper_2507_00156_gb300


def _rand_inputs(n, seed):
    rng = np.random.default_rng(seed)
    X = rng.standard_normal((n, 16)).astype(np.float32)
    X[:, 13:] = 0.0
    T = (0.3 * rng.standard_normal((n, 4))).astype(np.float32)
    T[:, 3] = 0.0
    return X, T


@pytest.mark.parametrize("n", [1, 127, 1000, 4099])
def test_tensor_core_inference_matches_reference_and_oracle(ers, n):
    import torch
    c = ers.Closure(seed=3)
    X, _ = _rand_inputs(n, n)
    Xd = torch.from_numpy(X).cuda()
    for layer in (0, 1):
        Ytc = c.infer(layer, Xd).cpu().numpy()[:, :3]
        Yref = c.infer(layer, Xd, reference=True).cpu().numpy()[:, :3]
        yo, _ = ref.forward(c.params(layer).astype(np.float64), X.astype(np.float64), quantize=True)
        scale = np.abs(yo).max()
        d_ref = np.abs(Ytc - Yref)
        d_ora = np.abs(Ytc - yo)
        # same BF16 operands, FP32 sums in another order: rare one-ulp BF16 flips of an activation
        assert d_ref.max() <= 2e-2 * scale, (layer, d_ref.max(), scale, Ytc[:2], Yref[:2])
        assert np.quantile(d_ref, 0.99) <= 1e-5 * scale
        assert d_ora.max() <= 2e-2 * scale and np.quantile(d_ora, 0.99) <= 1e-4 * scale
    assert not c.timed_out()


def test_gradient_matches_fp64_reference(ers):
    import torch
    c = ers.Closure(seed=5)
    X, T = _rand_inputs(777, 11)
    for layer in (0, 1):
        G, loss = c.grad(layer, torch.from_numpy(X).cuda(), torch.from_numpy(T).cuda())
        lo, go = ref.loss_and_grad(c.params(layer).astype(np.float64), X.astype(np.float64),
                                   T.astype(np.float64), quantize=True)
        G = G.cpu().numpy().astype(np.float64)
        # rare one-ulp BF16 flips of an activation (FP32 vs FP64 GELU before rounding) move the loss slightly
        assert abs(loss - lo) <= 1e-4 * abs(lo), (loss, lo)
        assert np.linalg.norm(G - go) <= 1e-3 * np.linalg.norm(go), np.linalg.norm(G - go) / np.linalg.norm(go)
        big = np.abs(go) > 1e-3 * np.abs(go).max()
        assert np.quantile(np.abs(G - go)[big] / np.abs(go)[big], 0.95) <= 1e-3


def test_training_reduces_loss(ers):
    import torch
    c = ers.Closure(seed=7)
    rng = np.random.default_rng(3)
    X = rng.uniform(-1, 1, (20000, 16)).astype(np.float32)
    X[:, 13:] = 0.0
    A = rng.standard_normal((13, 3))
    T = np.zeros((20000, 4), np.float32)
    T[:, :3] = np.tanh(X[:, :13] @ A / 3.0)
    Xd, Td = torch.from_numpy(X).cuda(), torch.from_numpy(T).cuda()
    _, l0 = c.grad(0, Xd, Td)
    l1 = c.train(0, Xd, Td, steps=600, batch=2048, lr=3e-3)
    _, l2 = c.grad(0, Xd, Td)
    assert l2 < 0.05 * l0, (l0, l1, l2)


def _problem(ers, s, wl_shape, fc, qc, y, precision):
    import torch
    dev = torch.device("cuda")
    yd = torch.from_numpy(np.ascontiguousarray(y)).to(dev)
    x0, n0, b = s.closest_point(yd)
    x0h = x0.cpu().numpy()
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    f0, q0 = t(workloads.poly_eval(fc, x0h)), t(workloads.poly_eval(qc, x0h))
    gf0, gq0 = t(workloads.poly_jacobian(fc, x0h)), t(workloads.poly_jacobian(qc, x0h))
    x = s.nodes()[0].cpu().numpy()
    s.set_density(t(workloads.poly_eval(fc, x)), t(workloads.poly_eval(qc, x)))
    u3, v3 = s.eval(yd, f0, q0, rho=(2, 3, 4), precision=precision, x0=x0, n0=n0, b=b)
    return dict(y=yd, x0=x0, n0=n0, b=b, f0=f0, q0=q0, gf0=gf0, gq0=gq0, u3=u3.clone(), v3=v3.clone())


def test_learned_closure_gains_over_the_single_delta_sum_and_falls_back(ers):
    """One regularized sum (delta_0) + the network against the same sum alone, both compared with the
    method (three deltas) on a held-out density; then the fallback path."""
    import torch
    shape = workloads.unit_sphere()
    h = 1 / 32
    s = ers.Surface(shape.center, shape.axes, h)
    x = s.nodes()[0].cpu().numpy()
    rng = np.random.default_rng(21)
    data = {1: [], 2: []}
    for k in range(6):
        fc, qc = workloads.density_coeffs(rng), workloads.density_coeffs(rng)
        band = workloads.near_band_targets(shape, 6000, 4 * h, rng)[0]
        P = _problem(ers, s, shape, fc, qc, np.concatenate([x, band]), 0)
        for nd in (1, 2):
            out = ers.closure_data(s, P["y"], P["x0"], P["n0"], P["b"], P["f0"], P["q0"], P["gf0"], P["gq0"],
                                   P["u3"], P["v3"], precision=0, ndelta=nd)
            sel = out[4].bool()
            data[nd].append([z[sel] for z in out[:4]])
    nets, zero = {}, ers.Closure(seed=2)
    for layer in (0, 1):
        zero.set_params(layer, np.zeros(ers.NPARAM, np.float32))
    for nd in (1, 2):
        Xs, Xd, Ts, Td = (torch.cat([d[i] for d in data[nd]]).contiguous() for i in range(4))
        nets[nd] = ers.Closure(seed=nd)
        for layer, (X, T) in enumerate(((Xs, Ts), (Xd, Td))):
            nets[nd].train(layer, X, T, steps=3000, batch=4096, lr=2e-3)
    # held-out density and targets
    fc, qc = workloads.density_coeffs(rng), workloads.density_coeffs(rng)
    band = workloads.near_band_targets(shape, 3000, 4 * h, rng)[0]
    P = _problem(ers, s, shape, fc, qc, np.concatenate([x, band]), 0)
    args = (P["y"], P["x0"], P["n0"], P["b"], P["f0"], P["q0"], P["gf0"], P["gq0"])
    u3, v3 = P["u3"].cpu().numpy(), P["v3"].cpu().numpy()
    uL, vL, errL, fb = ers.eval_learned(s, nets[1], *args, precision=0, tol=1.0, vstride=8, ndelta=1)
    assert not fb and not nets[1].timed_out()
    u1, v1, err1, _ = ers.eval_learned(s, zero, *args, precision=0, tol=1.0, vstride=8, ndelta=1)
    for (a, b_, ref3) in ((uL, u1, u3), (vL, v1, v3)):
        eL = np.abs(a.cpu().numpy() - ref3)
        e1 = np.abs(b_.cpu().numpy() - ref3)
        rL, r1 = np.sqrt((eL ** 2).mean()), np.sqrt((e1 ** 2).mean())
        assert rL < 0.2 * r1, (rL, r1)
        assert eL.max() < 0.5 * e1.max(), (eL.max(), e1.max())
    assert errL[0] < err1[0] and errL[1] < err1[1]
    # two deltas: the network predicts the c2 term of the two-delta combination.  c2 carries
    # quadrature error that local features do not determine, and at h = 1/32 the prediction gains
    # nothing (single layer RMS error 2.25e-4 with the network, 2.18e-4 without); it must not do
    # worse than the combination alone by more than that.
    u2, v2, err2, fb2 = ers.eval_learned(s, nets[2], *args, precision=0, tol=1.0, vstride=8, ndelta=2)
    assert np.isfinite(u2.cpu().numpy()).all() and np.isfinite(v2.cpu().numpy()).all() and not fb2
    u20, v20, err20, _ = ers.eval_learned(s, zero, *args, precision=0, tol=1.0, vstride=8, ndelta=2)
    for (a, b_, ref3) in ((u2, u20, u3), (v2, v20, v3)):
        rL = np.sqrt(((a.cpu().numpy() - ref3) ** 2).mean())
        r0 = np.sqrt(((b_.cpu().numpy() - ref3) ** 2).mean())
        print("two-delta RMS error with / without the network:", rL, r0)
        assert rL < 1.25 * r0, (rL, r0)
    # fallback: an impossible tolerance gives exactly the three-delta result
    uF, vF, _, fb = ers.eval_learned(s, nets[1], *args, precision=0, tol=1e-15, vstride=8, ndelta=1)
    assert fb
    assert np.array_equal(uF.cpu().numpy(), u3) and np.array_equal(vF.cpu().numpy(), v3)


def test_feature_range_tracks_the_training_features(ers):
    import torch
    c = ers.Closure(seed=5)
    assert c.feature_range(0) is None and c.feature_range(1) is None
    rng = np.random.default_rng(4)
    X = rng.uniform(-3, 2, (5000, 16)).astype(np.float32)
    X[:, 13:] = 0.0
    X[7, 2] = np.nan  # non-finite features are skipped
    X[9, 5] = np.inf
    T = np.zeros((5000, 4), np.float32)
    c.train(0, torch.from_numpy(X).cuda(), torch.from_numpy(T).cuda(), steps=2, batch=256)
    lo, hi = c.feature_range(0)
    F = X[:, :13].astype(np.float64)
    F[~np.isfinite(F)] = np.nan
    assert np.array_equal(lo, np.nanmin(F, 0).astype(np.float32))
    assert np.array_equal(hi, np.nanmax(F, 0).astype(np.float32))
    assert c.feature_range(1) is None
    # training again widens the extent
    X2 = X.copy()
    X2[0, 0] = 50.0
    c.train(0, torch.from_numpy(X2).cuda(), torch.from_numpy(T).cuda(), steps=1, batch=256)
    lo2, hi2 = c.feature_range(0)
    assert hi2[0] == 50.0 and np.array_equal(lo2, lo) and np.array_equal(hi2[1:], hi[1:])
    c.set_feature_range(1, lo - 1, hi + 1)
    lo1, hi1 = c.feature_range(1)
    assert np.array_equal(lo1, lo - 1) and np.array_equal(hi1, hi + 1)
    with pytest.raises(ers.ErsError):
        c.set_feature_range(1, hi + 1, lo)


def _outside(net, Xs, Xd, corrected):
    """The extent check of ers_eval_learned repeated on the host in the same FP32 roundings."""
    out = np.zeros(len(Xs), bool)
    f32 = np.float32
    for layer, X in ((0, Xs), (1, Xd)):
        lo, hi = net.feature_range(layer)
        tol = (f32(0.05) * (hi - lo) + f32(1e-3) * np.maximum(np.abs(lo), np.abs(hi))) + f32(1e-6)
        F = X[:, :13]
        out |= corrected & ~((F >= lo - tol) & (F <= hi + tol)).all(1)
    return out


def test_targets_outside_the_training_extent_take_the_method(ers):
    """A closure trained on the unit sphere at h = 1/32: on the training surface with a held-out
    density the targets whose features leave the extent (as the host computes it) get the
    three-delta value and the others the network's; on a sphere of radius 0.5 (twice the
    curvature) every corrected target leaves it; with the check off the network is used."""
    import torch
    h = 1 / 32
    rng = np.random.default_rng(31)
    shape = workloads.unit_sphere()
    s = ers.Surface(shape.center, shape.axes, h)
    x = s.nodes()[0].cpu().numpy()
    net = ers.Closure(seed=3)
    data = []
    for _ in range(4):
        fc, qc = workloads.density_coeffs(rng), workloads.density_coeffs(rng)
        band = workloads.near_band_targets(shape, 4000, 4 * h, rng)[0]
        P = _problem(ers, s, shape, fc, qc, np.concatenate([x, band]), 0)
        out = ers.closure_data(s, P["y"], P["x0"], P["n0"], P["b"], P["f0"], P["q0"], P["gf0"], P["gq0"],
                               P["u3"], P["v3"], precision=0, ndelta=1)
        sel = out[4].bool()
        data.append([z[sel] for z in out[:4]])
    Xs, Xd, Ts, Td = (torch.cat([d[i] for d in data]).contiguous() for i in range(4))
    net.train(0, Xs, Ts, steps=300, batch=2048, lr=2e-3)
    net.train(1, Xd, Td, steps=300, batch=2048, lr=2e-3)

    def run(surf, sh, xs, check=True):
        fc, qc = workloads.density_coeffs(rng), workloads.density_coeffs(rng)
        band = workloads.near_band_targets(sh, 2000, 4 * h, rng)[0]
        P = _problem(ers, surf, sh, fc, qc, np.concatenate([xs, band]), 0)
        args = (P["y"], P["x0"], P["n0"], P["b"], P["f0"], P["q0"], P["gf0"], P["gq0"])
        F = ers.closure_data(surf, *args, P["u3"], P["v3"], precision=0, ndelta=1)
        outside = _outside(net, F[0].cpu().numpy(), F[1].cpu().numpy(), F[4].cpu().numpy().astype(bool))
        net.set_range_check(check)
        u, v, _, fb = ers.eval_learned(surf, net, *args, precision=0, tol=1e30, vstride=1 << 20, ndelta=1)
        assert not fb
        return (u.cpu().numpy(), v.cpu().numpy(), P["u3"].cpu().numpy(), P["v3"].cpu().numpy(), outside,
                F[4].cpu().numpy().astype(bool))

    # the training surface, a held-out density: some targets leave the extent of the density
    # features, most do not
    u, v, u3, v3, outside, corr = run(s, shape, x)
    print("held-out density: targets outside the extent", outside.sum(), "of", corr.sum())
    assert net.last_out_of_range() == outside.sum() < corr.sum()
    if outside.any():
        assert rel_err_max(u[outside], u3[outside]) <= 1e-12 and rel_err_max(v[outside], v3[outside]) <= 1e-12
    inside = corr & ~outside
    assert np.abs(u[inside] - u3[inside]).max() > 1e-9 * np.abs(u3).max()
    # a sphere of radius 0.5: every target (within 4h of it) is corrected and leaves the extent
    small = workloads.Shape((0.0, 0.0, 0.0), (0.5, 0.5, 0.5))
    s2 = ers.Surface(small.center, small.axes, h)
    x2 = s2.nodes()[0].cpu().numpy()
    u, v, u3, v3, outside, corr = run(s2, small, x2)
    assert corr.all() and outside.all() and net.last_out_of_range() == len(u)
    assert rel_err_max(u, u3) <= 1e-12 and rel_err_max(v, v3) <= 1e-12
    # with the check off the network is used everywhere
    u, v, u3, v3, outside, corr = run(s2, small, x2, check=False)
    assert net.last_out_of_range() == 0
    assert rel_err_max(u, u3) > 1e-9


def rel_err_max(a, ref):
    return float(np.abs(a - ref).max() / np.abs(ref).max())


def test_curvature_features_of_an_ellipsoid(ers):
    """Features 1 and 2 are the principal curvatures at x0 times h (larger first): against the
    eigenvalues of the shape operator of the implicit surface sum((x/a)^2) = 1, i.e. of
    P H P / |grad F| on the tangent plane (P = I - n n), computed here in numpy."""
    import torch
    h = 1 / 32
    shape = workloads.Shape((0.1, -0.2, 0.05), (1.0, 0.8, 0.6))
    s = ers.Surface(shape.center, shape.axes, h)
    rng = np.random.default_rng(12)
    y = workloads.near_band_targets(shape, 300, 2 * h, rng)[0]
    fc, qc = workloads.density_coeffs(rng), workloads.density_coeffs(rng)
    P = _problem(ers, s, shape, fc, qc, y, 0)
    X = ers.closure_data(s, P["y"], P["x0"], P["n0"], P["b"], P["f0"], P["q0"], P["gf0"], P["gq0"], P["u3"],
                         P["v3"], precision=0, ndelta=1)[0].cpu().numpy()
    x0 = P["x0"].cpu().numpy() - np.asarray(shape.center)
    a2 = np.asarray(shape.axes) ** 2
    for i in range(len(y)):
        g = 2 * x0[i] / a2
        n = g / np.linalg.norm(g)
        Pm = np.eye(3) - np.outer(n, n)
        W = Pm @ np.diag(2 / a2) @ Pm / np.linalg.norm(g)
        k = np.sort(np.linalg.eigvalsh(W))[::-1][:2]  # the third eigenvalue is 0 (normal direction)
        assert np.allclose(X[i, 1:3], (k * h).astype(np.float32), rtol=2e-6, atol=1e-9), (i, X[i, 1:3], k * h)


def test_bounded_wait_runs_out_and_reports_it(ers):
    """The timeout path of the bounded mbarrier waits (tensor-core inference, treecode staging):
    a wait that nothing completes gives up after its poll limit and reports it through a flag the
    host reads; the context stays usable (inference afterwards runs and repeats bit for bit)."""
    import ctypes
    import torch
    L = ers.lib()
    L.ers_debug_wait_timeout.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_int)]
    flag = ctypes.c_int(-1)
    ers.check(L.ers_debug_wait_timeout(0, 20000, ctypes.byref(flag)))
    assert flag.value == 1
    ers.check(L.ers_debug_wait_timeout(1, 20000, ctypes.byref(flag)))
    assert flag.value == 0
    c = ers.Closure(seed=1)
    X, _ = _rand_inputs(300, 5)
    Xd = torch.from_numpy(X).cuda()
    Y1, Y2 = c.infer(0, Xd), c.infer(0, Xd)
    assert torch.isfinite(Y1).all() and torch.equal(Y1, Y2)
    assert not c.timed_out()
