"""The learned near-field closure: the one- and two-delta sums and the closure's features against
the oracle, tensor-core inference and training kernels against the FP64 reference network, what
the trained network gains over the sums alone, the per-layer gate, the extent check and the
fallback."""
import numpy as np
import pytest

import oracle
import workloads
from oracle import closure as ora_closure
from oracle import mlp as ref
from parity import per_target_rel_err, rel_err

pytestmark = pytest.mark.gpu
XSTR, JET_OFF, NJ = 48, 16, (18, 27)
FP64_TOL, MIXED_TOL = 1e-11, 1e-6


@pytest.fixture(scope="module")
def ers():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2507_00156_gb300
    return paper_2507_00156_gb300


def _records(n, seed, nj=NJ[1]):
    rng = np.random.default_rng(seed)
    X = np.zeros((n, XSTR), np.float32)
    X[:, :5] = rng.standard_normal((n, 5))
    X[:, JET_OFF:JET_OFF + nj] = rng.uniform(-1, 1, (n, nj))
    T = np.zeros((n, 4), np.float32)
    T[:, :3] = 0.3 * rng.standard_normal((n, 3))
    T[:, 3] = rng.uniform(0.0, 1.0, n)
    return X, T


def _random_params(ers, c, seed):
    rng = np.random.default_rng(seed)
    for layer in (0, 1):
        c.set_params(layer, (0.2 * rng.standard_normal(ers.NPARAM)).astype(np.float32))


@pytest.mark.parametrize("n", [1, 127, 1000, 4099])
def test_tensor_core_inference_matches_reference_and_oracle(ers, n):
    import torch
    c = ers.Closure(seed=3)
    _random_params(ers, c, n)
    for layer in (0, 1):
        X, _ = _records(n, n + layer, NJ[layer])
        Xd = torch.from_numpy(X).cuda()
        Ytc = c.infer(layer, Xd).cpu().numpy()
        Yref = c.infer(layer, Xd, reference=True).cpu().numpy()
        assert (Ytc[:, 3] == 0).all() and (Yref[:, 3] == 0).all()
        Ytc, Yref = Ytc[:, :3], Yref[:, :3]
        yo, _ = ref.forward(c.params(layer).astype(np.float64), X.astype(np.float64), NJ[layer], quantize=True)
        scale = np.abs(yo).max()
        d_ref, d_ora = np.abs(Ytc - Yref), np.abs(Ytc - yo)
        # same BF16 operands, FP32 sums in another order: one-ulp BF16 flips of a hidden activation
        # (192 per sample) move the coefficients, and the head sums up to 81 of them
        assert d_ref.max() <= 2e-2 * scale, (layer, d_ref.max(), scale)
        assert np.quantile(d_ref, 0.9) <= 1e-5 * scale and np.quantile(d_ref, 0.99) <= 1e-4 * scale
        assert d_ora.max() <= 2e-2 * scale and np.quantile(d_ora, 0.99) <= 2e-4 * scale
    assert not c.timed_out()


def test_untrained_network_predicts_no_correction(ers):
    import torch
    c = ers.Closure(seed=4)
    X, _ = _records(500, 1)
    for layer in (0, 1):
        assert (c.infer(layer, torch.from_numpy(X).cuda()).cpu().numpy() == 0).all()


def test_gradient_matches_fp64_reference(ers):
    import torch
    c = ers.Closure(seed=5)
    _random_params(ers, c, 5)
    for layer in (0, 1):
        X, T = _records(777, 11 + layer, NJ[layer])
        G, loss = c.grad(layer, torch.from_numpy(X).cuda(), torch.from_numpy(T).cuda())
        lo, go = ref.loss_and_grad(c.params(layer).astype(np.float64), X.astype(np.float64),
                                   T.astype(np.float64), NJ[layer], quantize=True)
        G = G.cpu().numpy().astype(np.float64)
        # rare one-ulp BF16 flips of an activation (FP32 vs FP64 GELU before rounding) move the loss slightly
        assert abs(loss - lo) <= 1e-4 * abs(lo), (loss, lo)
        assert np.linalg.norm(G - go) <= 1e-3 * np.linalg.norm(go), np.linalg.norm(G - go) / np.linalg.norm(go)
        big = np.abs(go) > 1e-3 * np.abs(go).max()
        assert np.quantile(np.abs(G - go)[big] / np.abs(go)[big], 0.95) <= 1e-3
        off_w4 = 1024 + 64 + 4096 + 64 + 4096 + 64
        assert (G[off_w4 + 3 * NJ[layer] * 64: off_w4 + 96 * 64] == 0).all()


def test_training_reduces_loss(ers):
    """A target that is linear in the jets with coefficients smooth in the geometry."""
    import torch
    c = ers.Closure(seed=7)
    rng = np.random.default_rng(3)
    n, nj = 20000, NJ[0]
    X = np.zeros((n, XSTR), np.float32)
    X[:, :5] = rng.uniform(-1, 1, (n, 5))
    X[:, JET_OFF:JET_OFF + nj] = rng.uniform(-1, 1, (n, nj))
    B = rng.standard_normal((5, 3 * nj))
    coef = np.tanh(X[:, :5] @ B / 2.0).reshape(n, 3, nj)
    T = np.zeros((n, 4), np.float32)
    T[:, :3] = np.einsum("nej,nj->ne", coef, X[:, JET_OFF:JET_OFF + nj])
    T[:, 3] = 1.0
    Xd, Td = torch.from_numpy(X).cuda(), torch.from_numpy(T).cuda()
    _, l0 = c.grad(0, Xd, Td)
    c.train(0, Xd, Td, steps=800, batch=2048, lr=3e-3)
    _, l2 = c.grad(0, Xd, Td)
    assert l2 < 0.05 * l0, (l0, l2)


# --- the one- and two-delta sums and the features against the oracle -----------------------

def _ell32():
    """Ellipsoid (1, 0.8, 0.6) at h = 1/32, band |b| <= 0.3 (inside its smallest radius of curvature
    0.36, so that every band target has one closest point)."""
    shape = workloads.Shape((0.0, 0.0, 0.0), (1.0, 0.8, 0.6))
    return workloads.make_workload("ell32", shape, 1 / 32, (2, 3, 4), 77, 1500, 0.3)


def _sphere32():
    """Unit sphere at h = 1/32, band |b| <= 18 h (the two-delta near radius) and box points."""
    return workloads.make_workload("sph32b", workloads.unit_sphere(), 1 / 32, (2, 3, 4), 78, 1500, 18 / 32,
                                   n_far=300)


def _oracle_side(wl, sel):
    x, n, w = oracle.quadrature(wl.shape, wl.h)
    f, q = workloads.poly_eval(wl.f_coef, x), workloads.poly_eval(wl.q_coef, x)
    y = np.concatenate([x, wl.extra_targets])[sel]
    x0, n0, b = oracle.closest_point(wl.shape, y)
    f0, q0 = workloads.poly_eval(wl.f_coef, x0), workloads.poly_eval(wl.q_coef, x0)
    return dict(x=x, n=n, w=w, f=f, q=q, y=y, x0=x0, n0=n0, b=b, f0=f0, q0=q0)


def _gpu_side(ers, wl, sel, precision):
    import torch
    from parity import GpuProblem
    g = GpuProblem(wl.name, wl)
    yd, x0, n0, b, f0, q0 = g.prepare(g.targets(sel))
    u3, v3 = g.s.eval(yd, f0, q0, rho=wl.rho, precision=precision, x0=x0, n0=n0, b=b)
    return g, dict(y=yd, x0=x0, n0=n0, b=b, f0=f0, q0=q0, u3=u3.clone(), v3=v3.clone())


def _selection(wl):
    N = len(oracle.quadrature(wl.shape, wl.h)[2])
    return np.concatenate([np.arange(0, N, 7), N + np.arange(len(wl.extra_targets))])


@pytest.mark.parametrize("make", [_sphere32, _ell32])
@pytest.mark.parametrize("nd", [1, 2])
def test_reduced_sums_match_oracle(ers, make, nd):
    """ers_eval_learned with a network that predicts nothing returns the one- or two-delta sums:
    element by element against the oracle's definition (every node, s_p = 1 beyond cutoff_t delta_k;
    plain sums beyond the reduced near radius) at FP64 and mixed precision."""
    wl = make()
    sel = _selection(wl)
    O = _oracle_side(wl, sel)
    uo, vo, go = oracle.evaluate_reduced(nd, O["x"], O["n"], O["w"], O["f"], O["q"], O["y"], O["x0"], O["n0"], O["b"],
                                         O["f0"], O["q0"], wl.h, wl.rho)
    zero = ers.Closure(seed=1)
    for precision, tol in ((0, FP64_TOL), (1, MIXED_TOL)):
        g, P = _gpu_side(ers, wl, sel, precision)
        assert np.abs(P["b"].cpu().numpy() - O["b"]).max() < 1e-13
        u, v, err, fb = ers.eval_learned(g.s, zero, P["y"], P["x0"], P["n0"], P["b"], P["f0"], P["q0"], rho=wl.rho,
                                         precision=precision, tol=1e30, vstride=1 << 30, ndelta=nd)
        assert not fb
        u, v = u.cpu().numpy(), v.cpu().numpy()
        assert rel_err(u, uo) <= tol and rel_err(v, vo) <= tol, (precision, rel_err(u, uo), rel_err(v, vo))
        if precision == 0:
            assert per_target_rel_err(u, uo) <= tol and per_target_rel_err(v, vo) <= tol
        # the reduced sums differ from the method by the term the closure has to supply (O(delta^3)
        # for two deltas, O(delta) for one: far above either parity bar)
        u3 = P["u3"].cpu().numpy()
        assert rel_err(u, u3) > 1e-5


@pytest.mark.parametrize("make", [_sphere32, _ell32])
@pytest.mark.parametrize("nd", [1, 2])
def test_closure_features_and_targets_match_oracle(ers, make, nd):
    """ers_closure_data: the sample records (geometry: lambda_0, principal curvatures times h, rho;
    density jets of the degree-4 least-squares fit, scaled by their largest magnitude) and the
    training targets (c in the principal frame, divided by S h^p, and the weights) against the
    oracle's features computed in numpy from the same definition, at FP32 tolerance."""
    wl = make()
    sel = _selection(wl)
    O = _oracle_side(wl, sel)
    g, P = _gpu_side(ers, wl, sel, 0)
    Xs, Xd, Ts, Td, valid = (z.cpu().numpy() for z in ers.closure_data(
        g.s, P["y"], P["x0"], P["n0"], P["b"], P["f0"], P["q0"], P["u3"], P["v3"], rho=wl.rho, precision=0,
        ndelta=nd))
    geom, frames, jets, scale = ora_closure.features(wl.shape, O["x"], O["f"], O["q"], O["x0"], O["n0"], O["b"],
                                                     wl.h, wl.rho, nd)
    u3, v3, _ = oracle.evaluate(O["x"], O["n"], O["w"], O["f"], O["q"], O["y"], O["x0"], O["n0"], O["b"], O["f0"],
                                O["q0"], wl.h, wl.rho)
    ur, vr, gm = oracle.evaluate_reduced(nd, O["x"], O["n"], O["w"], O["f"], O["q"], O["y"], O["x0"], O["n0"],
                                         O["b"], O["f0"], O["q0"], wl.h, wl.rho)
    (ts, td), (ws, wd) = ora_closure.targets(frames, scale, wl.h, nd, ur, vr, gm, u3, v3, wl.rho)
    for X in (Xs, Xd):
        np.testing.assert_allclose(X[:, :5], geom.astype(np.float32), rtol=2e-6, atol=1e-7)
        assert (X[:, 5:JET_OFF] == 0).all()
    for layer, (X, T, t, wt) in enumerate(((Xs, Ts, ts, ws), (Xd, Td, td, wd))):
        nj = NJ[layer]
        on = scale[:, layer] > 0
        assert on.sum() > 100 and (~on).sum() >= 0
        np.testing.assert_allclose(X[on, JET_OFF:JET_OFF + nj], jets[layer][on], rtol=0, atol=2e-6)
        assert (X[~on, JET_OFF:] == 0).all() and (X[:, JET_OFF + nj:] == 0).all()
        np.testing.assert_allclose(T[:, 3], wt, rtol=1e-6, atol=1e-7)
        w = wt > 0
        assert w.sum() > 100
        scale_t = np.abs(t[w]).max()
        np.testing.assert_allclose(T[w, :3], t[w], rtol=0, atol=2e-5 * scale_t)
    assert np.array_equal(valid.astype(bool), (ws > 0) | (wd > 0))


# --- training, the gate, the fallback ----------------------------------------------------------

def _problem(ers, s, fc, qc, y, precision):
    import torch
    dev = torch.device("cuda")
    yd = torch.from_numpy(np.ascontiguousarray(y)).to(dev)
    x0, n0, b = s.closest_point(yd)
    x0h = x0.cpu().numpy()
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    f0, q0 = t(workloads.poly_eval(fc, x0h)), t(workloads.poly_eval(qc, x0h))
    x = s.nodes()[0].cpu().numpy()
    s.set_density(t(workloads.poly_eval(fc, x)), t(workloads.poly_eval(qc, x)))
    u3, v3 = s.eval(yd, f0, q0, rho=(2, 3, 4), precision=precision, x0=x0, n0=n0, b=b)
    return dict(y=yd, x0=x0, n0=n0, b=b, f0=f0, q0=q0, u3=u3.clone(), v3=v3.clone())


def _args(P):
    return (P["y"], P["x0"], P["n0"], P["b"], P["f0"], P["q0"])


def _train_sphere(ers, s, x, shape, h, nd, ndens, rng, band_b, steps):
    import torch
    data = []
    for _ in range(ndens):
        fc, qc = workloads.density_coeffs(rng), workloads.density_coeffs(rng)
        band = workloads.near_band_targets(shape, 6000, band_b, rng)[0]
        P = _problem(ers, s, fc, qc, np.concatenate([x, band]), 0)
        out = ers.closure_data(s, *_args(P), P["u3"], P["v3"], precision=0, ndelta=nd)
        sel = out[4].bool()
        data.append([z[sel] for z in out[:4]])
    Xs, Xd, Ts, Td = (torch.cat([d[i] for d in data]).contiguous() for i in range(4))
    net = ers.Closure(seed=nd)
    for layer, (X, T) in enumerate(((Xs, Ts), (Xd, Td))):
        net.train(layer, X, T, steps=steps, batch=4096, lr=2e-3)
    return net


def test_learned_closure_gains_over_the_sums_alone(ers):
    """Unit sphere, h = 1/32: networks trained on six densities, evaluated on a held-out density at
    the nodes and band targets.  Against the method (three deltas): the two-delta sums with the
    network are several times closer than the same sums alone (the c2 term is linear in the jets
    the network weighs), the single sum with the network gains too; both layers keep the network in
    the gate.  With an impossible tolerance the call falls back to the method exactly."""
    shape = workloads.unit_sphere()
    h = 1 / 32
    s = ers.Surface(shape.center, shape.axes, h)
    x = s.nodes()[0].cpu().numpy()
    rng = np.random.default_rng(21)
    zero = ers.Closure(seed=9)
    for nd, band_b, gain in ((2, 18 * h, 0.3), (1, 12 * h, 0.5)):
        net = _train_sphere(ers, s, x, shape, h, nd, 6, rng, band_b, 3000)
        fc, qc = workloads.density_coeffs(rng), workloads.density_coeffs(rng)
        band = workloads.near_band_targets(shape, 3000, band_b, rng)[0]
        P = _problem(ers, s, fc, qc, np.concatenate([x, band]), 0)
        u3, v3 = P["u3"].cpu().numpy(), P["v3"].cpu().numpy()
        uL, vL, errL, fb = ers.eval_learned(s, net, *_args(P), precision=0, tol=1.0, vstride=8, ndelta=nd)
        assert not fb and not net.timed_out()
        used, ew, eo = net.last_gate()
        u0, v0, err0, _ = ers.eval_learned(s, zero, *_args(P), precision=0, tol=1.0, vstride=8, ndelta=nd)
        for layer, (a, b_, ref3) in enumerate(((uL, u0, u3), (vL, v0, v3))):
            eL = np.abs(a.cpu().numpy() - ref3)
            e0 = np.abs(b_.cpu().numpy() - ref3)
            rL, r0 = np.sqrt((eL ** 2).mean()), np.sqrt((e0 ** 2).mean())
            print(f"ndelta {nd} layer {layer}: RMS error with / without the network {rL:.3e} / {r0:.3e}, "
                  f"max {eL.max():.3e} / {e0.max():.3e}")
            assert rL < gain * r0, (nd, layer, rL, r0)
            assert eL.max() < 0.7 * e0.max(), (nd, layer, eL.max(), e0.max())
            assert used[layer] and ew[layer] < eo[layer]
            assert errL[layer] == ew[layer] and errL[layer] < err0[layer]
    # fallback: an impossible tolerance gives exactly the three-delta result
    uF, vF, _, fb = ers.eval_learned(s, net, *_args(P), precision=0, tol=1e-15, vstride=8, ndelta=1)
    assert fb
    assert np.array_equal(uF.cpu().numpy(), u3) and np.array_equal(vF.cpu().numpy(), v3)


def test_gate_takes_back_a_network_that_does_not_help(ers):
    """A network with random weights makes the two-delta sums worse on the validation sample: the
    gate takes its correction back for both layers, so the values are those of the sums alone,
    and reports the two errors."""
    shape = workloads.unit_sphere()
    h = 1 / 16
    s = ers.Surface(shape.center, shape.axes, h)
    x = s.nodes()[0].cpu().numpy()
    rng = np.random.default_rng(5)
    fc, qc = workloads.density_coeffs(rng), workloads.density_coeffs(rng)
    band = workloads.near_band_targets(shape, 2000, 6 * h, rng)[0]
    P = _problem(ers, s, fc, qc, np.concatenate([x, band]), 0)
    bad, zero = ers.Closure(seed=3), ers.Closure(seed=3)
    _random_params(ers, bad, 77)
    u0, v0, err0, _ = ers.eval_learned(s, zero, *_args(P), precision=0, tol=1.0, vstride=4, ndelta=2)
    u, v, err, fb = ers.eval_learned(s, bad, *_args(P), precision=0, tol=1.0, vstride=4, ndelta=2)
    used, ew, eo = bad.last_gate()
    assert not fb and used == (False, False)
    assert ew[0] > eo[0] and ew[1] > eo[1]
    assert err == pytest.approx(err0, rel=1e-9)
    for a, b_ in ((u, u0), (v, v0)):
        a, b_ = a.cpu().numpy(), b_.cpu().numpy()
        assert np.abs(a - b_).max() <= 1e-13 * np.abs(b_).max()


def test_feature_range_tracks_the_training_geometry(ers):
    import torch
    c = ers.Closure(seed=5)
    assert c.feature_range(0) is None and c.feature_range(1) is None
    X, T = _records(5000, 4)
    X[:, :5] = np.random.default_rng(4).uniform(-3, 2, (5000, 5))
    X[7, 2] = np.nan  # non-finite inputs are skipped
    X[9, 4] = np.inf
    c.train(0, torch.from_numpy(X).cuda(), torch.from_numpy(T).cuda(), steps=2, batch=256)
    lo, hi = c.feature_range(0)
    F = X[:, :5].astype(np.float64)
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
        F = X[:, :5]
        out |= corrected & ~((F >= lo - tol) & (F <= hi + tol)).all(1)
    return out


def rel_err_max(a, ref_):
    return float(np.abs(a - ref_).max() / np.abs(ref_).max())


def test_targets_outside_the_training_extent_take_the_method(ers):
    """A one-delta closure trained on the unit sphere at h = 1/32 with targets |b| <= 4h: evaluated
    with targets up to the near radius 12h, the targets whose geometry (here lambda_0) leaves the
    extent, as the host computes it, get the three-delta value and the others the network's; on a
    sphere of radius 0.5 (twice the curvature) every corrected target leaves it; with the check off
    the network is used."""
    import torch
    h = 1 / 32
    rng = np.random.default_rng(31)
    shape = workloads.unit_sphere()
    s = ers.Surface(shape.center, shape.axes, h)
    x = s.nodes()[0].cpu().numpy()
    net = _train_sphere(ers, s, x, shape, h, 1, 3, rng, 4 * h, 300)

    def run(surf, sh, xs, check=True):
        fc, qc = workloads.density_coeffs(rng), workloads.density_coeffs(rng)
        band = workloads.near_band_targets(sh, 2000, 12 * h, rng)[0]
        P = _problem(ers, surf, fc, qc, np.concatenate([xs, band]), 0)
        F = ers.closure_data(surf, *_args(P), P["u3"], P["v3"], precision=0, ndelta=1)
        corrected = (F[0][:, JET_OFF:].abs().sum(1) > 0).cpu().numpy() | (F[1][:, JET_OFF:].abs().sum(1) > 0).cpu().numpy()
        outside = _outside(net, F[0].cpu().numpy(), F[1].cpu().numpy(), corrected)
        net.set_range_check(check)
        u, v, _, fb = ers.eval_learned(surf, net, *_args(P), precision=0, tol=1e30, vstride=1 << 20, ndelta=1)
        assert not fb
        return (u.cpu().numpy(), v.cpu().numpy(), P["u3"].cpu().numpy(), P["v3"].cpu().numpy(), outside, corrected)

    u, v, u3, v3, outside, corr = run(s, shape, x)
    print("training surface, band to 12h: targets outside the extent", outside.sum(), "of", corr.sum())
    assert net.last_out_of_range() == outside.sum() and 0 < outside.sum() < corr.sum()
    assert rel_err_max(u[outside], u3[outside]) <= 1e-12 and rel_err_max(v[outside], v3[outside]) <= 1e-12
    inside = corr & ~outside
    assert np.abs(u[inside] - u3[inside]).max() > 1e-9 * np.abs(u3).max()
    small = workloads.Shape((0.0, 0.0, 0.0), (0.5, 0.5, 0.5))
    s2 = ers.Surface(small.center, small.axes, h)
    x2 = s2.nodes()[0].cpu().numpy()
    u, v, u3, v3, outside, corr = run(s2, small, x2)
    assert corr.sum() > 0 and (outside == corr).all() and net.last_out_of_range() == corr.sum()
    assert rel_err_max(u[corr], u3[corr]) <= 1e-12 and rel_err_max(v[corr], v3[corr]) <= 1e-12
    u, v, u3, v3, outside, corr = run(s2, small, x2, check=False)
    assert net.last_out_of_range() == 0
    assert rel_err_max(u, u3) > 1e-9


def test_curvature_features_of_an_ellipsoid(ers):
    """Inputs 1 and 2 are the principal curvatures at x0 times h (larger first): against the
    eigenvalues of the shape operator of the implicit surface sum((x/a)^2) = 1, i.e. of
    P H P / |grad F| on the tangent plane (P = I - n n), computed here in numpy."""
    h = 1 / 32
    shape = workloads.Shape((0.1, -0.2, 0.05), (1.0, 0.8, 0.6))
    s = ers.Surface(shape.center, shape.axes, h)
    rng = np.random.default_rng(12)
    y = workloads.near_band_targets(shape, 300, 2 * h, rng)[0]
    fc, qc = workloads.density_coeffs(rng), workloads.density_coeffs(rng)
    P = _problem(ers, s, fc, qc, y, 0)
    X = ers.closure_data(s, *_args(P), P["u3"], P["v3"], precision=0, ndelta=1)[0].cpu().numpy()
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
    _random_params(ers, c, 8)
    X, _ = _records(300, 5)
    Xd = torch.from_numpy(X).cuda()
    Y1, Y2 = c.infer(0, Xd), c.infer(0, Xd)
    assert torch.isfinite(Y1).all() and torch.equal(Y1, Y2)
    assert not c.timed_out()


@pytest.mark.gpu
def test_validation_reference_from_near_field_differences(ers):
    """ers_eval_learned validates against the three-delta method without its far field: the
    method's value is the closure's sums plus the difference of the near-field sums with three and
    with nd deltas, both over the three-delta near radius.  With an untrained network and every
    target validated, the reported error equals the error against the full three-delta evaluation
    to ~1e-8 (of the largest value; the remainder is the quadrature error of the subtraction
    identity at targets between the two near radii, which the two-delta sums leave unsubtracted)."""
    h = 1 / 64
    shape = workloads.unit_sphere()
    s = ers.Surface(shape.center, shape.axes, h)
    x = s.nodes()[0].cpu().numpy()
    rng = np.random.default_rng(3)
    fc, qc = workloads.density_coeffs(rng), workloads.density_coeffs(rng)
    band = workloads.near_band_targets(shape, 20000, 26 * h, rng)[0]
    for prec in (0, 1):
        P = _problem(ers, s, fc, qc, np.concatenate([x[::7], band]), prec)
        u3, v3 = P["u3"].cpu().numpy(), P["v3"].cpu().numpy()
        zero = ers.Closure(seed=0)
        for nd in (1, 2):
            u, v, err, fb = ers.eval_learned(s, zero, *_args(P), precision=prec, tol=1e30, vstride=1, ndelta=nd)
            assert not fb
            du = np.abs(u.cpu().numpy() - u3).max() / np.abs(u3).max()
            dv = np.abs(v.cpu().numpy() - v3).max() / np.abs(v3).max()
            print(f"precision {prec} ndelta {nd}: reported {err[0]:.6e} {err[1]:.6e}, direct {du:.6e} {dv:.6e}")
            assert du > 1e-6 and dv > 1e-6
            assert abs(err[0] - du) <= 1e-7 and abs(err[1] - dv) <= 1e-7


@pytest.mark.gpu
def test_closure_entry_points_reject_the_options(ers):
    """ers_closure_data and ers_eval_learned take none of the options f1-f3 (treecode, on-surface
    s#, four deltas): ERS_E_UNSUPPORTED, with nothing evaluated.  (The validation's near-field
    difference assumes the three-delta near radius for every target, which ERS_OPT_SHARP changes
    for targets on the surface.)"""
    import ctypes
    import torch
    shape = workloads.unit_sphere()
    s = ers.Surface(shape.center, shape.axes, 1 / 16)
    x = s.nodes()[0].cpu().numpy()
    rng = np.random.default_rng(8)
    P = _problem(ers, s, workloads.density_coeffs(rng), workloads.density_coeffs(rng), x[:64], 0)
    M = 64
    net = ers.Closure(seed=0)
    L = ers.lib()
    u = torch.zeros((M, 3), dtype=torch.float64, device="cuda")
    v = torch.zeros_like(u)
    X = torch.zeros((M, ers.XSTR), dtype=torch.float32, device="cuda")
    T = torch.zeros((M, 4), dtype=torch.float32, device="cuda")
    ok = torch.zeros((M,), dtype=torch.int32, device="cuda")
    ptrs = [ers._ptr(P[k]) for k in ("y", "x0", "n0", "b", "f0", "q0")]
    for kw in (dict(sharp=True), dict(rho=(2, 3, 4, 5)), dict(tree=True)):
        p = ers.params(precision=0, **kw)
        ve, fb = (ctypes.c_double * 2)(), ctypes.c_int()
        rc = L.ers_eval_learned(s.handle, net.handle, ctypes.byref(p), ptrs[0], M, *ptrs[1:], 2, ers._ptr(u),
                                ers._ptr(v), 1.0, 4, ve, ctypes.byref(fb), ers._stream(None))
        assert rc == ers.ERS_E_UNSUPPORTED, (kw, rc)
        rc = L.ers_closure_data(s.handle, ctypes.byref(p), ptrs[0], M, *ptrs[1:], ers._ptr(P["u3"]),
                                ers._ptr(P["v3"]), 2, ers._fptr(X), ers._fptr(X), ers._fptr(T), ers._fptr(T),
                                ers._fptr(ok), ers._stream(None))
        assert rc == ers.ERS_E_UNSUPPORTED, (kw, rc)
    assert not u.any() and not X.any()
