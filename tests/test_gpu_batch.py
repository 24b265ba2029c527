"""The batched persistent evaluation (ers_batch_*): several surfaces, several right-hand sides,
one graph-captured launch.  Each (problem, density) result must equal the single-density
ers_eval result of the same precision, and a sample must match the FP64 oracle."""
import numpy as np
import pytest

import oracle
import workloads
from parity import rel_err

pytestmark = pytest.mark.gpu
MIXED_TOL = 1e-6


@pytest.fixture(scope="module")
def ers():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2507_00156_gb300
    return paper_2507_00156_gb300


def _surface(ers, shape, h, nrhs, seed):
    import torch
    s = ers.Surface(shape.center, shape.axes, h)
    x = s.nodes()[0].cpu().numpy()
    rng = np.random.default_rng(seed)
    fc = [workloads.density_coeffs(rng) for _ in range(nrhs)]
    qc = [workloads.density_coeffs(rng) for _ in range(nrhs)]
    f = np.stack([workloads.poly_eval(c, x) for c in fc])
    q = np.stack([workloads.poly_eval(c, x) for c in qc])
    s.set_density_multi(torch.from_numpy(f).cuda(), torch.from_numpy(q).cuda())
    return s, x, fc, qc


def _problem(s, y, fc, qc):
    import torch
    yd = torch.from_numpy(np.ascontiguousarray(y)).cuda()
    x0, n0, b = s.closest_point(yd)
    x0h = x0.cpu().numpy()
    f0 = torch.from_numpy(np.stack([workloads.poly_eval(c, x0h) for c in fc])).cuda()
    q0 = torch.from_numpy(np.stack([workloads.poly_eval(c, x0h) for c in qc])).cuda()
    nr, M = len(fc), len(y)
    u = torch.full((nr, M, 3), float("nan"), dtype=torch.float64, device="cuda")
    v = torch.full((nr, M, 3), float("nan"), dtype=torch.float64, device="cuda")
    return dict(s=s, y=yd, x0=x0, n0=n0, b=b, f0=f0.contiguous(), q0=q0.contiguous(), u=u, v=v, fc=fc, qc=qc)


def _single(ers, pr, r):
    """The same problem and density r through ers_eval (mixed precision)."""
    import torch
    s = pr["s"]
    x = s.nodes()[0].cpu().numpy()
    s.set_density(torch.from_numpy(workloads.poly_eval(pr["fc"][r], x)).cuda(),
                  torch.from_numpy(workloads.poly_eval(pr["qc"][r], x)).cuda())
    u, v = s.eval(pr["y"], pr["f0"][r].contiguous(), pr["q0"][r].contiguous(), rho=(2, 3, 4), precision=1,
                  x0=pr["x0"], n0=pr["n0"], b=pr["b"])
    torch.cuda.synchronize()
    return u.cpu().numpy(), v.cpu().numpy()


@pytest.mark.parametrize("nrhs", [1, 2, 4, 8])
def test_two_spheres_and_bodies_match_single_evaluations(ers, nrhs):
    import torch
    h = 1 / 16
    gap = 0.05
    A = workloads.unit_sphere((0.0, 0.0, 0.0))
    B = workloads.unit_sphere((2.0 + gap, 0.0, 0.0))
    C = workloads.Shape((0.0, 5.0, 0.0), (0.9, 0.7, 0.6))
    sA, xA, fA, qA = _surface(ers, A, h, nrhs, 1)
    sB, xB, fB, qB = _surface(ers, B, h, nrhs, 2)
    sC, xC, fC, qC = _surface(ers, C, 1 / 24, nrhs, 3)
    yAB = np.concatenate([xA, xB])
    yC = np.concatenate([xC, workloads.near_band_targets(C, 300, 0.1, np.random.default_rng(4))[0]])
    probs = [_problem(sA, yAB, fA, qA), _problem(sB, yAB, fB, qB), _problem(sC, yC, fC, qC)]
    batch = ers.Batch(probs, nrhs, rho=(2, 3, 4))
    nitems, grid = batch.info()
    assert nitems == 2 * ((len(yAB) + 127) // 128) + (len(yC) + 127) // 128
    for rep in range(2):  # the graph is replayed; results must not depend on the replay
        for pr in probs:
            pr["u"].fill_(float("nan"))
            pr["v"].fill_(float("nan"))
        batch.launch()
        torch.cuda.synchronize()
        for pr in probs:
            ub, vb = pr["u"].cpu().numpy(), pr["v"].cpu().numpy()
            assert np.isfinite(ub).all() and np.isfinite(vb).all()
            if rep == 0:
                for r in range(nrhs):
                    us, vs = _single(ers, pr, r)
                    assert rel_err(ub[r], us) <= MIXED_TOL and rel_err(vb[r], vs) <= MIXED_TOL, (r, rel_err(ub[r], us))
    # the oracle on a sample of the gap problem (targets of B near A), last density
    pr = probs[0]
    sel = np.concatenate([np.arange(len(xA), len(yAB), 13), np.arange(0, len(xA), 29)])
    y = yAB[sel]
    xo, no, wo = oracle.quadrature(A, h)
    r = nrhs - 1
    x0, n0, b = oracle.closest_point(A, y)
    uo, vo, _ = oracle.evaluate(xo, no, wo, workloads.poly_eval(fA[r], xo), workloads.poly_eval(qA[r], xo), y, x0, n0,
                                b, workloads.poly_eval(fA[r], x0), workloads.poly_eval(qA[r], x0), h, (2, 3, 4))
    ub, vb = pr["u"].cpu().numpy()[r][sel], pr["v"].cpu().numpy()[r][sel]
    assert rel_err(ub, uo) <= MIXED_TOL and rel_err(vb, vo) <= MIXED_TOL


def test_batch_rejects_bad_plans(ers):
    import torch
    s, x, fc, qc = _surface(ers, workloads.unit_sphere(), 1 / 8, 2, 7)
    pr = _problem(s, x[:10], fc, qc)
    with pytest.raises(ers.ErsError) as e:
        ers.Batch([pr], 4)  # densities were set for 2 right-hand sides
    assert e.value.code == ers.ERS_E_STATE
    with pytest.raises(ers.ErsError):
        ers.Batch([pr], 3)
    p = ers.params(precision=ers.PREC_FP64)
    import ctypes
    arr = (ers._Problem * 1)()
    h = ctypes.c_void_p()
    assert ers.lib().ers_batch_create(arr, 1, ctypes.byref(p), 2, ctypes.byref(h)) == ers.ERS_E_UNSUPPORTED


@pytest.mark.parametrize("gap,n_bodies", [(0.1, 0), (0.05, 0), (0.01, 16)])
def test_batched_full_size_sampled(ers, gap, n_bodies):
    """The batched workload at full size, as the benchmark launches it: two unit spheres `gap`
    apart at h = 1/96 (about 153,000 nodes each), each evaluated at the nodes of both, 8
    densities per surface, and for gap 0.01 the 16 uneven bodies as well; seeded samples of
    (problem, density, target) against the FP64 oracle, most of them in the gap region."""
    import torch
    nrhs = 8
    pair, bodies = workloads.batched_config(gap=gap, nrhs=nrhs, n_bodies=n_bodies)
    rng = np.random.default_rng(int(gap * 1000) + 7)

    def surface(body):
        s = ers.Surface(body.shape.center, body.shape.axes, body.h)
        x = s.nodes()[0].cpu().numpy()
        f = np.stack([workloads.poly_eval(c, x) for c in body.f_coefs])
        q = np.stack([workloads.poly_eval(c, x) for c in body.q_coefs])
        s.set_density_multi(torch.from_numpy(f).cuda(), torch.from_numpy(q).cuda())
        return s, x

    (sA, xA), (sB, xB) = surface(pair[0]), surface(pair[1])
    yAB = np.concatenate([xA, xB])
    probs = [_problem(sA, yAB, pair[0].f_coefs, pair[0].q_coefs), _problem(sB, yAB, pair[1].f_coefs, pair[1].q_coefs)]
    shapes = [(pair[0], yAB), (pair[1], yAB)]
    for i, body in enumerate(bodies):
        s, x = surface(body)
        band = workloads.near_band_targets(body.shape, max(1, len(x) // 20), 4 * body.h,
                                           np.random.default_rng(2000 + i))[0]
        y = np.concatenate([x, band])
        probs.append(_problem(s, y, body.f_coefs, body.q_coefs))
        shapes.append((body, y))
    batch = ers.Batch(probs, nrhs, rho=(2, 3, 4))
    batch.launch()
    torch.cuda.synchronize()
    nA = len(xA)
    # A's integral at B's nodes that face A, B's at A's nodes that face B, and random targets
    gapA = nA + np.flatnonzero(xB[:, 0] < pair[1].shape.center[0] - 0.8)
    gapB = np.flatnonzero(xA[:, 0] > 0.8)
    checks = [(0, np.concatenate([rng.choice(gapA, 40, replace=False), rng.choice(len(yAB), 20, replace=False)]), 0),
              (0, rng.choice(gapA, 30, replace=False), nrhs - 1),
              (1, np.concatenate([rng.choice(gapB, 40, replace=False), rng.choice(len(yAB), 20, replace=False)]), 3)]
    for k in range(0, n_bodies, 5):
        checks.append((2 + k, rng.choice(len(shapes[2 + k][1]), 30, replace=False), k % nrhs))
    for p, sel, r in checks:
        body, y_all = shapes[p]
        ub, vb = probs[p]["u"][r].cpu().numpy(), probs[p]["v"][r].cpu().numpy()
        assert np.isfinite(ub).all() and np.isfinite(vb).all()
        xo, no, wo = oracle.quadrature(body.shape, body.h)
        y = y_all[sel]
        x0, n0, b = oracle.closest_point(body.shape, y)
        fc, qc = body.f_coefs[r], body.q_coefs[r]
        uo, vo, _ = oracle.evaluate(xo, no, wo, workloads.poly_eval(fc, xo), workloads.poly_eval(qc, xo), y, x0, n0, b,
                                    workloads.poly_eval(fc, x0), workloads.poly_eval(qc, x0), body.h, (2, 3, 4), 6.0,
                                    oracle.LOCALIZED)
        assert rel_err(ub[sel], uo) <= MIXED_TOL and rel_err(vb[sel], vo) <= MIXED_TOL, (p, r, rel_err(ub[sel], uo),
                                                                                          rel_err(vb[sel], vo))
