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
