"""The C-ABI library builds, loads without a GPU and exports every declared symbol; its host-side
set-up (quadrature, smoothing-function table) matches the oracle and the mathematics."""
import ctypes
import os
import re

import numpy as np
import pytest

import oracle
import paper_2507_00156_gb300 as ers
import workloads

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    ers.build()
    return ers.lib()


def declared_functions():
    text = open(os.path.join(ROOT, "include", "ers.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(ers_[A-Za-z0-9_]+)\s*\(", text)))


def test_exports_every_declared_symbol(L):
    names = declared_functions()
    assert len(names) >= 12
    for name in names:
        assert hasattr(L, name), name
    assert sorted(ers.EXPORTS) == names


def test_version_and_error_string(L):
    assert "sm_103a" in ers.version()
    assert L.ers_last_error() is not None


def test_null_arguments_return_codes_without_gpu(L):
    vp = ctypes.c_void_p
    assert L.ers_build_surface(None, 0.1, None) == ers.ERS_E_INVAL
    assert L.ers_surface_info(None, None, None, None, None, None) == ers.ERS_E_INVAL
    assert L.ers_surface_free(None) == ers.ERS_OK
    assert L.ers_closest_point(None, None, 0, None, None, None, None) == ers.ERS_E_INVAL
    p = ers.params()
    assert L.ers_eval(None, ctypes.byref(p), None, 0, None, None, None, None, None, None, None, None) == ers.ERS_E_INVAL
    shp = ers._Shape()
    for i in range(3):
        shp.axes[i] = 1.0
    h = vp()
    assert L.ers_build_surface(ctypes.byref(shp), -1.0, ctypes.byref(h)) == ers.ERS_E_INVAL
    assert "h must be" in L.ers_last_error().decode()
    shp.axes[1] = 0.0
    assert L.ers_build_surface(ctypes.byref(shp), 0.1, ctypes.byref(h)) == ers.ERS_E_INVAL


@pytest.mark.parametrize("shape,inv", [(workloads.unit_sphere(), 16), (workloads.unit_sphere((0.1, -0.05, 0.2)), 32),
                                       (workloads.Shape((0.0, 0.0, 0.0), (1.0, 0.8, 0.6)), 32),
                                       (workloads.Shape((0.0, 0.0, 0.0), (1.0, 0.5, 0.5)), 64)])
def test_library_quadrature_matches_oracle(L, shape, inv):
    L.ers_debug_quadrature.restype = ctypes.c_int64
    P = ctypes.POINTER(ctypes.c_double)
    L.ers_debug_quadrature.argtypes = [P, P, ctypes.c_double, P, P, P, ctypes.c_int64]
    c = np.array(shape.center)
    a = np.array(shape.axes)
    p = lambda v: v.ctypes.data_as(P)
    N = L.ers_debug_quadrature(p(c), p(a), 1 / inv, None, None, None, 0)
    x, n, w = np.empty((N, 3)), np.empty((N, 3)), np.empty(N)
    L.ers_debug_quadrature(p(c), p(a), 1 / inv, p(x), p(n), p(w), N)
    xo, no, wo = oracle.quadrature(shape, 1 / inv)
    assert N == len(wo)
    assert np.abs(x - xo).max() <= 2e-16 * 4
    assert np.abs(n - no).max() <= 1e-15
    assert np.abs(w - wo).max() <= 1e-15 * wo.max()


def _sigma_mp(mp, tau):
    t = mp.sqrt(mp.mpf(tau))
    c = 2 / mp.sqrt(mp.pi)
    if t == 0:
        return [c, c * 2 / 3, c * 4 / 15]
    e, g = mp.erf(t), mp.exp(-t * t)
    return [e / t, (e - c * t * g) / t**3, (e - c * (t + mp.mpf(2) / 3 * t**3) * g) / t**5]


NINT, DEG, INV_W = 384, 6, 16  # intervals of width 1/16 on tau in [0, 24)


F32 = np.float32


def _fmaf(a, b, c):
    """Fused multiply-add of floats: the product of two floats is exact in double, so one rounding
    of the double sum to float (a double rounding only in rare ties, below what the tests resolve)."""
    return F32(np.float64(a) * np.float64(b) + np.float64(c))


def _split_pair(x):
    """The kernel's split of a double into floats: h = x truncated to 24 bits, l = the rest."""
    h = F32(x)
    if abs(float(h)) > abs(x):
        h = np.nextafter(h, F32(0))
    return h, F32(x - float(h))


def _pair_mad(ph, pl, sh, sl, ch, cl):
    """p s + c in float pairs, as the kernel's pair_mad (two-product by FMA, two-sum, renormalize)."""
    th = F32(ph * sh)
    te = _fmaf(ph, sl, _fmaf(pl, sh, _fmaf(ph, sh, -th)))
    u = F32(th + ch)
    v = F32(u - th)
    e = F32(F32(th - F32(u - v)) + F32(ch - v))
    w = F32(F32(e + te) + cl)
    h = F32(u + w)
    return h, F32(w - F32(h - u))


def _fp_mul(a, b):
    """fp_mul of the kernels: the product of the leading floats exactly, plus the cross terms."""
    p = F32(a[0] * b[0])
    return p, _fmaf(a[0], b[1], _fmaf(a[1], b[0], _fmaf(a[0], b[0], -p)))


def _fp_add(a, b):
    """fp_add of the kernels: two-sum of the leading floats, the trailing ones added, renormalized."""
    s = F32(a[0] + b[0])
    v = F32(s - a[0])
    e = F32(F32(a[0] - F32(s - v)) + F32(b[0] - v))
    w = F32(e + F32(a[1] + b[1]))
    h = F32(s + w)
    return h, F32(w - F32(h - s))


def _fp_sum3(x, y, z):
    """fp_sum3 of the kernels: the leading floats by two two-sums, the rest added in float32,
    renormalized."""
    s = F32(x[0] + y[0])
    v = F32(s - x[0])
    e1 = F32(F32(x[0] - F32(s - v)) + F32(y[0] - v))
    t = F32(s + z[0])
    v = F32(t - s)
    e2 = F32(F32(s - F32(t - v)) + F32(z[0] - v))
    w = F32(F32(F32(x[1] + y[1]) + z[1]) + F32(e1 + e2))
    h = F32(t + w)
    return h, F32(w - F32(h - t))


def _fp_dot3(a, b):
    return _fp_sum3(*[_fp_mul(x, y) for x, y in zip(a, b)])


def _layout_eval(rec, s):
    """One function's 12 floats of the device layout (c6, c5, c4, 2i+1, c3 hi/lo, c2 hi/lo, c1 hi/lo,
    c0 hi/lo) at the local variable s, evaluated as the kernel does."""
    sh, sl = _split_pair(s)
    ph, pl = _fmaf(_fmaf(rec[0], sh, rec[1]), sh, rec[2]), F32(0)
    for k in range(4):
        ph, pl = _pair_mad(ph, pl, sh, sl, rec[4 + 2 * k], rec[5 + 2 * k])
    return float(ph) + float(pl)


def _device_layout(fn, nint):
    nbytes = nint * 3 * 48
    raw = np.empty(nbytes // 4, dtype=np.float32)
    fn.argtypes = [ctypes.c_void_p, ctypes.c_int64]
    assert fn(raw.ctypes.data, nbytes) == 0
    assert fn(raw.ctypes.data, nbytes - 8) != 0
    return raw.reshape(nint, 3, 12)


def _taus():
    rng = np.random.default_rng(1)
    return np.concatenate([[0.0, 1e-12, 0.0625, 0.125, 22.09, 23.99], rng.uniform(0, 24, 300)])


def test_sigma_table_accuracy(L):
    """The interpolation table reproduces s_p(t)/t^p (Eqs. (s1)-(s3)) to ~1e-15 on tau = t^2 in [0, 24)."""
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = max(mp.mp.dps, 40)
    tab = np.empty(NINT * 3 * (DEG + 1))
    assert L.ers_debug_sigma_table(tab.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), tab.size) == 0
    tab = tab.reshape(NINT, 3, DEG + 1)
    worst = 0.0
    for tau in _taus():
        i = min(int(tau * INV_W), NINT - 1)
        s = 2 * INV_W * tau - (2 * i + 1)
        ref = _sigma_mp(mp, tau)
        for p_ in range(3):
            got = np.polyval(tab[i, p_], s)
            worst = max(worst, abs(got - float(ref[p_])) / abs(float(ref[p_])))
    assert worst < 3e-15, worst


def test_sigma_device_layout_accuracy(L):
    """The device copy, evaluated as the near-field kernel does (degrees 6..4 in FP32, 3..0 in float
    pairs), stays within ~1e-14 of s_p(t)/t^p: the FP32 part carries less than 2e-8 of the value,
    the float pairs carry the rest to ~2^-46."""
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = max(mp.mp.dps, 40)
    tab = _device_layout(L.ers_debug_sigma_device, NINT)
    assert np.array_equal(tab[:, 0, 3], 2 * np.arange(NINT) + 1)
    host = np.empty(NINT * 3 * (DEG + 1))
    assert L.ers_debug_sigma_table(host.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), host.size) == 0
    host = host.reshape(NINT, 3, DEG + 1)
    for i in range(NINT):
        for p_ in range(3):
            hi_lo = tab[i, p_, 4:].astype(np.float64).reshape(4, 2).sum(1)
            assert np.all(np.abs(hi_lo - host[i, p_, 3:]) <= 2.0**-46 * np.abs(host[i, p_, 3:]))
            assert abs(tab[i, p_, 2]) <= 2e-8 * abs(host[i, p_, 6]), (i, p_)
    worst = 0.0
    for tau in _taus():
        i = min(int(np.float32(tau) * INV_W), NINT - 1)
        s = 2 * INV_W * tau - float(tab[i, 0, 3])
        ref = _sigma_mp(mp, tau)
        for p_ in range(3):
            v = _layout_eval(tab[i, p_], s)
            worst = max(worst, abs(v - float(ref[p_])) / abs(float(ref[p_])))
    assert worst < 2e-14, worst


def test_sigma_device_layout_beyond_the_interval_ends(L):
    """The near kernel picks the interval from the FP32 product r2f * idf (three roundings, at most
    ~1.8e-7 of tau), so the local variable s = r^2 (2 INV_W / delta^2) - (2 i + 1) can leave [-1, 1]
    by up to 2 INV_W tau 1.8e-7 < 1.4e-4 for tau < 24.  Each piece, evaluated as the kernel does at
    |s| = 1 + 2e-4 (just past that bound, on both sides of every interval), still reproduces
    s_p(t)/t^p of Eqs. (s1)-(s3) to ~1e-14."""
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = max(mp.mp.dps, 40)
    tab = _device_layout(L.ers_debug_sigma_device, NINT)
    over = 1.0 + 2e-4
    worst = 0.0
    for i in range(NINT):
        for s in (-over, over):
            tau = (s + 2 * i + 1) / (2 * INV_W)
            if tau < 0:
                continue
            ref = _sigma_mp(mp, tau)
            for p_ in range(3):
                v = _layout_eval(tab[i, p_], s)
                worst = max(worst, abs(v - float(ref[p_])) / abs(float(ref[p_])))
    assert worst < 2e-14, worst


def test_sigma_sharp_device_layout_accuracy(L):
    """The on-surface table (s#_p(t)/t^p of Sec. 2.1, intervals of 1/32 on tau in [0, 64)), as the
    kernel evaluates it (degrees 6..4 in FP32, 3..0 in float pairs), stays within ~1e-14 of 60-digit
    values."""
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = max(mp.mp.dps, 60)
    nint, inv_w = 2048, 32
    tab = _device_layout(L.ers_debug_sigma_sharp_device, nint)

    rng = np.random.default_rng(2)
    taus = np.concatenate([[0.0, 1e-10, 0.5, 1.0, 35.99, 36.0, 63.9], rng.uniform(0, 64, 200)])
    worst = 0.0
    c = 2 / mp.sqrt(mp.pi)
    for tau in taus:
        i = min(int(np.float32(tau) * inv_w), nint - 1)
        s = 2 * inv_w * tau - float(tab[i, 0, 3])
        t = mp.sqrt(mp.mpf(tau))
        if t == 0:
            ref = [c * mp.mpf(8) / 3, c * mp.mpf(16) / 3, c * mp.mpf(32) / 45]
        else:
            e, g = mp.erf(t), mp.exp(-t * t)
            ref = [(e + c / 3 * (5 * t - 2 * t**3) * g) / t, (e - c / 3 * (3 * t - 14 * t**3 + 4 * t**5) * g) / t**3,
                   (e - c / 9 * (9 * t + 6 * t**3 - 4 * t**5) * g) / t**5]
        for p_ in range(3):
            v = _layout_eval(tab[i, p_], s)
            worst = max(worst, abs(v - float(ref[p_])) / abs(float(ref[p_])))
            c0 = float(tab[i, p_, 10]) + float(tab[i, p_, 11])
            assert abs(tab[i, p_, 2]) <= 2e-8 * abs(c0), (i, p_)
    assert worst < 2e-14, worst


@pytest.mark.parametrize("n0", [1, 37, 500, 4000])
def test_library_octree_matches_oracle(L, n0):
    """The host octree of the treecode (Sec. 3.4) is the oracle's: same leaf order of the nodes,
    and every cluster (matched by its node range and level) has the same centre, half-widths and
    radius, bit for bit."""
    import oracle
    x, _, _ = oracle.quadrature(workloads.Shape((0.1, -0.2, 0.05), (1.0, 0.8, 0.6)), 1 / 32)
    N = len(x)
    cap = 4 * N + 64
    geom = np.empty((cap, 7))
    info = np.empty((cap, 5), dtype=np.int32)
    perm = np.empty(N, dtype=np.int32)
    fn = L.ers_debug_octree
    fn.restype = ctypes.c_int64
    fn.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p,
                   ctypes.c_void_p]
    nc = fn(np.ascontiguousarray(x).ctypes.data, N, n0, cap, geom.ctypes.data, info.ctypes.data, perm.ctypes.data)
    t = oracle.tree_info(x, n0)
    assert nc == len(t["rc"])
    assert np.array_equal(perm, t["perm"])
    ref = {(int(s), int(c), int(l)): k for k, (s, c, l) in enumerate(zip(t["start"], t["count"], t["level"]))}
    for c in range(nc):
        k = ref[(int(info[c, 0]), int(info[c, 1]), int(info[c, 4]))]
        lo, hi = t["lo"][k], t["hi"][k]
        assert np.array_equal(geom[c, :3], 0.5 * (lo + hi)) and np.array_equal(geom[c, 3:6], 0.5 * (hi - lo))
        assert geom[c, 6] == t["rc"][k]
        assert info[c, 3] == t["nchild"][k]
        if info[c, 3]:  # children contiguous, one level down, covering the parent's range
            kids = range(info[c, 2], info[c, 2] + info[c, 3])
            assert all(info[j, 4] == info[c, 4] + 1 for j in kids)
            assert sum(info[j, 1] for j in kids) == info[c, 1] and info[info[c, 2], 0] == info[c, 0]


def test_treecode_defaults(L):
    """Eq. (optimal_params): theta = 0.6; N0 = 2000, p = 6 at h = 1/64, doubling N0 and adding 2
    to p per halving of h; held at N0 >= 1000, p >= 6 for coarser h (Table 2's values)."""
    import paper_2507_00156_gb300 as ers
    assert ers.treecode_defaults(1 / 64) == (0.6, 2000, 6)
    assert ers.treecode_defaults(1 / 128) == (0.6, 4000, 8)
    assert ers.treecode_defaults(1 / 256) == (0.6, 8000, 10)
    assert ers.treecode_defaults(1 / 32) == (0.6, 1000, 6)
    assert ers.treecode_defaults(1 / 16) == (0.6, 1000, 6)
    with pytest.raises(ers.ErsError):
        ers.treecode_defaults(0.0)


def test_missing_library_fails_loudly(monkeypatch, tmp_path):
    """Without libers.so the package raises instead of falling back to anything."""
    import paper_2507_00156_gb300 as ers
    monkeypatch.setattr(ers, "_lib", None)
    monkeypatch.setattr(ers, "LIB_PATH", str(tmp_path / "libers.so"))
    with pytest.raises(ImportError, match="not built"):
        ers.lib()
    with pytest.raises(ImportError):
        ers.Surface((0.0, 0.0, 0.0), (1.0, 1.0, 1.0), 1 / 8)


def test_float_pair_primitives_meet_their_bounds():
    """The float-pair operations of the near field (fp_mul, fp_add, fp_fma = fp_add(fp_mul)),
    restated with float32 roundings, against exact rational arithmetic on random operands over six
    decades, with mixed signs, near-cancelling sums and unnormalized inputs (products): the errors
    stay within the bounds derived in the kernels' comments (u = 2^-24, operands split by
    truncation, |l| <= 2u |h|): 12 u^2 |a b| for a product (the neglected product of the trailing
    floats, 4 u^2, and two roundings of the cross terms, 3 u^2 and 5 u^2), 6 u^2 (|a| + |b|) for a
    sum, 24 u^2 (|a b| + |c|) for a product added to a pair, 20 u^2 (sum |a_i b_i|) for the
    three-term dot product and for an accumulator plus two products (fp_sum3)."""
    from fractions import Fraction as Fr
    rng = np.random.default_rng(17)
    u2 = Fr(1, 2 ** 48)
    val = lambda p: Fr(float(p[0])) + Fr(float(p[1]))
    worst = [Fr(0), Fr(0), Fr(0)]
    for _ in range(20000):
        x, y, z = rng.standard_normal(3) * 10.0 ** rng.uniform(-3, 3, 3)
        if rng.random() < 0.3:
            y = -x * (1 + rng.standard_normal() * 1e-6)  # cancellation in the sum
        a, b, c = _split_pair(x), _split_pair(y), _split_pair(z)
        A, B, C = val(a), val(b), val(c)
        m = _fp_mul(a, b)
        worst[0] = max(worst[0], abs(val(m) - A * B) / (abs(A * B) * u2))
        sm = _fp_add(a, b)
        worst[1] = max(worst[1], abs(val(sm) - (A + B)) / ((abs(A) + abs(B)) * u2))
        f = _fp_add(m, c)  # fp_fma: an unnormalized product as an operand
        worst[2] = max(worst[2], abs(val(f) - (A * B + C)) / ((abs(A * B) + abs(C)) * u2))
    worst_dot = Fr(0)
    for _ in range(5000):  # fp_dot3: <= 20 u^2 (|a0 b0| + |a1 b1| + |a2 b2|)
        xs = rng.standard_normal(6) * 10.0 ** rng.uniform(-3, 3, 6)
        if rng.random() < 0.3:
            xs[5] = -(xs[0] * xs[3] + xs[1] * xs[4]) / xs[2] * (1 + rng.standard_normal() * 1e-6)
        a, b = [_split_pair(z) for z in xs[:3]], [_split_pair(z) for z in xs[3:]]
        A, B = [val(z) for z in a], [val(z) for z in b]
        exact = sum(p * q for p, q in zip(A, B))
        worst_dot = max(worst_dot, abs(val(_fp_dot3(a, b)) - exact) / (sum(abs(p * q) for p, q in zip(A, B)) * u2))
    worst_acc = Fr(0)
    for _ in range(5000):  # fp_acc2 = fp_sum3(acc, a b, c d): <= 20 u^2 (|acc| + |a b| + |c d|)
        xs = rng.standard_normal(5) * 10.0 ** rng.uniform(-3, 3, 5)
        if rng.random() < 0.3:
            xs[0] = -(xs[1] * xs[2] + xs[3] * xs[4]) * (1 + rng.standard_normal() * 1e-6)
        acc, a, b, c, d = [_split_pair(z) for z in xs]
        ACC, A, B, C, D = [val(z) for z in (acc, a, b, c, d)]
        got = val(_fp_sum3(acc, _fp_mul(a, b), _fp_mul(c, d)))
        worst_acc = max(worst_acc, abs(got - (ACC + A * B + C * D)) / ((abs(ACC) + abs(A * B) + abs(C * D)) * u2))
    print("worst errors in units of u^2:", [float(w) for w in worst], float(worst_dot), float(worst_acc))
    assert worst[0] <= 12 and worst[1] <= 6 and worst[2] <= 24 and worst_dot <= 20 and worst_acc <= 20
