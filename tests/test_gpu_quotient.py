"""The quotient of the FP64 stencils' van Leer slope (a Newton step for the
reciprocal from a single-precision estimate, then a product) against the host's correctly
rounded IEEE division: within 2 ulp everywhere, the IEEE division itself
where the estimate's range ends, and odd in each argument, which the exact
mirror symmetry of the operator relies on."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def run(n, d):
    from paper_1610_10053_gb300 import binding as B
    q = B.quotients(torch.from_numpy(n).cuda(), torch.from_numpy(d).cuda())
    torch.cuda.synchronize()
    return q.cpu().numpy()


def within_ulps(q, ref, k):
    finite = np.isfinite(ref)
    err = np.abs(q[finite] - ref[finite])
    return bool(np.all(err <= k * np.spacing(np.abs(ref[finite])))), float(np.max(err / np.spacing(np.abs(ref[finite]))))


def test_random_quotients_within_two_ulp():
    rng = np.random.default_rng(7)
    m = 1 << 20
    # |d| from 1e-40 to 1e40 (beyond the single-precision estimate's range
    # at both ends), |n| from 1e-200 to 1e200, random signs
    d = 10.0 ** rng.uniform(-40, 40, m) * rng.choice([-1.0, 1.0], m)
    n = 10.0 ** rng.uniform(-200, 200, m) * rng.choice([-1.0, 1.0], m)
    # and the operator's own kind: differences of O(1) values
    a = rng.standard_normal(m // 4)
    b = a + rng.standard_normal(m // 4) * 10.0 ** rng.uniform(-16, 0, m // 4)
    d[: m // 4] = a + b
    n[: m // 4] = (2.0 * a) * b
    q = run(n, d)
    ref = n / d
    ok, worst = within_ulps(q, ref, 2)
    assert ok, worst


def test_subnormal_quotients_within_two_ulp():
    rng = np.random.default_rng(8)
    d = 10.0 ** rng.uniform(10, 30, 4096)
    n = 10.0 ** rng.uniform(-300, -290, 4096) * rng.choice([-1.0, 1.0], 4096)
    q = run(n, d)
    ref = n / d
    assert np.any(np.abs(ref) < np.finfo(np.float64).tiny)
    ok, worst = within_ulps(q, ref, 2)
    assert ok, worst


def test_outside_the_estimates_range_is_the_ieee_division():
    tiny = np.finfo(np.float64).smallest_subnormal
    d = np.array([0.0, -0.0, np.inf, -np.inf, np.nan, tiny, -tiny, 2.0 ** -121, 2.0 ** 121, -2.0 ** 125,
                  1e-300, 1e300])
    for nv in (1.0, -3.5, 0.0, np.inf, 1e-300):
        n = np.full_like(d, nv)
        with np.errstate(all="ignore"):
            ref = n / d
        q = run(n, d)
        same = (q == ref) | (np.isnan(q) & np.isnan(ref))
        assert np.all(same), (nv, d[~same], q[~same], ref[~same])
        assert np.all(np.signbit(q[ref == 0]) == np.signbit(ref[ref == 0]))


def test_special_numerators():
    d = np.array([3.0, -3.0, 0.7, 1e30, -1e-30])
    for nv in (0.0, -0.0, np.inf, -np.inf, np.nan):
        n = np.full_like(d, nv)
        ref = n / d
        q = run(n, d)
        same = (q == ref) | (np.isnan(q) & np.isnan(ref))
        assert np.all(same), (nv, q, ref)
        assert np.all(np.signbit(q[~np.isnan(ref)]) == np.signbit(ref[~np.isnan(ref)]))


def test_odd_in_each_argument():
    rng = np.random.default_rng(9)
    m = 1 << 16
    d = 10.0 ** rng.uniform(-40, 40, m)
    n = 10.0 ** rng.uniform(-100, 100, m)
    q = run(n, d)
    assert np.array_equal(run(-n, -d), q)
    assert np.array_equal(run(-n, d), -q)
    assert np.array_equal(run(n, -d), -q)


def test_empty_call():
    from paper_1610_10053_gb300 import binding as B
    e = torch.empty(0, dtype=torch.float64, device="cuda")
    assert B.quotients(e, e).numel() == 0
