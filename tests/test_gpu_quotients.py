"""The quotients the FP64 stencils stage (Sec. 2): the specific internal
energy E / rho and the face velocities m_d / rbar, formed by a Newton step
for the reciprocal from a single-precision estimate.  Held against the
host's IEEE division: within 2 ulp wherever the divisor lies within 2^+-120
and the quotient is a normal number, the host's own value (the IEEE
division) for every other divisor, and odd in either operand, which the
exact mirror symmetry of the operator relies on (u = m / rbar changes sign
with m)."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def run(n, d):
    from paper_1610_10053_gb300 import binding as B
    q = B.stencil_quotients(torch.from_numpy(np.ascontiguousarray(n)).cuda(),
                            torch.from_numpy(np.ascontiguousarray(d)).cuda())
    torch.cuda.synchronize()
    return q.cpu().numpy()


def ulps(q, ref):
    return np.abs(q - ref) / np.spacing(np.abs(ref))


def test_random_quotients_within_two_ulp():
    rng = np.random.default_rng(11)
    m = 1 << 20
    # divisors across the estimate's whole range 2^+-120 (and numerators so
    # the quotients stay normal), random signs
    n = 10.0 ** rng.uniform(-100, 100, m) * rng.choice([-1.0, 1.0], m)
    d = 2.0 ** rng.uniform(-119.9, 119.9, m) * rng.choice([-1.0, 1.0], m)
    # and the operator's own kind: E / rho and m / rbar on O(1) densities
    k = m // 2
    rho = 1.0 + rng.uniform(0.0, 1.0, (2, k))
    n[:k // 2] = 120.0 * rng.uniform(0.5, 2.0, k // 2)
    d[:k // 2] = rho[0, :k // 2]
    n[k // 2:k] = rng.standard_normal(k - k // 2) * 10.0 ** rng.uniform(-12, 0, k - k // 2)
    d[k // 2:k] = 0.5 * (rho[0, k // 2:] + rho[1, k // 2:])
    q, ref = run(n, d), n / d
    assert np.max(ulps(q, ref)) <= 2.0


def test_divisors_outside_the_estimate_take_the_ieee_division():
    tiny = np.finfo(np.float64).smallest_subnormal
    dvals = np.array([0.0, -0.0, np.inf, -np.inf, np.nan, tiny, -tiny, 1e-300, 1e300, 2.0 ** -121, -2.0 ** 121,
                      2.0 ** -125, 2.0 ** 125])
    nvals = np.array([0.0, -0.0, 1.0, -3.5, 7e-20, 1e20, np.inf, np.nan])
    n, d = np.meshgrid(nvals, dvals)
    n, d = n.ravel(), d.ravel()
    q = run(n, d)
    with np.errstate(all="ignore"):
        ref = n / d
    nan = np.isnan(ref)
    assert np.array_equal(np.isnan(q), nan)
    assert np.array_equal(q[~nan], ref[~nan])


def test_edges_of_the_estimate_range():
    # divisors at and just inside 2^+-120: the estimate path, still 2 ulp
    d = np.array([2.0 ** -120, 2.0 ** 120 * (1 - 2.0 ** -52), 2.0 ** -120 * 1.5, 2.0 ** 119 * 1.9999,
                  -(2.0 ** -120), 1.0, 1.0 + 2.0 ** -52, 2.0 - 2.0 ** -52])
    n = np.array([1.0, 1e30, -3.0, 7.0, 2.0, 1.0, 3.0, -5.0])
    q, ref = run(n, d), n / d
    assert np.max(ulps(q, ref)) <= 2.0


def test_odd_in_either_operand():
    rng = np.random.default_rng(13)
    m = 1 << 16
    n = 10.0 ** rng.uniform(-60, 60, m) * rng.choice([-1.0, 1.0], m)
    d = 10.0 ** rng.uniform(-40, 40, m) * rng.choice([-1.0, 1.0], m)
    q = run(n, d)
    assert np.array_equal(run(-n, d), -q)
    assert np.array_equal(run(n, -d), -q)


def test_empty_call():
    from paper_1610_10053_gb300 import binding as B
    e = torch.empty(0, dtype=torch.float64, device="cuda")
    assert B.stencil_quotients(e, e).numel() == 0
