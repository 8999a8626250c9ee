"""The FP64 stencils' van Leer slope 2ab/(a+b) (Sec. 2) against the host's
IEEE arithmetic, (2a b) / (a + b) where a b > 0 and else 0: within 2 ulp
wherever the product is a normal number (the kernel takes the quotient by a
Newton step for the reciprocal from a single-precision estimate, and the
sign test on the bit patterns), the same zero where the test fails or the
product underflows, NaN where the host's is, and odd and symmetric, which
the exact mirror symmetry of the operator relies on."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def run(a, b):
    from paper_1610_10053_gb300 import binding as B
    s = B.vanleer_slopes(torch.from_numpy(np.ascontiguousarray(a)).cuda(),
                         torch.from_numpy(np.ascontiguousarray(b)).cuda())
    torch.cuda.synchronize()
    return s.cpu().numpy()


def host(a, b):
    with np.errstate(all="ignore"):
        return np.where(a * b > 0.0, ((2.0 * a) * b) / (a + b), 0.0)


def ulps(s, ref):
    return np.abs(s - ref) / np.spacing(np.abs(ref))


def test_random_slopes_within_two_ulp():
    rng = np.random.default_rng(7)
    m = 1 << 20
    # magnitudes from 1e-150 to 1e150: a + b on both sides of the single-
    # precision estimate's range 2^+-120, products normal; random signs
    a = 10.0 ** rng.uniform(-150, 150, m) * rng.choice([-1.0, 1.0], m)
    b = 10.0 ** rng.uniform(-150, 150, m) * rng.choice([-1.0, 1.0], m)
    # and the operator's own kind: one-sided differences of O(1) values
    x = rng.standard_normal((3, m // 2)) * 10.0 ** rng.uniform(-12, 0, (3, m // 2)) + 1.0
    a[: m // 2] = x[1] - x[0]
    b[: m // 2] = x[2] - x[1]
    s, ref = run(a, b), host(a, b)
    live = ref != 0.0
    assert np.all(s[~live] == 0.0)
    assert live.mean() > 0.3
    assert np.max(ulps(s[live], ref[live])) <= 2.0


def test_special_values():
    tiny = np.finfo(np.float64).smallest_subnormal
    vals = np.array([0.0, -0.0, 1.0, -1.0, 2.5e-37, 3e38, np.inf, -np.inf, np.nan, tiny, -tiny, 1e-170, -1e-170,
                     1e-300, 1e300, 0.75, 2.0 ** -121, 2.0 ** 121])
    a, b = np.meshgrid(vals, vals)
    a, b = a.ravel(), b.ravel()
    s, ref = run(a, b), host(a, b)
    nan = np.isnan(ref)
    assert np.array_equal(np.isnan(s), nan)
    same = s[~nan] == ref[~nan]
    with np.errstate(all="ignore"):
        close = ulps(s[~nan], ref[~nan]) <= 2.0
    # the host's products 2ab of subnormal size round differently from the
    # kernel's 2 (ab); every other case is the host's value or within 2 ulp
    with np.errstate(all="ignore"):
        sub = (np.abs(a * b) < np.finfo(np.float64).tiny)[~nan] & (ref[~nan] != 0.0)
    assert np.all(same | close | sub), np.stack([a[~nan], b[~nan], s[~nan], ref[~nan]], 1)[~(same | close | sub)]


def test_odd_and_symmetric():
    rng = np.random.default_rng(9)
    m = 1 << 16
    a = 10.0 ** rng.uniform(-60, 60, m) * rng.choice([-1.0, 1.0], m)
    b = 10.0 ** rng.uniform(-60, 60, m) * rng.choice([-1.0, 1.0], m)
    s = run(a, b)
    assert np.array_equal(run(b, a), s)
    assert np.array_equal(run(-a, -b), -s)


def test_empty_call():
    from paper_1610_10053_gb300 import binding as B
    e = torch.empty(0, dtype=torch.float64, device="cuda")
    assert B.vanleer_slopes(e, e).numel() == 0
