"""Host-side statistics of the BER/FER reports (CPU): the exact FER interval against scipy's own
exact binomial interval, and the frame-clustered BER interval against the normal interval of the
explicit per-frame error counts it is built from."""
import numpy as np
import pytest

scipy_stats = pytest.importorskip("scipy.stats")


def test_clopper_pearson_matches_scipy_exact_interval():
    from paper_1204_0334_gb300.noms import clopper_pearson

    for k, n in ((0, 50), (3, 1000), (100, 262774), (49, 50), (50, 50)):
        lo, hi = clopper_pearson(k, n)
        ref = scipy_stats.binomtest(k, n).proportion_ci(confidence_level=0.95, method="exact")
        assert abs(lo - ref.low) <= 1e-12 and abs(hi - ref.high) <= 1e-12, (k, n)


def test_ber_interval_from_sums_equals_per_frame_interval():
    from paper_1204_0334_gb300.noms import ber_interval

    rng = np.random.default_rng(1)
    N = 18360
    e = np.where(rng.random(20000) < 0.01, rng.integers(1, 400, 20000), 0)  # bursts of wrong bits
    r = {"frames": len(e), "frame_errors": int((e > 0).sum()), "bit_errors": int(e.sum()),
         "bit_errors_sq": int((e.astype(np.int64) ** 2).sum())}
    lo, hi = ber_interval(r, N)
    z = scipy_stats.norm.ppf(0.975)
    half = z * e.std(ddof=1) / np.sqrt(len(e))
    assert abs(lo - (e.mean() - half) / N) < 1e-15 and abs(hi - (e.mean() + half) / N) < 1e-15
    # wider than treating the bits as independent trials
    assert hi - lo > 3 * (2 * z * np.sqrt(e.sum() / (len(e) * N) / (len(e) * N)))


def test_ber_interval_without_errors_is_bounded_by_the_fer_limit():
    from paper_1204_0334_gb300.noms import ber_interval, clopper_pearson

    r = {"frames": 1 << 20, "frame_errors": 0, "bit_errors": 0, "bit_errors_sq": 0}
    assert ber_interval(r, 18360) == (0.0, clopper_pearson(0, 1 << 20)[1])
