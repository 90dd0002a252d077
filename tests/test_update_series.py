"""The solver's update evaluates ln(1 + q) for |q| < 1/4 as 2 atanh(z),
z = q / (2 + q), with the atanh Taylor series up to z^11 / 11 (a published
identity, not a library routine).  These checks bound that approximation on
the host: the truncation error in float64, and the float32 evaluation in the
kernel's operation order.  CPU only."""
import numpy as np


def _series(q, dtype):
    q = np.asarray(q, dtype=dtype)
    z = q / (dtype(2) + q)
    w = z * z
    p = w * dtype(1 / 11) + dtype(1 / 9)
    for c in (1 / 7, 1 / 5, 1 / 3, 1.0):
        p = w * p + dtype(c)
    return dtype(2) * z * p


def test_truncation_error_is_negligible():
    q = np.linspace(-0.25, 0.25, 200001)
    q = q[q != 0]
    err = np.abs(_series(q, np.float64) - np.log1p(q)) / np.abs(np.log1p(q))
    assert err.max() < 1e-11


def test_float32_evaluation_within_a_few_ulp():
    g = np.random.default_rng(0)
    q = np.concatenate([g.uniform(-0.25, 0.25, 200000), 10.0 ** g.uniform(-12, -1, 20000),
                        -(10.0 ** g.uniform(-12, -1, 20000))]).astype(np.float32)
    ref = np.log1p(q.astype(np.float64))
    got = _series(q, np.float32).astype(np.float64)
    rel = np.abs(got - ref) / np.abs(ref)
    # the division is approximate on the device (2 ulp); allow 8 ulp in all
    assert rel.max() < 8 * 2.0 ** -24
