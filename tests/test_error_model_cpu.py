"""The error model behind the mixed-precision bars, checked numerically on the
CPU (no GPU, no kernel code): the FP32 products of the mixed GEMM tile round
each FP64 operand to FP32, sum each 32-wide K chunk in FP32 and add the chunk
sums to a running FP32 sum.  The rounding error of such a dot product should
stay within a small multiple of sqrt(32 + K/32) 2^-24 relative to the sum of
|a_t b_t|, and below that of one FP32 running sum over all of K; the operand
rounding adds about sqrt(2) 2^-24 per term.  The parity tests' mixed bars are
derived from this model (0.75 cond(J_g) sqrt(128) 2^-24, with
sqrt(32 + K/32) <= sqrt(128) for K <= 3072)."""
import numpy as np

U = 2.0 ** -24


def _two_level(a32, b32, chunk=32):
    """sum_t a_t b_t per row: FP32 products summed in FP32 within each chunk,
    then the chunk sums added to a running FP32 sum (row-vectorised)."""
    n, k = a32.shape
    run = np.zeros(n, dtype=np.float32)
    for c0 in range(0, k, chunk):
        part = np.zeros(n, dtype=np.float32)
        for t in range(c0, min(k, c0 + chunk)):
            part = (part + a32[:, t] * b32[t]).astype(np.float32)
        run = (run + part).astype(np.float32)
    return run


def _sequential(a32, b32):
    n, k = a32.shape
    run = np.zeros(n, dtype=np.float32)
    for t in range(k):
        run = (run + a32[:, t] * b32[t]).astype(np.float32)
    return run


def test_two_level_sums_follow_the_model():
    rng = np.random.default_rng(20080323)
    for k in (32, 128, 550, 1500):
        a = rng.standard_normal((256, k))
        b = rng.standard_normal(k)
        a32, b32 = a.astype(np.float32), b.astype(np.float32)
        exact = a @ b
        scale = np.abs(a) @ np.abs(b)
        err_2l = np.abs(_two_level(a32, b32).astype(np.float64) - exact) / scale
        err_seq = np.abs(_sequential(a32, b32).astype(np.float64) - exact) / scale
        model = np.sqrt(32.0 + k / 32.0) * U
        # the products of FP32-rounded operands carry their own sqrt(2) u
        # (random, per term); the summation part follows sqrt(32 + K/32) u
        assert np.sqrt(np.mean(err_2l ** 2)) <= 2.0 * model + np.sqrt(2.0) * U, k
        assert err_2l.max() <= 8.0 * model + 4.0 * U, k
        if k >= 550:   # long sums: the two levels beat one running FP32 sum
            assert np.sqrt(np.mean(err_2l ** 2)) < np.sqrt(np.mean(err_seq ** 2)), k
    # the bound the mixed bars use covers every K of the workloads (m <= 1500)
    assert np.sqrt(32.0 + 1500 / 32.0) <= np.sqrt(128.0)
