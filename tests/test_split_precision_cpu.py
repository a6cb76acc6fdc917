"""The split-precision scheme of the tensor-core contraction, emulated on the
CPU: every FP32 operand v is written as hi + lo with hi = tf32(v) and
lo = tf32(v - hi) (tf32: FP32 with the 13 low mantissa bits rounded off,
round to nearest, ties away -- cvt.rna.tf32.f32), and a product a b is formed
as hi_a hi_b + hi_a lo_b + lo_a hi_b.  Each of those three products is exact
in FP32 (11 x 11 significant bits), so the error is the dropped lo_a lo_b
term plus the two representation errors: at most about 3 * 2^-22 of |a b|.
A single TF32 product (hi only) is checked to be far worse, so the test would
catch a scheme that lost its lo terms.  The kernels split by truncation (the
low bits cleared, so both parts are exact TF32 values whatever the tensor
core's own input conversion does); the last tests pin that split and the
tensor-core reduce's packed form, where one MMA per K step forms all four
partial products of [Y_hi; Y_lo] against [Z_hi; Z_lo]."""
import numpy as np


def tf32_rna(v):
    """Round FP32 values to TF32 (10 explicit mantissa bits), to nearest with
    ties away from zero, keeping the FP32 bit layout."""
    u = np.asarray(v, dtype=np.float32).view(np.uint32).astype(np.uint64)
    u = (u + 0x1000) & 0xFFFFE000
    return u.astype(np.uint32).view(np.float32)


def split(v):
    hi = tf32_rna(v)
    lo = tf32_rna(np.asarray(v, dtype=np.float32) - hi)
    return hi, lo


def test_tf32_rounding_keeps_ten_mantissa_bits():
    x = np.float32(1.0) + np.float32(2.0 ** -11)          # exactly half an ulp of tf32 at 1
    assert tf32_rna(x) == np.float32(1.0 + 2.0 ** -10)      # ties away from zero
    assert tf32_rna(np.float32(1.0 + 2.0 ** -12)) == np.float32(1.0)
    assert tf32_rna(np.float32(-3.0)) == np.float32(-3.0)
    r = np.random.default_rng(0).normal(size=1000).astype(np.float32)
    assert np.all((tf32_rna(r).view(np.uint32) & 0x1FFF) == 0)


def test_split_product_error_bound():
    rng = np.random.default_rng(1)
    a = (rng.normal(size=200000) * np.exp(rng.uniform(-20, 20, 200000))).astype(np.float32)
    b = (rng.normal(size=200000) * np.exp(rng.uniform(-20, 20, 200000))).astype(np.float32)
    ah, al = split(a)
    bh, bl = split(b)
    # the three partial products are exact in FP32 (11 x 11 bits), as on the
    # tensor core; sum them in FP64 to isolate the scheme's own error
    three = ah.astype(np.float64) * bh + ah.astype(np.float64) * bl + al.astype(np.float64) * bh
    exact = a.astype(np.float64) * b.astype(np.float64)
    rel = np.abs(three - exact) / np.abs(exact)
    assert rel.max() <= 3 * 2.0 ** -22
    one = ah.astype(np.float64) * bh
    assert (np.abs(one - exact) / np.abs(exact)).max() > 2.0 ** -13   # hi alone: ~2^-11


def test_split_contraction_meets_fp32_tolerance():
    # [X - mu, 1, s]^T Z over 4096 points at the step's distributions, the
    # products split as above and summed in FP64: relative error far below
    # the 1e-5 tolerance (the kernel's FP32 accumulation adds its own, measured
    # on the GPU)
    rng = np.random.default_rng(2)
    X = (rng.normal(0, 10, size=(16, 8))[rng.integers(0, 16, 4096)] +
         rng.normal(size=(4096, 8))).astype(np.float32)
    Z = rng.normal(size=(4096, 4)).astype(np.float32)
    Xc = (X - X.mean(0).astype(np.float32)).astype(np.float32)
    A = np.concatenate([Xc, np.ones((4096, 1), np.float32),
                        (Xc.astype(np.float32) ** 2).sum(1, keepdims=True).astype(np.float32)], 1)
    Ah, Al = split(A)
    Zh, Zl = split(Z)
    got = Ah.T.astype(np.float64) @ Zh + Ah.T.astype(np.float64) @ Zl + Al.T.astype(np.float64) @ Zh
    want = A.T.astype(np.float64) @ Z.astype(np.float64)
    err = np.linalg.norm(got - want) / np.linalg.norm(want)
    assert err <= 1e-6, err


# ---------------------------------------------------------------------------
# The split the kernels use: truncation instead of rounding (hi = v with its
# 13 low mantissa bits cleared, lo the same of v - hi), so that both parts are
# exact TF32 values whatever conversion the tensor core applies to its inputs.

def split_trunc(v):
    v = np.asarray(v, dtype=np.float32)
    hi = (v.view(np.uint32) & np.uint32(0xFFFFE000)).view(np.float32)
    lo = ((v - hi).astype(np.float32).view(np.uint32) & np.uint32(0xFFFFE000)).view(np.float32)
    return hi, lo


def test_truncating_split_representation_bound():
    rng = np.random.default_rng(3)
    v = (rng.normal(size=200000) * np.exp(rng.uniform(-30, 30, 200000))).astype(np.float32)
    hi, lo = split_trunc(v)
    assert np.all((hi.view(np.uint32) & 0x1FFF) == 0) and np.all((lo.view(np.uint32) & 0x1FFF) == 0)
    rel = np.abs(v.astype(np.float64) - hi - lo) / np.abs(v.astype(np.float64))
    assert rel.max() < 2.0 ** -20


def packed_contraction(Y, Z, d2, kp):
    """The tensor-core reduce's one-MMA form: A = [Y_hi; Y_lo] (rows 0..d2-1,
    d2..2 d2-1), B = [Z_hi; Z_lo] (rows 0..kp-1, kp..2 kp-1, k <= kp), the
    accumulator D = A B^T (partial products exact, summed in FP64 here), and
    the entry (c, j) of Y^T Z read back as the sum of D's four blocks."""
    n, k = Z.shape
    Yh, Yl = split_trunc(Y)
    Zh, Zl = split_trunc(Z)
    A = np.zeros((2 * d2, n))
    A[:d2], A[d2:] = Yh.T, Yl.T
    B = np.zeros((2 * kp, n))
    B[:k], B[kp:kp + k] = Zh.T, Zl.T
    D = A @ B.T
    return D[:d2, :k] + D[:d2, kp:kp + k] + D[d2:, :k] + D[d2:, kp:kp + k]


def test_packed_split_contraction_meets_fp32_tolerance():
    rng = np.random.default_rng(4)
    n, d, k = 4096, 12, 12
    X = (rng.normal(0, 10, size=(16, d))[rng.integers(0, 16, n)] + rng.normal(size=(n, d))).astype(np.float32)
    Z = rng.normal(size=(n, k)).astype(np.float32)
    Xc = (X - X.mean(0).astype(np.float32)).astype(np.float32)
    Y = np.concatenate([Xc, np.ones((n, 1), np.float32),
                        (Xc ** 2).sum(1, keepdims=True).astype(np.float32)], 1)
    got = packed_contraction(Y, Z, d + 2, 16)
    want = Y.T.astype(np.float64) @ Z.astype(np.float64)
    assert np.linalg.norm(got - want) / np.linalg.norm(want) <= 1e-6
    # each entry within the per-term bound: |Y||Z| summed, times ~2 2^-20
    bound = np.abs(Y).T.astype(np.float64) @ np.abs(Z).astype(np.float64) * 3 * 2.0 ** -20
    assert np.all(np.abs(got - want) <= bound)
    # dropping the lo rows of either operand (a packing that lost a block)
    # is far outside that bound
    Yh, _ = split_trunc(Y)
    hi_only = Yh.T.astype(np.float64) @ Z.astype(np.float64)
    assert (np.abs(hi_only - want) / bound).max() > 10
