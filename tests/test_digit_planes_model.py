"""CPU model of the arithmetic behind the tensor-core digit-plane products (tc_digits.cu).

The kernels cut each FP64 operand row into six planes of balanced base-256 digits with a
power-of-two row scale, multiply plane pairs on FP16 tensor cores with FP32 accumulation,
and rely on three facts that this file checks in plain numpy, independent of the GPU:

1. the digits are integers in [-128, 128] (so FP16 holds them exactly) and the planes
   reconstruct each row to 2^-47 of its largest entry;
2. the FP32 sums the tensor cores form are exact where it matters: a group g collects the
   g + 1 plane pairs with s + t = g, each product at most 2^14, over an accumulation period
   of 192 columns, so up to group 4 the largest possible sum 5 * 192 * 2^14 stays below
   2^24 -- checked with worst-case digits and summed in float32 in every order -- and group
   5 (weight 2^-40 of group 0) rounds by a few units at most, below 2^-54 of the period's
   scale;
3. the epilogue's integer conversion of a float pair (hi, lo) times 2^e to FP64 agrees with
   the exact value up to the dropped bits of lo.

Together they bound the product's error by the 47-bit truncation, which the GPU parity
tests then confirm against the oracle (1e-12 and below).  The last tests restate the index
arithmetic the kernels share: the forward product's side-by-side work split against its
reduction, and the accumulation periods against the exact bound."""

import numpy as np

S = 6  # planes


def digits(v):
    """Balanced base-256 digits of integers |v| <= 2^47, most significant first."""
    v = np.asarray(v, dtype=np.int64).copy()
    out = [None] * S
    for k in range(S - 1):
        dk = ((v & 255) ^ 128) - 128
        out[S - 1 - k] = dk
        v = (v - dk) >> 8
    out[0] = v
    return np.stack(out)


def slice_rows(X):
    mx = np.abs(X).max(axis=1)
    e = np.where(mx > 0, np.frexp(mx)[1], 0)
    v = np.rint(np.ldexp(X, (47 - e)[:, None])).astype(np.int64)
    return digits(v), e


def test_digits_are_exact_fp16_integers_and_reconstruct_rows():
    rng = np.random.default_rng(3)
    X = rng.standard_normal((64, 300)) * np.exp(3 * rng.standard_normal((64, 1)))
    X[5, :] = 0.0  # an all-zero row
    X[7, 11] = -np.abs(X[7]).max() * 1.0  # a row whose maximum is negative
    P, e = slice_rows(X)
    assert P.min() >= -128 and P.max() <= 128
    assert np.array_equal(P.astype(np.float16).astype(np.int64), P)  # exact in FP16
    rec = sum(P[s].astype(np.float64) * 2.0 ** (-8 * s) for s in range(S)) * np.ldexp(1.0, e - 7)[:, None]
    rowmax = np.maximum(np.abs(X).max(axis=1), 1e-300)
    assert np.all(np.abs(rec - X).max(axis=1) <= 2.0 ** -47 * rowmax * 1.0001)
    assert np.all(rec[5] == 0.0)


PERIOD = 192  # columns per accumulation period (12 K-steps of 16)


def test_period_group_sums_are_exact_in_float32_at_the_worst_case():
    # every digit at +-128 with signs that make all products +2^14: the largest sum a group
    # can reach over one accumulation period
    for g in range(S):
        pairs = g + 1
        prod = np.full(pairs * PERIOD, 128.0 * 128.0, dtype=np.float32)
        total = pairs * PERIOD * 128 * 128
        sums = [np.float32(0)]
        for x in prod:
            sums[0] = np.float32(sums[0] + x)
        sums += [np.sum(prod, dtype=np.float32), np.sum(prod[::-1], dtype=np.float32)]
        if g <= 4:
            # sequential, pairwise and reversed float32 sums all equal the exact integer
            assert total < 2 ** 24
            assert all(int(v) == total for v in sums)
        else:
            # group 5 may pass 2^24: its rounding, at weight 2^-40 of group 0, stays below
            # 2^-54 of the period's bound on group 0 (PERIOD * 2^14)
            err = max(abs(int(v) - total) for v in sums)
            assert err * 2.0 ** -40 <= 2.0 ** -54 * PERIOD * 2 ** 14
    # one more K-step (16 columns) would already take group 4 past 2^24: the period is at its limit
    assert 5 * (PERIOD + 16) * 128 * 128 > 2 ** 24


def test_digit_plane_product_matches_fp64_to_the_truncation():
    rng = np.random.default_rng(4)
    n, B = 700, 5
    A = rng.standard_normal((n, n)) * np.exp(rng.standard_normal((n, 1)))
    D = rng.standard_normal((B, n))
    P, ea = slice_rows(A)
    Q, eb = slice_rows(D)
    acc = np.zeros((n, B))
    for c0 in range(0, n, PERIOD):
        sl = slice(c0, c0 + PERIOD)
        for g in range(S):
            G = np.zeros((n, B), dtype=np.float32)
            for s in range(g + 1):
                # float32 accumulation, as in the tensor memory
                G = (G + (P[s][:, sl].astype(np.float32) @ Q[g - s][:, sl].astype(np.float32).T)).astype(np.float32)
            exact = sum(P[s][:, sl].astype(np.int64) @ Q[g - s][:, sl].astype(np.int64).T for s in range(g + 1))
            assert np.array_equal(G.astype(np.int64), exact)
            acc += G.astype(np.float64) * 2.0 ** (-8 * g)
    X = acc * np.ldexp(1.0, ea[:, None] + eb[None, :] - 14)
    ref = A @ D.T
    assert np.linalg.norm(X - ref) / np.linalg.norm(ref) < 1e-12


def pair_to_double_scaled(hi, lo, e):
    """Python restatement of the epilogue's integer conversion (two-sum renormalisation,
    64-bit significand alignment, exponent add)."""
    hi, lo = np.float32(hi), np.float32(lo)
    sm = np.float32(hi + lo)
    bb = np.float32(sm - hi)
    lo = np.float32(np.float32(hi - np.float32(sm - bb)) + np.float32(lo - bb))
    hi = sm
    hb = int(np.array(hi, dtype=np.float32).view(np.uint32))
    Eh = (hb >> 23) & 255
    if Eh == 0:
        return 0.0
    X = ((hb & 0x7FFFFF) | 0x800000) << 29
    lb = int(np.array(lo, dtype=np.float32).view(np.uint32))
    El = (lb >> 23) & 255
    if El != 0:
        ml = (lb & 0x7FFFFF) | 0x800000
        sh = El - Eh + 29
        ml = ml << sh if sh >= 0 else (ml >> -sh if sh > -40 else 0)
        X = X - ml if (lb ^ hb) >> 31 else X + ml
    E = Eh
    if X >= 1 << 53:
        X >>= 1
        E += 1
    elif X < 1 << 52:
        X <<= 1
        E -= 1
    bits = ((hb >> 31) << 63) | ((E - 127 + 1023 + e) << 52) | (X & ((1 << 52) - 1))
    return float(np.array(bits, dtype=np.uint64).view(np.float64))


def test_pair_to_double_conversion():
    rng = np.random.default_rng(5)
    for _ in range(2000):
        hi = np.float32(rng.standard_normal() * 10.0 ** rng.integers(-6, 6))
        lo = np.float32(hi * rng.uniform(-2.0 ** -24, 2.0 ** -24))
        e = int(rng.integers(-60, 60))
        exact = (float(hi) + float(lo)) * 2.0 ** e
        got = pair_to_double_scaled(hi, lo, e)
        assert abs(got - exact) <= 2.0 ** -50 * abs(exact)
    assert pair_to_double_scaled(0.0, 0.0, 5) == 0.0
    assert pair_to_double_scaled(-1.5, 0.0, 3) == -12.0
    # a pair whose low part flips the sign of the residual and crosses a power of two
    assert pair_to_double_scaled(1.0, -2.0 ** -30, 0) == 1.0 - 2.0 ** -30


def _complex_case(seed, R=7, Nm=9, B=3):
    rng = np.random.default_rng(seed)
    F = rng.standard_normal((R, Nm)) + 1j * rng.standard_normal((R, Nm))
    m = rng.standard_normal((B, Nm)) + 1j * rng.standard_normal((B, Nm))
    d = rng.standard_normal((B, R)) + 1j * rng.standard_normal((B, R))
    return F, m, d


def test_forward_complex_product_as_interleaved_real_gemm():
    """d-hat[b][i] = sum_j F[i][j] m-hat[b][j] as D[n][i] = sum_k V[n][k] A[i][k], k = 2 j + c, with
    A[i][2j] = Re F, A[i][2j+1] = Im F, V[2b] = (Re m, -Im m), V[2b+1] = (Im m, Re m)."""
    F, m, _ = _complex_case(6)
    R, Nm = F.shape
    B = m.shape[0]
    A = np.empty((R, 2 * Nm))
    A[:, 0::2], A[:, 1::2] = F.real, F.imag
    V = np.empty((2 * B, 2 * Nm))
    V[0::2, 0::2], V[0::2, 1::2] = m.real, -m.imag
    V[1::2, 0::2], V[1::2, 1::2] = m.imag, m.real
    D = V @ A.T
    ref = m @ F.T
    np.testing.assert_allclose(D[0::2], ref.real, rtol=0, atol=1e-13)
    np.testing.assert_allclose(D[1::2], ref.imag, rtol=0, atol=1e-13)


def test_adjoint_complex_product_as_interleaved_real_gemm():
    """m-hat[b][j] = sum_i conj(F[i][j]) d-hat[b][i] as D[j][n] = sum_k A'[j][k] B[n][k], k = 2 i + c,
    with A'[j][2i] = Re F, A'[j][2i+1] = Im F, B[2b] = (Re d, Im d), B[2b+1] = (Im d, -Re d)."""
    F, _, d = _complex_case(7)
    R, Nm = F.shape
    B = d.shape[0]
    Ap = np.empty((Nm, 2 * R))
    Ap[:, 0::2], Ap[:, 1::2] = F.real.T, F.imag.T
    Bv = np.empty((2 * B, 2 * R))
    Bv[0::2, 0::2], Bv[0::2, 1::2] = d.real, d.imag
    Bv[1::2, 0::2], Bv[1::2, 1::2] = d.imag, -d.real
    D = Ap @ Bv.T
    ref = d @ F.conj()
    np.testing.assert_allclose(D[:, 0::2].T, ref.real, rtol=0, atol=1e-13)
    np.testing.assert_allclose(D[:, 1::2].T, ref.imag, rtol=0, atol=1e-13)


def test_adjoint_digit_product_with_per_column_and_per_vector_scales():
    """The whole adjoint pipeline in exact integer arithmetic: A' sliced with one exponent per
    row j (a column of F-hat, over the contraction i), B with one per vector pair (2b, 2b+1);
    the group sums are exact integers and the result matches the complex FP64 product to the
    47-bit truncation."""
    F, _, d = _complex_case(8, R=40, Nm=50, B=4)
    F = F * np.exp(np.random.default_rng(9).standard_normal((1, F.shape[1])))  # columns of very different size
    R, Nm = F.shape
    B = d.shape[0]
    Ap = np.empty((Nm, 2 * R))
    Ap[:, 0::2], Ap[:, 1::2] = F.real.T, F.imag.T
    Bv = np.empty((2 * B, 2 * R))
    Bv[0::2, 0::2], Bv[0::2, 1::2] = d.real, d.imag
    Bv[1::2, 0::2], Bv[1::2, 1::2] = d.imag, -d.real
    P, ea = slice_rows(Ap)
    # one exponent per vector: both rows of a pair share the larger row maximum
    mx = np.maximum(np.abs(Bv[0::2]).max(axis=1), np.abs(Bv[1::2]).max(axis=1))
    eb = np.repeat(np.frexp(mx)[1], 2)
    Q = digits(np.rint(np.ldexp(Bv, (47 - eb)[:, None])).astype(np.int64))
    acc = np.zeros((Nm, 2 * B))
    for g in range(S):
        G = sum(P[s].astype(np.int64) @ Q[g - s].astype(np.int64).T for s in range(g + 1))
        assert np.abs(G).max() < 2 ** 24  # one accumulation period (2R = 80 columns): the FP32 sums are exact
        acc += G.astype(np.float64) * 2.0 ** (-8 * g)
    D = acc * np.ldexp(1.0, ea[:, None] + eb[None, :] - 14)
    ref = d @ F.conj()
    got = D[:, 0::2].T + 1j * D[:, 1::2].T
    assert np.linalg.norm(got - ref) / np.linalg.norm(ref) < 1e-12


# ---------------------------------------------------------------- work split of the products
# Python restatements of the index arithmetic the tensor-core products share between their
# kernels (tc_digits.cu): which CTA takes which (frequency, row group, chunk) unit, where it
# writes each partial tile, and where the fixed-order reduction looks for them; and the
# accumulation periods both the MMA warp and the epilogue derive.

def _fwd_side_by_side(nf, NRG, kpt, slots=152):
    """The forward product's plan: units (w, chunk), each taken by NRG CTAs side by side."""
    total = nf * kpt
    groups = max(1, slots // NRG)
    per = -(-total // groups)
    ctas = -(-total // per) * NRG
    span = (per + kpt - 1) // kpt + 1
    return total, per, ctas, span


def test_forward_side_by_side_split_covers_every_unit_once_and_the_reduction_finds_it():
    import itertools
    for nf, NRG, kpt in itertools.product([1, 5, 51, 201, 211], [1, 2, 3, 10, 18], [1, 7, 64, 256]):
        total, per, ctas, span = _fwd_side_by_side(nf, NRG, kpt)
        written, cover = {}, {}
        for b in range(ctas):  # the kernel: CTA b takes row group b % NRG of units [(b / NRG) per, + per)
            rg, q = b % NRG, b // NRG
            u0, u1 = q * per, min(total, (q + 1) * per)
            first = (q * per) // kpt
            for u in range(u0, u1):
                wt, c = divmod(u, kpt)
                cover[(wt, rg, c)] = cover.get((wt, rg, c), 0) + 1
                if u + 1 == u1 or (u + 1) // kpt != wt:  # the tile's last chunk in this CTA's share
                    slot = wt - first
                    assert 0 <= slot < span
                    assert (b, slot) not in written
                    written[(b, slot)] = (wt, rg)
        assert len(cover) == nf * NRG * kpt and set(cover.values()) == {1}
        found = set()
        for w in range(nf):  # fwd_reduce_kernel: the CTA groups whose runs cover frequency w
            for rg in range(NRG):
                for q in range(w * kpt // per, ((w + 1) * kpt - 1) // per + 1):
                    key = (q * NRG + rg, w - (q * per) // kpt)
                    assert written.get(key) == (w, rg)
                    found.add(key)
        assert found == set(written)


def _period_closes(k, ksteps, tail_cols, share_last, drain_k=12, period_cols=204):
    if share_last:
        return True
    if (k + 1) % drain_k != 0:
        return False
    return not (k + 2 == ksteps and drain_k * 16 + tail_cols <= period_cols)


def test_accumulation_periods_stay_within_the_exact_bound():
    """Every period the schedule forms holds at most 204 data columns (so groups 0-4 sum exactly
    in FP32), for K axes split into CTA shares at any K-step, and the batched adjoint's
    2R = 200 drains once per unit."""
    import random
    rnd = random.Random(7)
    for K in list(range(1, 700)) + [8192, 20000]:
        ksteps = (K + 15) // 16
        tail = K - 16 * (ksteps - 1)
        cuts = sorted({0, ksteps} | {rnd.randrange(ksteps + 1) for _ in range(3)})
        for a, b in zip(cuts, cuts[1:]):  # one CTA share: K-steps [a, b)
            if a == b:
                continue
            start = a
            for k in range(a, b):
                if _period_closes(k, ksteps, tail, k + 1 == b):
                    cols = sum(16 if j < ksteps - 1 else tail for j in range(start, k + 1))
                    assert cols <= 204, (K, a, b, start, k)
                    start = k + 1
            assert start == b  # the share's last K-step closed its period
    assert sum(_period_closes(k, 13, 8, k == 12) for k in range(13)) == 1
