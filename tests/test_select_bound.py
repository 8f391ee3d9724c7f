"""The dense-candidate preselection's rule, on the host (Sec. 3.2 selection).

On lattices of 2^20 sites or more the tail preselects dense Ehrenfests'
candidates by their FP32 dS, which is within 1/64 of the FP64 key.  It takes
R = the candidates with FP32 dS > delta (1 + 1/64), finds by two 12-bit radix
levels over the FP32 bit patterns (bits 30..19, then 18..7) the lower end T of
the bin holding the k-th largest FP32 dS in R, lists every valid candidate with
FP32 dS >= T_low = T (1 - 1/32) (every valid one when |R| < k), and counts a
candidate as valid by its FP64 key where it is keyed (listed, or FP32 dS within
1/64 of delta) and by FP32 dS > delta (1 + 1/64) elsewhere.

This is a model of that rule in numpy (the same bit operations and FP32
roundings), checked on seeded candidate sets whose FP32 values sit at the
extremes of the 1/64 band, with exact ties across the k-th key: the list must
hold the exact top k (key descending, site ascending) and the count must equal
the number of keys above delta.  A flaw in the bound (a wrong factor, a bin
edge taken from the wrong side) fails here.
"""
import numpy as np
import pytest

DELTA = 1e-3


def f32(x):
    return np.float32(x)


def bits(a):
    return np.asarray(a, dtype=np.float32).view(np.int32)


def pick_bin(hist, rem):
    """Bin (from the top) holding the rem-th largest entry, and the rank left in it."""
    acc = 0
    for b in range(len(hist) - 1, -1, -1):
        if acc < rem <= acc + hist[b]:
            return b, rem - acc
        acc += int(hist[b])
    return -1, 0


def preselect(ds32, key, k):
    u = bits(ds32)
    dhi = int(bits(f32(DELTA * (1 + 1 / 64))))
    in_r = (u > dhi) & (u < 0x7F800000)
    h1 = np.bincount(u[in_r] >> 19, minlength=4096)
    if h1.sum() < k:
        tlow_bits = 0
    else:
        b1, rem = pick_bin(h1, k)
        sel = in_r & ((u >> 19) == b1)
        h2 = np.bincount((u[sel] >> 7) & 4095, minlength=4096)
        b2, _ = pick_bin(h2, rem)
        ulb = np.array([(b1 << 19) | (b2 << 7)], dtype=np.int32).view(np.float32)[0]
        tlow_bits = int(bits(f32(ulb) * f32(0.96875)))
    listed_side = u >= tlow_bits
    keyed = listed_side | (u <= dhi)
    valid = np.where(keyed, key > DELTA, in_r)
    listed = np.nonzero(valid & listed_side)[0]
    return listed, int(valid.sum())


def exact_top(key, site, k):
    idx = np.nonzero(key > DELTA)[0]
    order = np.lexsort((site[idx], -key[idx]))
    return np.sort(idx[order[:k]])


def candidates(seed, n, spread, tie_at=None):
    rng = np.random.default_rng(seed)
    # keys log-uniform over three decades around delta, some at or below delta
    key = DELTA * 10.0 ** rng.uniform(-0.3, spread, n)
    if tie_at is not None:
        # a block of exact ties straddling the k-th largest key
        srt = np.sort(key)[::-1]
        key[rng.choice(n, 64, replace=False)] = srt[tie_at]
    # FP32 value at the edges of the +-1/64 band (or inside it)
    e = rng.choice([-1.0, 1.0, 0.0], n) * (1 / 64 - 1e-6) + rng.uniform(-1e-3, 1e-3, n)
    e = np.clip(e, -(1 / 64 - 1e-6), 1 / 64 - 1e-6)
    ds32 = (key * (1.0 + e)).astype(np.float32)
    rec = ds32 > f32(DELTA * (1 - 1 / 64))  # the step kernels' recording threshold
    site = rng.permutation(10 * n)[:n]
    return key[rec], ds32[rec], site[rec]


@pytest.mark.parametrize("seed,k,spread,tie", [
    (1, 104, 2.5, None), (2, 1677, 2.5, 1676), (3, 5000, 1.0, 4990), (4, 40000, 0.5, None),
    (5, 1, 3.0, 0), (6, 777, 0.05, 700)])
def test_list_holds_the_exact_top_k_and_the_count_is_exact(seed, k, spread, tie):
    key, ds32, site = candidates(seed, 60000, spread, tie)
    listed, n_valid = preselect(ds32, key, k)
    assert n_valid == int((key > DELTA).sum())
    top = exact_top(key, site, k)
    assert np.all(np.isin(top, listed))
    # selecting among the list gives the exact selection
    lk, ls = key[listed], site[listed]
    ok = lk > DELTA
    order = np.lexsort((ls[ok], -lk[ok]))
    np.testing.assert_array_equal(np.sort(listed[ok][order[:k]]), top)


def test_bound_fails_without_its_margin():
    """The rule depends on T_low's margin: with T itself as the cut (no
    1 - 1/32 factor) some top-k candidate whose FP32 value sits at the low edge
    of its band falls below the cut."""
    key, ds32, site = candidates(2, 60000, 2.5, 1676)
    k = 1677
    u = bits(ds32)
    dhi = int(bits(f32(DELTA * (1 + 1 / 64))))
    in_r = (u > dhi) & (u < 0x7F800000)
    kth = np.sort(ds32[in_r])[::-1][k - 1]
    top = exact_top(key, site, k)
    assert np.any(ds32[top] < kth)
