"""CPU oracle for the CAFS count-and-emit frequency sort.

TEST INFRASTRUCTURE ONLY.  This module is the plain, slow, obviously correct
restatement of what the CAFS paper ("CAFS: A Cache-Aware Frequency Sort for
Low-Cardinality Integer Data on x86-64") computes.  Only the test-suite,
``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may import
it.  The CUDA library never calls it and it never calls the CUDA library: the
two share no code, constants tables or helpers.

Every function works on a 1-D numpy array of signed ``int32`` or ``int64``
keys, uses Python integers (unbounded) for every derived quantity and follows
the paper's steps in the paper's order:

* ``frequency_sort`` -- the result itself (Sec. 3.1): the unique
  non-decreasing rearrangement of the input multiset, produced as the paper's
  count-then-emit skeleton (Sec. 4.1): count each distinct key, then emit each
  key ``count`` times in increasing key order.
* ``stable_argsort`` -- the permutation of Sec. 3.1's problem statement, with
  equal keys in input order, by the same count-then-emit skeleton: the
  positions of each distinct key collected in input order, then emitted in
  increasing key order.
* ``ordered_signed`` / ``frequency_sort_any`` / ``final_path_any`` /
  ``stable_argsort_any`` -- more key types: unsigned integers in their natural
  order and IEEE-754 binary32/binary64 in the standard's totalOrder (negative
  NaNs, -inf, negative numbers, -0, +0, positive numbers, +inf, positive
  NaNs; equal keys are equal bit patterns).  Each maps onto the signed
  integers of its width by an order-preserving bijection, and the signed
  functions do the rest.
* ``sample_positions`` / ``chao1`` -- the strided sampler and the smoothed
  Chao1 estimator (Sec. 2.4, Sec. 4.3, Algorithm 2, Eq. 5).
* ``table_size`` -- the hash-table sizing of Eq. 6 with its clamps (Sec. 4.5).
* ``dispatch`` -- the adaptive dispatcher (Table 2, Algorithm 3).
* ``final_path`` -- which branch actually produces the output once the
  tiny-count check (Sec. 4.4) and the overflow guard (Sec. 4.5, Algorithm 4,
  read as "distinct keys > C/2", see ``overflow_limit``) have run.

Readings of points the paper leaves open:

* keys are signed two's-complement integers sorted ascending (the paper states
  the problem for unsigned 64-bit keys in Sec. 3.1 but ships ``int32_t`` and
  ``int64_t`` specialisations, Sec. 5);
* the Chao1 correction is an integer floor division (Eq. 5);
* the sampling loop of Algorithm 2 stops before ``min(N, s*stride)``
  (exclusive bound), so N >= 1024 gives exactly 1024 samples and N < 1024 gives
  N samples; saturation (``u == s``) can then only happen for N >= 1024;
* ``M = min(max(bit_ceil(8*K_hat/cap), 8), bit_ceil(ceil(N/cap)))`` where
  ``bit_ceil`` is the smallest power of two >= its argument (Eq. 6 and the
  clamps stated under it; the lower clamp is applied first);
* the high-entropy test is the strict ``2*K_hat > N`` of Algorithm 3;
* a failed tiny count (Sec. 4.4) continues in the main path with the same
  K_hat and without re-testing ``2*K_hat > N``;
* the spill guard of Algorithm 4 depends on insertion order, which a parallel
  GPU cannot reproduce; it is replaced by an order-independent guard that
  fires when the number of distinct keys exceeds ``L = C/2`` slots.

Parity status: every function here is pinned by tests under ``tests/``
(brute force on tiny inputs, the paper's worked table sizes, closed-form
examples of the estimator and inputs that force each dispatcher branch).
"""

from __future__ import annotations

import collections
from dataclasses import dataclass

import numpy as np

# Algorithm 2 / Sec. 4.3: number of strided samples s.
SAMPLE_COUNT = 1024
# Table 2 / Algorithm 3: arrays shorter than this bypass sampling.
SMALL_N_LIMIT = 2048
# Table 2 / Algorithm 3: the tiny-count branch handles K_hat <= 8 and u <= 8.
TINY_LIMIT = 8
# Eq. 6: keys per 64-byte bucket.
BUCKET_CAP = {4: 8, 8: 4}

# Branch labels.  The values match the C ABI's cafs_path enumeration so that
# tests can compare them directly; the labels come from Table 2 and
# Algorithms 3-4.
EMPTY = 0
BYPASS_SORTED = 1
SMALL_N = 2
TINY = 3
MAIN = 4
HIGH_ENTROPY_RADIX = 5
MAIN_OVERFLOW_RADIX = 6
TINY_MISS_MAIN = 7
TINY_MISS_MAIN_OVERFLOW_RADIX = 8

PATH_NAMES = {
    EMPTY: "empty",
    BYPASS_SORTED: "bypass_sorted",
    SMALL_N: "small_n",
    TINY: "tiny",
    MAIN: "main",
    HIGH_ENTROPY_RADIX: "high_entropy_radix",
    MAIN_OVERFLOW_RADIX: "main_overflow_radix",
    TINY_MISS_MAIN: "tiny_miss_main",
    TINY_MISS_MAIN_OVERFLOW_RADIX: "tiny_miss_main_overflow_radix",
}


def _check_keys(keys: np.ndarray) -> np.ndarray:
    keys = np.asarray(keys)
    if keys.ndim != 1 or keys.dtype not in (np.int32, np.int64):
        raise TypeError("keys must be a 1-D int32 or int64 array")
    return keys


def frequency_sort(keys: np.ndarray) -> np.ndarray:
    """Sec. 3.1 and Sec. 4.1: count every distinct key, emit in key order.

    ``np.unique`` returns the distinct keys in increasing order together with
    how often each occurs (the count step); ``np.repeat`` writes each key that
    many times (the emit step, the paper's ``fill_n`` per pair).
    """
    keys = _check_keys(keys)
    distinct, counts = np.unique(keys, return_counts=True)
    return np.repeat(distinct, counts).astype(keys.dtype, copy=False)


def stable_argsort(keys: np.ndarray) -> np.ndarray:
    """Sec. 3.1's permutation pi (keys[pi] non-decreasing) with equal keys in
    input order, as count-then-emit (Sec. 4.1) over positions: every distinct
    key collects the positions where it occurs, in input order; the position
    lists are then emitted in increasing key order.  Returns uint32 positions.
    """
    keys = _check_keys(keys)
    positions: dict[int, list[int]] = {}
    for i, k in enumerate(keys.tolist()):
        positions.setdefault(k, []).append(i)
    out = [i for k in sorted(positions) for i in positions[k]]
    return np.asarray(out, dtype=np.uint32)


# More key types: the order each one sorts in, as signed integers of the
# same width (an order- and equality-preserving bijection).
_SIGNED_OF = {np.dtype(np.uint32): np.int32, np.dtype(np.uint64): np.int64,
              np.dtype(np.float32): np.int32, np.dtype(np.float64): np.int64,
              np.dtype(np.int32): np.int32, np.dtype(np.int64): np.int64}


def ordered_signed(keys: np.ndarray) -> np.ndarray:
    """Signed integers ordered like ``keys``: unsigned keys with the sign bit
    flipped (0 becomes the signed minimum); IEEE floats by their bits, with
    the magnitude bits of negative values inverted (a larger magnitude is a
    smaller number), which is the totalOrder of IEEE 754."""
    keys = np.asarray(keys)
    if keys.dtype not in _SIGNED_OF:
        raise TypeError("unsupported key type")
    it = _SIGNED_OF[keys.dtype]
    if keys.dtype.kind == "i":
        return keys
    bits = keys.view(it)
    sign = np.array(np.iinfo(it).min, dtype=it)
    if keys.dtype.kind == "u":
        return bits ^ sign
    return np.where(bits < 0, bits ^ ~sign, bits).astype(it)


def from_ordered_signed(ordered: np.ndarray, dtype) -> np.ndarray:
    """Inverse of ``ordered_signed`` (both maps are their own inverse on the
    bits)."""
    dtype = np.dtype(dtype)
    if dtype.kind == "i":
        return ordered.astype(dtype, copy=False)
    it = _SIGNED_OF[dtype]
    sign = np.array(np.iinfo(it).min, dtype=it)
    if dtype.kind == "u":
        return (ordered ^ sign).view(dtype)
    return np.where(ordered < 0, ordered ^ ~sign, ordered).astype(it).view(dtype)


def frequency_sort_any(keys: np.ndarray) -> np.ndarray:
    """``frequency_sort`` for any supported key type."""
    keys = np.asarray(keys)
    return from_ordered_signed(frequency_sort(ordered_signed(keys)), keys.dtype)


def final_path_any(keys: np.ndarray) -> int:
    """``final_path`` for any supported key type (the dispatcher sees the keys
    in their order; distinct bit patterns are distinct keys)."""
    return final_path(ordered_signed(keys))


def stable_argsort_any(keys: np.ndarray) -> np.ndarray:
    """``stable_argsort`` for any supported key type."""
    return stable_argsort(ordered_signed(keys))


def is_monotone(keys: np.ndarray) -> bool:
    """Algorithm 3, IsMonotone: true iff the keys are non-decreasing."""
    keys = _check_keys(keys)
    return bool(np.all(keys[:-1] <= keys[1:])) if keys.size > 1 else True


def sample_positions(n: int) -> np.ndarray:
    """Algorithm 2: positions 0, stride, 2*stride, ... below min(N, s*stride)."""
    stride = max(1, n // SAMPLE_COUNT)
    end = min(n, SAMPLE_COUNT * stride)
    return np.arange(0, end, stride, dtype=np.int64)


def bit_ceil(x: int) -> int:
    """Smallest power of two >= x (1 for x <= 1), as C++20 std::bit_ceil."""
    x = int(x)
    if x <= 1:
        return 1
    return 1 << (x - 1).bit_length()


@dataclass(frozen=True)
class Estimate:
    """Everything the sampler, Chao1 and Eq. 6 produce for one input."""

    n: int
    stride: int
    n_samples: int
    u: int
    f1: int
    f2: int
    k_hat: int
    saturated: bool
    M: int
    C: int
    L: int
    sample_keys: tuple  # distinct sample values, increasing


def chao1_from_spectrum(u: int, f1: int, f2: int, n: int) -> tuple[int, bool]:
    """Eq. 5 with the saturation rule of Algorithm 2.

    Returns (K_hat, saturated).  K_hat = u + floor(f1^2 / (2 (f2 + 1))); when
    every one of the s samples is distinct (u == s) the estimate saturates to N.
    """
    if u == SAMPLE_COUNT:
        return n, True
    return u + (f1 * f1) // (2 * (f2 + 1)), False


def table_size(k_hat: int, n: int, key_bytes: int) -> tuple[int, int, int]:
    """Eq. 6 and its clamps (Sec. 4.5): returns (M buckets, C slots, L limit).

    cap is 4 keys per bucket for 64-bit keys and 8 for 32-bit keys, so
    8*K_hat/cap is an integer.  C = M*cap slots, L = C/2 is the overflow limit
    on the number of distinct keys.
    """
    cap = BUCKET_CAP[key_bytes]
    m = bit_ceil((8 * k_hat) // cap)
    m = max(m, 8)
    m = min(m, bit_ceil(-(-n // cap)))
    c = m * cap
    return m, c, c // 2


def chao1(keys: np.ndarray) -> Estimate:
    """Algorithm 2: strided sample, frequency spectrum, Chao1 estimate."""
    keys = _check_keys(keys)
    n = int(keys.size)
    stride = max(1, n // SAMPLE_COUNT)
    pos = sample_positions(n)
    sample = keys[pos]
    distinct, counts = np.unique(sample, return_counts=True)
    u = int(distinct.size)
    f1 = int(np.count_nonzero(counts == 1))
    f2 = int(np.count_nonzero(counts == 2))
    k_hat, saturated = chao1_from_spectrum(u, f1, f2, n)
    m, c, lim = table_size(k_hat, n, keys.dtype.itemsize)
    return Estimate(
        n=n, stride=stride, n_samples=int(pos.size), u=u, f1=f1, f2=f2,
        k_hat=int(k_hat), saturated=bool(saturated), M=m, C=c, L=lim,
        sample_keys=tuple(int(v) for v in distinct),
    )


def dispatch(keys: np.ndarray) -> int:
    """Algorithm 3 and Table 2: the branch the dispatcher selects."""
    keys = _check_keys(keys)
    n = int(keys.size)
    if n == 0:
        return EMPTY
    if is_monotone(keys):
        return BYPASS_SORTED
    if n < SMALL_N_LIMIT:
        return SMALL_N
    est = chao1(keys)
    if est.k_hat <= TINY_LIMIT and est.u <= TINY_LIMIT:
        return TINY
    if 2 * est.k_hat > n:
        return HIGH_ENTROPY_RADIX
    return MAIN


def distinct_count(keys: np.ndarray) -> int:
    """K of Sec. 3.1: the number of distinct keys in the whole input."""
    return int(np.unique(_check_keys(keys)).size)


def overflow_limit(keys: np.ndarray) -> int:
    """The guard's limit L = C/2 for this input's estimate (Eq. 6)."""
    return chao1(keys).L


def final_path(keys: np.ndarray) -> int:
    """Which branch produces the output.

    TINY succeeds when the tiny counters add up to N, i.e. every key is one
    of the sampled keys (Sec. 4.4); otherwise control falls into the main path
    with the same K_hat.  The main path keeps its result unless the guard
    fires (distinct keys > L), in which case the radix fallback sorts.
    """
    keys = _check_keys(keys)
    d = dispatch(keys)
    if d not in (TINY, MAIN):
        return d
    est = chao1(keys)
    k_true = distinct_count(keys)
    if d == TINY:
        if set(np.unique(keys).tolist()) <= set(est.sample_keys):
            return TINY
        return TINY_MISS_MAIN_OVERFLOW_RADIX if k_true > est.L else TINY_MISS_MAIN
    return MAIN_OVERFLOW_RADIX if k_true > est.L else MAIN


def sort_and_report(keys: np.ndarray) -> dict:
    """Sorted output plus the decisions a caller can compare against."""
    keys = _check_keys(keys)
    est = chao1(keys) if keys.size else None
    path = final_path(keys)
    counted = path in (TINY, MAIN, TINY_MISS_MAIN)
    return {
        "out": frequency_sort(keys),
        "dispatch": dispatch(keys),
        "path": path,
        "estimate": est,
        "k_distinct": distinct_count(keys) if counted else None,
    }


def histogram(keys) -> collections.Counter:
    """Per-key counts as a Counter (used by invariant checks)."""
    return collections.Counter(int(v) for v in np.asarray(keys).tolist())
