"""Pins for the oracle's random block sampling (Algorithm 1, 'pick j with
probability ||A_{:,J_j}||_F^2 / ||A||_F^2').  The generator is Philox4x64-10
(Salmon et al., SC'11); numpy ships an independent implementation of it."""
import numpy as np
import pytest

import oracle as O
from workloads import contiguous_offsets, gaussian_problem


def _numpy_block(key, ctr_int):
    """Philox4x64-10 block at counter ctr_int via numpy, which adds one to
    the counter (with carry through all four words) before encrypting."""
    c = (ctr_int - 1) % (1 << 256)
    words = np.array([(c >> (64 * i)) & ((1 << 64) - 1) for i in range(4)], dtype=np.uint64)
    bg = np.random.Philox(key=np.array(key, dtype=np.uint64), counter=words)
    return bg.random_raw(4)


@pytest.mark.parametrize("key", [(0, 0), (5, 7), (2**64 - 1, 12345), (0xDEADBEEF, 2**63)])
@pytest.mark.parametrize("ctr", [0, 1, 2, 77, 2**32 + 5, 2**64 - 1, 3 * 2**64 + 9])
def test_philox_matches_numpy(key, ctr):
    words = [(ctr >> (64 * i)) & ((1 << 64) - 1) for i in range(4)]
    assert np.array_equal(O.philox(words, key), _numpy_block(key, ctr))


def test_uniform_is_top_53_bits_of_word0():
    for d in [0, 1, 2, 1000, 2**40]:
        w0 = int(_numpy_block((11, 3), d)[0])
        u = O.uniform(11, 3, d)
        assert u == (w0 >> 11) * 2.0 ** -53
        assert 0.0 <= u < 1.0


def test_pick_smallest_index_above_target():
    cdf = np.array([1.0, 1.0, 3.0, 3.0, 6.0])      # blocks 1 and 3 have zero norm
    # u * 6 = target; the pick is the first cdf entry strictly above it
    assert O.pick(cdf, 0.0) == 0
    assert O.pick(cdf, 1.0 / 6.0 - 1e-12) == 0
    assert O.pick(cdf, 1.0 / 6.0) == 2               # target == 1.0 exactly: block 0 excluded
    assert O.pick(cdf, 0.49) == 2
    assert O.pick(cdf, 0.5) == 4
    assert O.pick(cdf, 1.0 - 2**-53) == 4
    # a target that rounds to the total falls back to the last nonzero block
    cdf2 = np.array([2.0, 5.0, 5.0])
    assert O.pick(cdf2, 1.0) == 1
    # zero-norm blocks are never picked
    rng = np.random.default_rng(0)
    picks = {O.pick(cdf, float(u)) for u in rng.random(2000)}
    assert picks <= {0, 2, 4}


def test_block_norms_are_block_sums_of_squares():
    rng = np.random.default_rng(3)
    A = rng.standard_normal((23, 17))
    ro = contiguous_offsets(23, 5)
    co = contiguous_offsets(17, 4)
    nr, nc = O.block_norms(A, ro, co)
    for i in range(len(ro) - 1):
        assert nr[i] == pytest.approx(np.sum(A[ro[i]:ro[i + 1]] ** 2), rel=1e-14)
    for j in range(len(co) - 1):
        assert nc[j] == pytest.approx(np.sum(A[:, co[j]:co[j + 1]] ** 2), rel=1e-14)
    assert np.sum(nr) == pytest.approx(np.sum(A * A), rel=1e-14)
    assert np.array_equal(O.cdf(nr), np.cumsum(nr))   # numpy cumsum is left to right


def test_partition_offsets_follow_section_3():
    off = contiguous_offsets(1000, 20)
    assert off[0] == 0 and off[-1] == 1000 and len(off) == 51
    assert np.all(np.diff(off) == 20)
    off = contiguous_offsets(23, 5)
    assert list(off) == [0, 5, 10, 15, 20, 23]       # last block holds what is left


def _chi2_pvalue(counts, probs):
    from scipy.stats import chisquare
    n = counts.sum()
    return chisquare(counts, probs * n).pvalue


def test_sampled_block_frequencies_follow_norms():
    """Empirical frequencies of the row and column picks of the sampler over
    1e5 draws against ||block||_F^2 / ||A||_F^2 (chi-square)."""
    p = gaussian_problem(60, 40, seed=1)
    A = p.A.copy()
    A[10:20] *= 3.0          # uneven row-block norms
    A[:, 0:8] *= 0.2         # uneven column-block norms
    ro = contiguous_offsets(60, 10)
    co = contiguous_offsets(40, 8)
    nr, nc, cr, cc = O.tables(A, ro, co)
    N = 100000
    jc = np.zeros(len(nc), dtype=np.int64)
    ic = np.zeros(len(nr), dtype=np.int64)
    for k in range(1, N + 1):
        jc[O.pick(cc, O.uniform(9, 0, 2 * (k - 1)))] += 1
        ic[O.pick(cr, O.uniform(9, 0, 2 * (k - 1) + 1))] += 1
    assert _chi2_pvalue(jc, nc / nc.sum()) > 1e-4
    assert _chi2_pvalue(ic, nr / nr.sum()) > 1e-4


def test_recorded_indices_are_the_sampler_draws():
    p = gaussian_problem(30, 20, seed=2)
    ro = contiguous_offsets(30, 4)
    co = contiguous_offsets(20, 3)
    nr, nc, cr, cc = O.tables(p.A, ro, co)
    r = O.rebk(p.A, p.b, ro, co, 1.0, seed=42, stream=3, k0=5, iters=50, record=True)
    for it in range(50):
        k = 5 + it + 1
        assert r["idx"][it, 0] == O.pick(cc, O.uniform(42, 3, 2 * (k - 1)))
        assert r["idx"][it, 1] == O.pick(cr, O.uniform(42, 3, 2 * (k - 1) + 1))
