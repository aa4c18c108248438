"""Pins for the oracle's depth binning (Sec. 4.4 quantile binning with the
median plane distance; uniform-in-disparity bins; the culling, depth-sort and
chunking steps of Algorithm 1)."""
import numpy as np
import pytest

from paper_2508_18540_gb300 import synth as S


def _ref(orc):
    return orc.make_ref(S.identity_camera(64), S.display_for(3.0, 0.1))


@pytest.mark.parametrize("n,N", [(1000, 16), (1037, 64), (10, 64), (5, 5), (1, 3)])
def test_quantile_partition_and_median(orc, n, N):
    r = _ref(orc)
    rng = np.random.default_rng(n + N)
    z = rng.uniform(0.5, 9.0, n)
    z[: n // 4] = np.round(z[: n // 4], 1)   # plenty of exact ties
    valid = (rng.uniform(size=n) < 0.9).astype(np.uint8)
    if valid.sum() == 0:
        valid[0] = 1
    order, chunk, d, count, M = orc.bin_primitives(r, z, valid, N, "quantile")
    idx = np.nonzero(valid)[0]
    assert M == idx.size
    # order = lexicographic (z, index) sort of the culled-in primitives
    ref_order = idx[np.lexsort((idx, z[idx]))]
    assert np.array_equal(order, ref_order)
    # partition: every culled-in primitive in exactly one chunk, culled ones in none
    assert np.all(chunk[valid == 0] == -1)
    assert np.all((chunk[idx] >= 0) & (chunk[idx] < N))
    assert np.array_equal(np.bincount(chunk[idx], minlength=N), count)
    # equal-count chunks: sizes differ by at most one, non-decreasing along the order
    nz = count[count > 0]
    assert nz.max() - nz.min() <= 1
    assert np.all(np.diff(chunk[order]) >= 0)
    # chunk k begins at rank ceil(k M / N): rank r belongs to chunk k exactly
    # when k M <= r N < (k + 1) M (the reading chunk = floor(r N / M))
    starts = np.concatenate([[0], np.cumsum(count)[:-1]])
    assert [int(x) for x in starts] == [-(-k * M // N) for k in range(N)]
    # plane distance = median member depth (base frame: + D_forward)
    for k in range(N):
        if count[k]:
            assert d[k] == pytest.approx(np.median(z[chunk == k]) + r.D_forward, rel=1e-15)
        else:
            assert d[k] == 0.0
    assert np.all(np.diff(d[count > 0]) >= 0)


def test_disparity_bins(orc):
    r = _ref(orc)
    rng = np.random.default_rng(3)
    n, N = 5000, 16
    z = rng.uniform(1.8, 5.8, n)
    valid = np.ones(n, np.uint8)
    order, chunk, d, count, M = orc.bin_primitives(r, z, valid, N, "disparity")
    edges = np.linspace(1 / z.min(), 1 / z.max(), N + 1)   # uniform in disparity
    disp = 1 / z
    for k in range(N):
        members = disp[chunk == k]
        if members.size:
            assert members.max() <= edges[k] + 1e-12 and members.min() >= edges[k + 1] - 1e-12
    mids = 0.5 * (edges[:-1] + edges[1:])
    assert np.allclose(d, 1 / mids + r.D_forward, rtol=1e-13)
    assert chunk[np.argmin(z)] == 0 and chunk[np.argmax(z)] == N - 1
    assert np.all(np.diff(chunk[order]) >= 0)


def test_empty_input(orc):
    r = _ref(orc)
    order, chunk, d, count, M = orc.bin_primitives(r, np.zeros(3), np.zeros(3, np.uint8), 4, "quantile")
    assert M == 0 and count.sum() == 0 and np.all(chunk == -1)
