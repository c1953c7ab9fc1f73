"""Host logic of the DCSC auxiliary column index (no GPU): the index the
library builds at handle creation, checked against its definition (a lower
bound of every chunk start among the stored column ids) and by simulating the
work scan's lookup for every column id: a column is found exactly when it is
stored.  Malformed column-id arrays are refused."""
import numpy as np
import pytest

from paper_1610_07902_gb300 import spmspv as S


def lookup(jc, aux, s, j):
    """The work scan's search: binary search of j among the stored ids of its chunk."""
    k = j >> s
    lo, hi = int(aux[k]), int(aux[k + 1])
    end = hi
    while lo < hi:
        mid = (lo + hi) // 2
        if jc[mid] < j:
            lo = mid + 1
        else:
            hi = mid
    return lo < end and jc[lo] == j


@pytest.mark.parametrize("n,nzc,seed", [(1, 0, 1), (1, 1, 2), (100, 4, 3), (5000, 37, 4), (5000, 5000, 5),
                                        (4096, 4096, 6), (70000, 1, 7), (1 << 20, 1000, 8)])
def test_index_matches_definition_and_lookup(n, nzc, seed):
    rng = np.random.default_rng(seed)
    jc = np.sort(rng.choice(n, size=nzc, replace=False)).astype(np.int32)
    aux, s = S.spmspv_dcsc_index(n, jc)
    # smallest s with n / 2^s <= max(nzc, 1)
    assert (n >> s) <= max(nzc, 1) and (s == 0 or (n >> (s - 1)) > max(nzc, 1))
    naux = ((n - 1) >> s) + 2
    assert aux.shape == (naux,)
    starts = np.arange(naux, dtype=np.int64) << s
    np.testing.assert_array_equal(aux, np.searchsorted(jc, starts, side="left"))
    # about one stored column per chunk: the lookup is constant time on average
    assert nzc <= 2 * (naux - 1) + 2
    ids = np.arange(n) if n <= 70000 else np.concatenate([jc, rng.integers(0, n, 20000)])
    stored = set(jc.tolist())
    for j in ids.tolist():
        assert lookup(jc, aux, s, j) == (j in stored), j


@pytest.mark.parametrize("jc", [[3, 1], [1, 1], [0, 100], [-1, 4]])
def test_malformed_column_ids_are_refused(jc):
    with pytest.raises(S.SpmspvError) as e:
        S.spmspv_dcsc_index(100, np.array(jc, np.int32))
    assert e.value.code == S.SPMSPV_ERR_ARG
