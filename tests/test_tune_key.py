"""Host logic of the batched-form autotuner: the profile key (no GPU needed)."""
import pytest

from paper_1610_07902_gb300 import spmspv as S


@pytest.fixture(scope="module")
def key():
    S.load()
    return S.spmspv_tune_key


def test_same_power_of_two_profile_shares_a_key(key):
    # B in (128, 256] and mean nnz(x) in [512, 1023] -> one key
    assert key(0, 0, 0, 256, 256 * 600) == key(0, 0, 0, 200, 200 * 1000)
    assert key(0, 0, 0, 256, 256 * 600) != key(0, 0, 0, 257, 257 * 600)
    assert key(0, 0, 0, 256, 256 * 600) != key(0, 0, 0, 256, 256 * 2000)


def test_kind_semiring_and_mask_separate_keys(key):
    base = key(0, 0, 0, 64, 6400)
    assert len({base, key(1, 0, 0, 64, 6400), key(2, 0, 0, 64, 6400), key(0, 1, 0, 64, 6400),
                key(0, 2, 0, 64, 6400), key(0, 0, 1, 64, 6400)}) == 6


def test_degenerate_profiles(key):
    assert key(0, 0, 0, 1, 0) == key(0, 0, 0, 1, 0)
    assert key(0, 0, 0, 1, 0) != key(0, 0, 0, 2, 0)
    k = key(0, 0, 0, 1 << 20, (1 << 20) * (1 << 20))  # large totals stay in their fields
    assert k >> 40 == 0 and (k >> 8) & 0xFFFF == 20 and k & 0xFF == 21
