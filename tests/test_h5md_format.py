"""The test-side HDF5 reader's checksum against the check values Bob Jenkins
published with lookup3 (the self-test of lookup3.c): the HDF5 format checksums
its metadata with hashlittle, initial value 0, so the files the library
writes are verified against an independently pinned hash."""
import pytest

from _h5read import hashlittle

FOUR_SCORE = b"Four score and seven years ago"


@pytest.mark.parametrize("data,init,expected", [
    (b"", 0, 0xDEADBEEF),
    (b"", 0xDEADBEEF, 0xBD5B7DDE),
    (FOUR_SCORE, 0, 0x17770551),
    (FOUR_SCORE, 1, 0xCD628161),
])
def test_hashlittle_published_check_values(data, init, expected):
    assert hashlittle(data, init) == expected


def test_hashlittle_every_tail_length_differs():
    # one call per tail length 0..12 past a full block: a dropped or misplaced
    # tail byte would make two of these inputs collide
    base = bytes(range(1, 40))
    seen = {hashlittle(base[:k]) for k in range(12, 25)}
    assert len(seen) == 13
