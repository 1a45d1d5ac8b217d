"""The test-side Philox4x32-10 against the published known-answer vectors."""
from philox_ref import philox4x32_10


def test_philox_known_answers():
    assert philox4x32_10((0, 0, 0, 0), (0, 0)) == (0x6627E8D5, 0xE169C58D, 0xBC57AC4C, 0x9B00DBD8)
    ff = 0xFFFFFFFF
    assert philox4x32_10((ff, ff, ff, ff), (ff, ff)) == (0x408F276D, 0x41C83B0E, 0xA20BC7C6, 0x6D5451FD)
