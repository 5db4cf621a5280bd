"""Pins of oracle.philox: published Philox4x32-10 known-answer vectors and the Box-Muller map."""
import numpy as np
import pytest

from oracle.philox import philox4x32_10, uniforms_from_bits, white_noise

# Known-answer vectors published with the Random123 library (Salmon et al., SC'11):
# (counter, key) -> output for philox4x32 with 10 rounds.
KAT = [
    ((0x00000000, 0x00000000, 0x00000000, 0x00000000), (0x00000000, 0x00000000),
     (0x6627E8D5, 0xE169C58D, 0xBC57AC4C, 0x9B00DBD8)),
    ((0xFFFFFFFF, 0xFFFFFFFF, 0xFFFFFFFF, 0xFFFFFFFF), (0xFFFFFFFF, 0xFFFFFFFF),
     (0x408F276D, 0x41C83B0E, 0xA20BC7C6, 0x6D5451FD)),
    ((0x243F6A88, 0x85A308D3, 0x13198A2E, 0x03707344), (0xA4093822, 0x299F31D0),
     (0xD16CFE09, 0x94FDCCEB, 0x5001E420, 0x24126EA1)),
]


@pytest.mark.parametrize("ctr,key,expect", KAT)
def test_philox_known_answers(ctr, key, expect):
    out = philox4x32_10(np.array([ctr], dtype=np.uint32), np.array([key], dtype=np.uint32))[0]
    assert tuple(int(x) for x in out) == expect


def test_uniforms_in_half_open_unit_interval():
    r = np.array([0, 255, 256, 0xFFFFFFFF], dtype=np.uint32)
    u = uniforms_from_bits(r)
    assert u[0] == 2.0**-24 and u[1] == 2.0**-24 and u[2] == 2.0**-23 and u[3] == 1.0
    assert np.all(u.astype(np.float32).astype(np.float64) == u)  # exact in float32


def test_box_muller_pairs_and_counter_layout():
    # cells 4g..4g+3 come from counter block g: (z_4g)^2 + (z_4g+1)^2 = -2 ln u(r0), etc.
    seed = 0x123456789
    n = 6
    z = white_noise(n, seed).reshape(-1)
    for g in (0, 7, (n**3 - 1) // 4):
        ctr = np.array([[g, 0, 0, 0]], dtype=np.uint32)
        key = np.array([[seed & 0xFFFFFFFF, seed >> 32]], dtype=np.uint32)
        r = philox4x32_10(ctr, key)[0]
        u = uniforms_from_bits(r)
        for pair in (0, 1):
            i = 4 * g + 2 * pair
            if i + 1 < n**3:
                assert z[i] ** 2 + z[i + 1] ** 2 == pytest.approx(-2 * np.log(u[2 * pair]), rel=1e-12)
                ang = np.arctan2(z[i + 1], z[i]) % (2 * np.pi)
                assert ang == pytest.approx((2 * np.pi * u[2 * pair + 1]) % (2 * np.pi), abs=1e-9)


def test_white_noise_statistics():
    z = white_noise(64, 1).reshape(-1)
    assert abs(z.mean()) < 0.01
    assert z.var() == pytest.approx(1.0, abs=0.01)
    assert np.mean(z**4) == pytest.approx(3.0, abs=0.05)
    # different seeds give different fields, same seed the same field
    assert not np.array_equal(white_noise(8, 1), white_noise(8, 2))
    assert np.array_equal(white_noise(8, 5), white_noise(8, 5))
