"""The pipe and SHA-2 mix probes behind the bench's roofline peaks.

A SHA-256 compression needs at least 1024 operations that only the ALU pipe
executes (rotations, shifts, three-input logic; FIPS 180-4 Sec. 6.2.2) and
a SHA-512 compression on 32-bit halves 2624, so the measured compression
rates can never beat the measured ALU-pipe rate divided by those counts.
"""
import pytest


@pytest.mark.gpu
def test_int_pipe_rates_are_plausible(hs):
    r = hs.hs_probe_int_pipes()
    assert set(r) == set(hs.PIPE_FORMS)
    for form, v in r.items():
        # a pipe takes at most 4 SMSPs x 32 lanes per clock; the interleaved
        # LOP3 + IMAD form runs on two pipes at once
        assert 1.0 < v <= (260.0 if form == "lop3+imad" else 130.0), (form, v)


@pytest.mark.gpu
def test_sha_mix_rates_respect_the_alu_pipe(hs):
    pipes = hs.hs_probe_int_pipes()
    alu = min(pipes["lop3"], pipes["shf"])
    r = hs.hs_probe_sha_mix()
    assert set(r) == set(hs.SHA_MIX_FORMS)
    c256, c512, add64 = r["sha256_per_clk_sm"], r["sha512_per_clk_sm"], r["add64_lane_ops_per_clk_sm"]
    plain = r["sha256_plain_per_clk_sm"]
    for rate in (c256, plain):
        assert 0 < rate * 1024 <= 1.05 * alu, (rate, alu)
    assert 0 < c512 * 2624 <= 1.05 * alu, (c512, alu)
    assert c512 < c256
    assert 1.0 < add64 <= 130.0, add64
