"""Pins of the track-model compression oracle (the paper's compression
section): the decompression repeats the fit and restores every fixed-point
cluster exactly; the residuals have the width the measurement and track
errors predict; the residual coding needs far fewer bits than the
fixed-point coordinates; a decoder that drifts from the encoder is caught."""
import numpy as np
import pytest

import oracle

UNIT = 0.01  # cm


@pytest.fixture(scope="module")
def case(small_event, small_oracle):
    inp = oracle.codec_input(small_oracle, small_event.clusters, UNIT)
    enc = oracle.codec(inp)
    return inp, enc


def entropy_bits(v):
    _, c = np.unique(v, return_counts=True)
    p = c / c.sum()
    return float(-(p * np.log2(p)).sum())


def test_decompression_is_exact(case, small_oracle):
    inp, enc = case
    dec = oracle.codec(inp, decode=True, ry=enc["ry"], rz=enc["rz"])
    # the codec runs wherever the refit runs: both stop at the same |sin phi|
    # limit; such tracks keep their clusters in fixed point (reading)
    assert np.array_equal(enc["ok"].astype(bool), (small_oracle["t_flags"] & oracle.F_REFIT_FAIL) == 0)
    ok = np.repeat(enc["ok"].astype(bool), np.diff(inp["off"]))
    assert ok.mean() > 0.9
    assert np.array_equal(dec["qy"][ok], inp["qy"][ok]) and np.array_equal(dec["qz"][ok], inp["qz"][ok])


def test_residuals_have_the_expected_width(case):
    """A residual is the cluster minus the track extrapolated from the
    clusters outside it: its spread is the 0.1 cm resolution widened by the
    extrapolation error, so between 1 and 2 sigma; centred on zero."""
    inp, enc = case
    first = np.zeros(len(inp["qy"]), bool)
    first[inp["off"][:-1][np.diff(inp["off"]) > 0]] = True  # the outermost cluster has no prediction yet
    ok = np.repeat(enc["ok"].astype(bool), np.diff(inp["off"])) & ~first
    for r in (enc["ry"][ok], enc["rz"][ok]):
        core = r[np.abs(r) < 100]
        assert len(core) > 0.98 * len(r)
        assert abs(np.median(core)) <= 1
        w = 0.5 * (np.percentile(core, 84.13) - np.percentile(core, 15.87)) * UNIT
        assert 0.1 <= w <= 0.2, w


def test_residual_coding_beats_fixed_point(case):
    """Entropy of the residuals and of the row steps against the fixed-point
    coordinates of the same clusters (their own entropy)."""
    inp, enc = case
    ok = np.repeat(enc["ok"].astype(bool), np.diff(inp["off"]))
    steps = -np.diff(inp["rows"])[np.diff(np.repeat(np.arange(len(inp["off"]) - 1), np.diff(inp["off"]))) == 0]
    coded = entropy_bits(enc["ry"][ok]) + entropy_bits(enc["rz"][ok]) + entropy_bits(steps)
    raw = entropy_bits(inp["qy"][ok]) + entropy_bits(inp["qz"][ok])
    assert coded < 0.6 * raw, (coded, raw)


def test_a_drifting_decoder_is_caught(case):
    """The decoder must repeat the encoder's fit: with another unit for the
    fit positions the restored clusters differ."""
    inp, enc = case
    bad = dict(inp, unit=UNIT * (1 + 1e-6))
    dec = oracle.codec(bad, decode=True, ry=enc["ry"], rz=enc["rz"])
    assert not np.array_equal(dec["qy"], inp["qy"])
