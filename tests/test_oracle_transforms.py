"""Pins of the oracle transforms (Section 3.2.2, Tables 2-3, Eq. 7)."""
import os

import numpy as np
import pytest
import scipy.fft as sfft

from oracle import transforms as tr

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
TYPES = [tr.DCT1, tr.DCT3, tr.DST1, tr.DST3, tr.DFT]
SIZES = [2, 3, 4, 5, 6, 7, 8, 16, 33, 48, 97, 129]


@pytest.mark.parametrize("n", SIZES)
@pytest.mark.parametrize("t", TYPES)
def test_round_trip_and_orthogonality(t, n):
    F = tr.forward_matrix(t, n)
    B = tr.inverse_matrix(t, n)
    sel, _, _ = tr.selection(t, n)
    assert np.abs(F @ B - np.eye(len(sel))).max() < 1e-13
    proj = np.zeros((tr.node_count(t, n),) * 2)
    proj[sel, sel] = 1.0
    assert np.abs(B @ F - proj).max() < 1e-13


@pytest.mark.parametrize("n", SIZES)
@pytest.mark.parametrize("t", TYPES)
def test_against_library_routines(t, n):
    """scipy.fft's DCT/DST types I and III are twice the oracle's sums (fftw
    normalisation); the DFT is numpy's."""
    x = np.random.default_rng(n).standard_normal(tr.node_count(t, n))
    X = tr.forward_matrix(t, n) @ x
    if t == tr.DCT1:
        ref = sfft.dct(x, type=1) / 2
    elif t == tr.DCT3:
        ref = sfft.dct(x[:n], type=3) / 2
    elif t == tr.DST1:
        if n < 2:
            return
        ref = sfft.dst(x[1:n], type=1) / 2
    elif t == tr.DST3:
        ref = sfft.dst(x[1:n + 1], type=3) / 2
    else:
        ref = np.fft.fft(x)
    assert np.abs(X - ref).max() < 1e-12 * max(1.0, np.abs(ref).max())


def _extend4(q, n, s0, s1):
    """4n-periodic extension of q on [0:n] with symmetry s0 about node 0 and s1 about
    node n (+1 = S, -1 = A), Table 1 / Table 2."""
    e = {}
    for j in range(n + 1):
        e[j] = q[j]
        e[2 * n - j] = s1 * q[j]
    for j in range(0, 2 * n + 1):
        e[-j] = s0 * e[j]
    return np.array([e[j if j <= 2 * n else j - 4 * n] for j in range(4 * n)])


def _golden_table3():
    rows = {}
    with open(os.path.join(GOLDEN, "table3_selection.txt")) as fh:
        for line in fh:
            if line.startswith("#") or not line.strip():
                continue
            name, sr, s4, al = [p.strip() for p in line.split("|")]
            re_, im_ = [float(v) for v in al.split()]
            rows[name] = ([int(v) for v in sr.split()], [int(v) for v in s4.split()], complex(re_, im_))
    return rows


@pytest.mark.parametrize("t,sym", [(tr.DCT1, (1, 1)), (tr.DCT3, (1, -1)), (tr.DST1, (-1, -1)),
                                   (tr.DST3, (-1, 1))])
def test_eq7_table3_selection(t, sym):
    """Eq. 7: S_4F(DFT(q_4)) = alpha * DTT(S_R(q)) with the paper's printed Table 3
    (golden file, n = 4); DTT in fftw normalisation = 2x the oracle sums."""
    n = 4
    sr, s4f, alpha = _golden_table3()[t]
    sel, _, _ = tr.selection(t, n)
    assert list(sel) == sr
    q = np.random.default_rng(7).standard_normal(n + 1)
    q[[j for j in range(n + 1) if j not in sr]] = 0.0       # antisymmetry nodes vanish
    q4 = _extend4(q, n, *sym)
    Q4 = np.fft.fft(q4)
    X = tr.forward_matrix(t, n) @ q
    assert np.abs(Q4[s4f] - alpha * 2.0 * X).max() < 1e-12


@pytest.mark.parametrize("n", [4, 6, 9])
def test_wave_numbers_match_extended_frequencies(n):
    """q_k of each type equals 2*pi*S_4F/(4n) (Table 3)."""
    table = _golden_table3()
    for t in (tr.DCT1, tr.DCT3, tr.DST1, tr.DST3):
        _, k, q = tr.selection(t, n)
        if t == tr.DCT1:
            idx = 2 * k
        elif t == tr.DST1:
            idx = 2 * k
        else:
            idx = 2 * k + 1
        if n == 4:
            assert list(idx) == table[t][1]
        assert np.allclose(q, 2 * np.pi * idx / (4 * n))


def test_transform_type_table2():
    P, D, N = tr.BC_P, tr.BC_D, tr.BC_N
    assert tr.transform_type(N, N) == tr.DCT1
    assert tr.transform_type(N, D) == tr.DCT3
    assert tr.transform_type(D, D) == tr.DST1
    assert tr.transform_type(D, N) == tr.DST3
    assert tr.transform_type(P, P) == tr.DFT
    with pytest.raises(ValueError):
        tr.transform_type(P, N)


def test_known_closed_forms():
    """A pure cosine mode transforms to a single spectral line of height n/2."""
    n = 12
    j = np.arange(n + 1)
    for m in range(1, n):
        X = tr.forward_matrix(tr.DCT1, n) @ np.cos(np.pi * m * j / n)
        ref = np.zeros(n + 1)
        ref[m] = n / 2
        assert np.abs(X - ref).max() < 1e-12
    for m in range(n):
        x = np.sin(np.pi * j * (2 * m + 1) / (2 * n))
        X = tr.forward_matrix(tr.DST3, n) @ x
        ref = np.zeros(n)
        ref[m] = n / 2
        assert np.abs(X - ref).max() < 1e-12
