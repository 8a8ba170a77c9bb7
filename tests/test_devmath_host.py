"""The library's own spectral densities and Bessel sequences (csrc/devmath.cuh, compiled
for the host by tests/devmath_harness.cpp) against the oracle's direct interface solve
and against scipy, on the CPU.

Sigma_c(lambda) (Sec. 3.1, Cases I-III on the recursions of eqs. Rellrecursionup,
Rellrecursiondown and generaltransmission, referenced at the interfaces) must equal the
amplitude of the same (arrival, departure) pair of the oracle's 2L x 2L solve, which
uses none of those recursions.
"""

import os
import shutil
import subprocess

import numpy as np
import pytest
from scipy.special import hankel1, jv

from oracle import core
from workloads import Medium

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
WORK = os.path.join(ROOT, "tests", "_build")   # git-ignored
CSRC = os.path.join(ROOT, "paper_2511_12450_gb300", "csrc")


@pytest.fixture(scope="module")
def harness():
    cxx = shutil.which("g++") or shutil.which("c++")
    inc = None
    for d in [os.environ.get("CUDA_HOME", ""), "/usr/local/cuda"]:
        if d and os.path.exists(os.path.join(d, "include", "cuda_runtime.h")):
            inc = os.path.join(d, "include")
    if cxx is None or inc is None:
        pytest.skip("needs a C++ compiler and the CUDA headers")
    os.makedirs(WORK, exist_ok=True)
    exe = os.path.join(WORK, "devmath_harness")
    res = subprocess.run([cxx, "-std=c++17", "-O2", "-ffp-contract=off", "-Wall", "-I", inc, "-I", CSRC,
                          os.path.join(ROOT, "tests", "devmath_harness.cpp"), "-o", exe],
                         capture_output=True, text=True)
    assert res.returncode == 0, res.stderr
    return exe


def _call(exe, mode, payload: bytes, tag: str) -> bytes:
    src = os.path.join(WORK, f"devmath_in_{tag}.bin")
    dst = os.path.join(WORK, f"devmath_out_{tag}.bin")
    with open(src, "wb") as f:
        f.write(payload)
    res = subprocess.run([exe, mode, src, dst], capture_output=True, text=True, timeout=300)
    assert res.returncode == 0, res.stderr
    out = open(dst, "rb").read()
    os.unlink(src)
    os.unlink(dst)
    return out


def _sigma(exe, med, queries, tag):
    nl = med.n_layers
    buf = [np.array([nl], np.int32).tobytes(), np.asarray(med.interfaces, np.float64).tobytes(),
           np.asarray(med.k, np.float64).tobytes(), np.asarray(med.eta, np.float64).tobytes(),
           np.array([len(queries)], np.int32).tobytes()]
    for lf, a, ls, b, lam in queries:
        buf.append(np.array([lf, a, ls, b], np.int32).tobytes())
        buf.append(np.array([lam.real, lam.imag], np.float64).tobytes())
    out = _call(exe, "sigma", b"".join(buf), tag)
    return np.frombuffer(out, np.complex128)


MEDIA = [
    Medium(interfaces=[0.0], k=[2.0, 4.0], eta=[1.0, 2.0]),
    Medium(interfaces=[0.0, -2.0], k=[4.0, 6.0, 8.0], eta=[1.0, 2.0, 3.0]),                 # C2's stack
    Medium(interfaces=[0.0, -0.9, -1.7], k=[3.0, 5.5, 2.0, 4.2], eta=[1.0, 2.5, 1.3, 3.0]),
    Medium(interfaces=[0.0, -1.0, -2.0, -3.0, -4.0], k=[1.2, 2.3, 4.5, 6.1, 7.7, 10.0],      # Example 2's stack
           eta=[1.1, 2.3, 3.4, 4.6, 5.0, 6.6]),
]


@pytest.mark.parametrize("mi", range(len(MEDIA)))
def test_reaction_densities_equal_the_direct_interface_solve(harness, mi):
    med = MEDIA[mi]
    L = med.n_layers - 1
    kmax = float(np.max(med.k))
    rng = np.random.default_rng(40 + mi)
    # the kernels' lambda range: the fourth-quadrant detour, the real axis past k_max
    # (evanescent in every layer) and points along the rays into the lower half plane
    lams = np.concatenate([
        rng.uniform(0.0, 1.2 * kmax + 1.0, 12) - 1j * rng.uniform(0.0, 0.5, 12),
        rng.uniform(kmax + 0.1, 4.0 * kmax + 20.0, 6) + 0j,
        (1.2 * kmax + 1.0) + rng.uniform(0.0, 30.0, 6) * np.exp(-1j * rng.uniform(0.0, 1.4, 6)),
    ])
    queries, want = [], []
    for lf in range(L + 1):
        for ls in range(L + 1):
            S = core.spectral_amp(med, lf, ls, lams)   # columns 2 a + b: (arrival a, departure b)
            for a in (0, 1):
                for b in (0, 1):
                    # components that cannot exist (no wave arrives up in the bottom layer, ...)
                    if (a == 0 and lf == L) or (a == 1 and lf == 0) or (b == 0 and ls == 0) or (b == 1 and ls == L):
                        continue
                    for i, lam in enumerate(lams):
                        queries.append((lf, a, ls, b, lam))
                        want.append(S[i, 2 * a + b])
    got = _sigma(harness, med, queries, f"s{mi}")
    want = np.asarray(want)
    err = np.abs(got - want) / np.maximum(np.abs(want), 1e-300)
    big = np.abs(want) > 1e-250   # deep evanescent values underflow on both sides alike
    assert big.sum() > 0.9 * len(want)
    assert np.max(err[big]) <= 1e-12, float(np.max(err[big]))
    assert np.all(np.abs(got[~big]) <= 1e-200)


def test_bessel_and_hankel_sequences_against_scipy(harness):
    # J_0..J_p by Miller's recurrence (P2M / L2P) and H_0..H_p by forward recurrence (M2L
    # tables), over the argument range of the expansions: k rho from 1e-3 to ~kR of the
    # coarsest levels
    p = 80
    x = np.concatenate([np.geomspace(1e-3, 1.0, 10), np.linspace(1.5, 120.0, 30)])
    out = _call(harness, "bessel", np.array([x.size, p], np.int32).tobytes() + x.tobytes(), "bes")
    nJ = x.size * (p + 1)
    J = np.frombuffer(out, np.float64, nJ).reshape(x.size, p + 1)
    H = np.frombuffer(out, np.complex128, nJ, offset=8 * nJ).reshape(x.size, p + 1)
    n = np.arange(p + 1)
    Jref = jv(n[None, :], x[:, None])
    # Miller's algorithm normalises with J_0 + 2 sum J_2k = 1: absolute accuracy near
    # rounding of O(1) values (measured 7e-15) plus relative accuracy of the small
    # high orders; a pure relative test would fail only near the zeros of J_n
    dJ = np.abs(J - Jref)
    assert np.all(dJ <= 1e-12 * np.abs(Jref) + 1e-14), float(np.max(dJ / (1e-12 * np.abs(Jref) + 1e-14)))
    # H_n: relative accuracy while |H_n| stays finite (the forward recurrence follows Y_n).
    # On the host the seeds H_0, H_1 come from the C library's j0/y0/j1/y1, on the device
    # from CUDA's: this checks the recurrence, measured 1e-13
    Href = hankel1(n[None, :], x[:, None])
    ok = np.isfinite(Href) & (np.abs(Href) < 1e250)
    errH = np.abs(H - Href) / np.abs(Href)
    assert np.max(errH[ok]) <= 1e-12, float(np.max(errH[ok]))


def test_free_space_entries_equal_the_oracles(harness):
    # single layer (i/4) H_0(k r) and the combined field's n_e . grad_{c_e} (i/4) H_0 - i k (i/4) H_0
    # (Sec. 3.3; the combined-field reading), (dx, dy) = c_e - c_i, against oracle/nystrom.gf and
    # oracle/combined.grad_free
    from oracle import combined as ocf
    from oracle import nystrom as onys

    rng = np.random.default_rng(50)
    m = 400
    k = rng.uniform(1.0, 12.0, m)
    r = np.geomspace(1e-4, 30.0, m)
    th = rng.uniform(0, 2 * np.pi, m)
    dx, dy = r * np.cos(th), r * np.sin(th)
    ph = rng.uniform(0, 2 * np.pi, m)
    nx, ny = np.cos(ph), np.sin(ph)
    for cf in (0.0, 1.0):
        q = np.stack([k, dx, dy, np.full(m, cf), nx, ny], axis=1)
        out = _call(harness, "free", np.array([m], np.int32).tobytes() + q.tobytes(), f"free{int(cf)}")
        got = np.frombuffer(out, np.complex128)
        g = np.array([onys.gf(k[i], r[i]) for i in range(m)])
        if cf:
            ce = np.stack([dx, dy], axis=1)
            grad = [ocf.grad_free(k[i], ce[i:i + 1], np.zeros((1, 2))) for i in range(m)]
            want = np.array([nx[i] * gx[0, 0] + ny[i] * gy[0, 0] for i, (gx, gy) in enumerate(grad)]) - 1j * k * g
        else:
            want = g
        err = np.abs(got - want) / np.abs(want)
        assert np.max(err) <= 1e-12, (cf, float(np.max(err)))


def test_diagonal_entries_equal_the_oracles(harness):
    # I^s = [i/4 - (1/2 pi)(gamma + ln(k w / 4) - 1)] w (eq. ApproximateComputation), and the
    # combined field's 1/2 - i k I^s
    from oracle import nystrom as onys

    rng = np.random.default_rng(51)
    m = 200
    k = rng.uniform(1.0, 12.0, m)
    w = np.geomspace(1e-5, 0.5, m)
    for cf in (0.0, 1.0):
        q = np.stack([k, w, np.full(m, cf)], axis=1)
        out = _call(harness, "self", np.array([m], np.int32).tobytes() + q.tobytes(), f"self{int(cf)}")
        got = np.frombuffer(out, np.complex128)
        Is = onys.self_term(k, w)
        want = 0.5 - 1j * k * Is if cf else Is
        assert np.max(np.abs(got - want) / np.abs(want)) <= 1e-13
