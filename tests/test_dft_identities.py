"""The algebraic identities behind the FFT-structured stages of the 32-point spot kernels, checked
in FP64 against the dense definitions (Sec. 4: spot by DFT, elongation, binning).  These are the
kernels' rewrites of the same sums -- results equal up to rounding order -- written out lane by
lane as the kernels arrange them, so a wrong sign, twiddle, index or fold fails here without a
GPU.  numpy only."""
import numpy as np
import pytest


def centred_F(N, n):
    """F[k][p] = exp(-2 pi i (k - cN)(p - cn) / N), the centred DFT of the zero-padded field."""
    cN, cn = (N - 1) / 2, (n - 1) / 2
    return np.exp(-2j * np.pi * np.outer(np.arange(N) - cN, np.arange(n) - cn) / N)


def bitrev(i, bits):
    return int(format(i, f"0{bits}b")[::-1], 2)


@pytest.mark.parametrize("n,N", [(10, 32), (8, 32), (8, 16), (6, 24)])
def test_paired_rows_of_the_first_dft_stage(n, N):
    """U = F X with the rows k and k + N/2 paired: F[k + N/2][p] = F[k][p] (-1)^p i^(n-1), so the
    lane k sums the even pupil rows p (E) and the lane k + N/2 the odd ones (O), both with row k
    of F, and U[k] = E + O, U[k + N/2] = i^(n-1) (E - O)."""
    rng = np.random.default_rng(n * 100 + N)
    F = centred_F(N, n)
    X = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
    U = F @ X
    H, rot = N // 2, 1j ** (n - 1)
    for k in range(H):
        E = sum(F[k, p] * X[p] for p in range(0, n, 2))
        O = sum(F[k, p] * X[p] for p in range(1, n, 2))
        assert np.allclose(E + O, U[k], rtol=0, atol=1e-12)
        assert np.allclose(rot * (E - O), U[k + H], rtol=0, atol=1e-12)
    # the rotation the kernels apply for (n - 1) mod 4 == 1 is +i, else -i
    assert rot == (1j if (n - 1) % 4 == 1 else -1j)


@pytest.mark.parametrize("n", [10, 8])
def test_column_quadruples_of_y_and_ta(n):
    """The FP32 kernel's Y = U F^T and Ta = I Ga^T by column quadruples m + 8j (N = 32):
    |Y[m + 8j]| = |T_j| with T = the 4-point DFT of the sums S_r over q = r mod 4, and
    Ga[d][m + 8j] = i^(jd) Ga[d][m], so Ta[d] adds (sum_j i^(jd) I[m + 8j]) Ga[d][m]."""
    N = 32
    rng = np.random.default_rng(n)
    F = centred_F(N, n)
    cN = (N - 1) / 2
    Ga = np.exp(2j * np.pi * np.outer(np.arange(n), np.arange(N) - cN) / N)
    U = rng.standard_normal(n) + 1j * rng.standard_normal(n)  # one lane's row of U
    I = np.abs(F @ U) ** 2
    Ta = Ga @ I
    Iq, Tq = np.zeros(N), np.zeros(n, complex)
    for m in range(N // 4):
        S = [sum(U[q] * F[m, q] for q in range(r, n, 4)) for r in range(4)]
        A, B, C, D = S[0] + S[2], S[0] - S[2], S[1] + S[3], S[1] - S[3]
        T = [A + C, B - 1j * D, A - C, B + 1j * D]
        iv = [abs(t) ** 2 for t in T]
        for j in range(4):
            Iq[m + 8 * j] = iv[j]
        P, M, Q, R = iv[0] + iv[2], iv[0] - iv[2], iv[1] + iv[3], iv[1] - iv[3]
        for d in range(n):
            V = {0: P + Q, 1: M + 1j * R, 2: P - Q, 3: M - 1j * R}[d % 4]
            Tq[d] += V * Ga[d, m]
    assert np.allclose(Iq, I, rtol=1e-12, atol=0)
    assert np.allclose(Tq, Ta, rtol=0, atol=1e-10 * np.abs(Ta).max())


@pytest.mark.parametrize("n", [10, 8])
def test_folded_16_point_dft_of_the_elongation_tail(n):
    """Q[iy][dx] = sum_dy G(dy, iy) M[dy][dx] with G(dy, i) = sum_{r<2} exp(-2 pi i (2 i + r - cN)
    dy / 32): G = h(dy) exp(-2 pi i i dy / 16), so Q is the 16-point DFT of h M folded modulo 16.
    Written lane by lane: the 32-point decimation-in-frequency DFT across the lanes leaves
    frequency bitrev5(lane); times ph(dy) h(dy) = sum_{r<2} exp(-2 pi i r dy / 32) (zero outside
    |dy| < n) and K~; folded with lane ^ 1; a decimation-in-time DFT across the positions
    lane >> 1; then B = Re Q G^T as in the kernel."""
    N, nd, b = 32, 16, 2
    cN = (N - 1) / 2
    rng = np.random.default_rng(7 + n)
    T = rng.standard_normal((32, n)) + 1j * rng.standard_normal((32, n))  # T[k][dx], lane k
    kt = rng.standard_normal((2 * n - 1, n)) + 1j * rng.standard_normal((2 * n - 1, n))
    Gt = np.array([[sum(np.exp(-2j * np.pi * (b * i + r - cN) * d / N) for r in range(b)) for i in range(nd)]
                   for d in range(n)])
    G = lambda dy, i: Gt[dy, i] if dy >= 0 else np.conj(Gt[-dy, i])
    # the definition
    A = {dy: sum(np.exp(2j * np.pi * (k - cN) * dy / N) * T[k] for k in range(32)) for dy in range(-(n - 1), n)}
    M = {dy: A[dy] * kt[dy + n - 1] for dy in A}
    Q = np.array([sum(G(dy, iy) * M[dy] for dy in M) for iy in range(nd)])
    B = np.real(Q @ Gt)
    # the lanes: DIF across 32 lanes (upper lane of a butterfly: sum; lower: difference times the
    # twiddle w^((lane mod h) 16 / h), w = exp(2 pi i / 32))
    x = T.copy()
    for st in range(5):
        h = 16 >> st
        y = x.copy()
        for l in range(32):
            tw = np.exp(2j * np.pi * ((l & (h - 1)) * (16 // h)) / 32) if l & h else 1
            y[l] = ((-1 if l & h else 1) * x[l] + x[l ^ h]) * tw
        x = y
    m = np.zeros_like(x)
    for l in range(32):
        f = bitrev(l, 5)
        dy = f if f < 16 else f - 32
        if -n < dy < n:
            ph = sum(np.exp(-2j * np.pi * r * dy / N) for r in range(b))
            m[l] = x[l] * ph * kt[dy + n - 1]
    v = np.array([m[l] + m[l ^ 1] for l in range(32)])
    for st in range(4):  # DIT across the positions p = lane >> 1
        q = 1 << st
        w = v.copy()
        for l in range(32):
            p = l >> 1
            lower = bool(p & q)
            tw = lambda pp: np.exp(-2j * np.pi * (pp % q) / (2 * q))
            own = v[l] * (tw(p) if lower else 1)
            pl = l ^ (2 * q)
            par = v[pl] * (tw(pl >> 1) if not lower else 1)
            w[l] = (-own if lower else own) + par
        v = w
    Qk = np.array([v[2 * iy] for iy in range(nd)])
    assert np.allclose(Qk, np.array([v[2 * iy + 1] for iy in range(nd)]))  # both lanes of a position agree
    assert np.allclose(Qk, Q, rtol=0, atol=1e-11 * np.abs(Q).max())
    assert np.allclose(np.real(Qk @ Gt), B, rtol=0, atol=1e-11 * np.abs(B).max())
    # a planted mistake -- the fold without h(dy) -- is caught
    bad = np.array([sum(np.exp(-2j * np.pi * iy * dy / 16) * M[dy] for dy in M) for iy in range(nd)])
    assert not np.allclose(bad, Q, rtol=0, atol=1e-6 * np.abs(Q).max())
