"""CPU checks of the index algebra behind the cluster kernels (256^2 and 512^2 fields split over the CTAs
of a thread-block cluster), restated in FP64 NumPy from the decomposition the kernels use:

* rows: the packed-complex row transform of length L = R M as R interleaved M-point transforms, twiddles
  W_L^(h k'), then radix-R butterflies; X[K] kept at slot R (K mod M) + K / M (digit-reversed order);
* columns: CTA b holds rows y = P a + b; an M-point transform per CTA, twiddles W_N^(b k'), then one radix-P
  stage across the CTAs; the inverse runs the same steps backwards;
* the work units of the radix-P stage (k' = u with its mirror M - u, and u = 0 with M/2) hold every mode
  pair (ky, N - ky) of a column exactly once, in units of equal size, so the pairwise s-draw and the
  Hermitian edge column can be done inside a unit and every thread of the cluster gets the same share;
* and the shared-memory transform of the global-memory kernels (R-point DFTs across S strided
  subsequences, then S-point transforms).

No GPU: these are the identities the kernels rely on, checked against numpy.fft.
"""
import numpy as np
import pytest

GEOMETRIES = [(256, 64), (512, 32), (512, 64)]  # (N, M): M rows per CTA, P = N / M CTAs


def _units(N, M):
    """Mode pairs (ky1, ky2) of one column as the radix-P stage enumerates them, unit by unit: unit u in
    [0, M/2) holds the butterflies u and v = M - u (u = 0 with v = M/2, the two half-size ones)."""
    P = N // M
    out, sizes = [], []
    for u in range(M // 2):
        v = M // 2 if u == 0 else M - u
        if u == 0:
            pairs = [(0, N // 2)] + [(M * m, N - M * m) for m in range(1, P // 2)] + \
                    [(M // 2 + M * m, N - M // 2 - M * m) for m in range(P // 2)]
        else:
            pairs = [(u + M * m, N - u - M * m) for m in range(P // 2)] + \
                    [(v + M * m, N - v - M * m) for m in range(P // 2)]
        # every mode of a pair belongs to the unit's butterflies u or v
        for a, b in pairs:
            assert a % M in (u, v % M) and b % M in (u, v % M)
        out.extend(pairs)
        sizes.append(len(pairs))
    assert sizes == [P] * (M // 2)             # equal units: the cluster's threads get equal shares
    return out


@pytest.mark.parametrize("N,M", GEOMETRIES)
def test_units_cover_every_mode_pair_once(N, M):
    pairs = _units(N, M)
    modes = sorted(k for p in pairs for k in p)
    assert modes == list(range(N))                         # every ky exactly once
    for a, b in pairs:
        assert a < N // 2 and (b == (N - a) % N or (a == 0 and b == N // 2))   # Hermitian partner
    # the s-draw's Philox group of a pair is its ky1 (< N/2): groups are distinct
    assert len({a for a, _ in pairs}) == len(pairs) == N // 2


def _row_forward(z, M):
    """Packed-complex row transform of length L = R M by the row threads' decomposition; returns the
    digit-reversed slots."""
    L = z.size
    R = L // M
    slots = np.empty(L, complex)
    for h in range(R):                                     # thread h: every R-th slot
        Z = np.fft.fft(z[h::R])                            # M-point transform
        slots[R * np.arange(M) + h] = Z * np.exp(-2j * np.pi * h * np.arange(M) / L)
    out = np.empty(L, complex)
    for k in range(M):                                     # radix-R butterflies over the R threads
        t = slots[R * k + np.arange(R)]
        for m in range(R):
            K = k + M * m
            out[R * (K % M) + K // M] = np.sum(t * np.exp(-2j * np.pi * np.arange(R) * m / R))
    return out


@pytest.mark.parametrize("N,M", GEOMETRIES)
def test_row_transform_in_digit_reversed_slots(N, M):
    rng = np.random.default_rng(N + M)
    L = N // 2
    z = rng.standard_normal(L) + 1j * rng.standard_normal(L)
    slots = _row_forward(z, M)
    ref = np.fft.fft(z)
    R = L // M
    for K in range(L):
        assert abs(slots[R * (K % M) + K // M] - ref[K]) < 1e-9 * np.sqrt(L)


def _column_forward(x, M):
    """Column transform of length N = P M: CTA b holds x[P a + b]; M-point transforms, twiddles
    W_N^(b k'), then the radix-P stage across CTAs."""
    N = x.size
    P = N // M
    Y = np.array([np.fft.fft(x[b::P]) * np.exp(-2j * np.pi * b * np.arange(M) / N) for b in range(P)])
    X = np.empty(N, complex)
    for k in range(M):
        for m in range(P):
            X[k + M * m] = np.sum(Y[:, k] * np.exp(-2j * np.pi * np.arange(P) * m / P))
    return X, Y


def _column_inverse(X, M):
    """The inverse steps: radix-P stage back to CTA b, untwiddle W_N^(-b k'), inverse M-point transforms
    (unnormalised, as the kernels)."""
    N = X.size
    P = N // M
    x = np.empty(N, complex)
    for b in range(P):
        y = np.array([np.sum(X[k + M * np.arange(P)] * np.exp(2j * np.pi * b * np.arange(P) / P))
                      for k in range(M)])
        y = y * np.exp(2j * np.pi * b * np.arange(M) / N)
        x[b::P] = np.fft.ifft(y) * M
    return x


@pytest.mark.parametrize("N,M", GEOMETRIES)
def test_column_split_over_cluster(N, M):
    rng = np.random.default_rng(3 * N + M)
    x = rng.standard_normal(N) + 1j * rng.standard_normal(N)
    X, _ = _column_forward(x, M)
    assert np.max(np.abs(X - np.fft.fft(x))) < 1e-9 * N
    back = _column_inverse(X, M)
    assert np.max(np.abs(back - N * x)) < 1e-8 * N   # unnormalised round trip = N


def test_table_rows_of_a_cta_are_contiguous():
    """The pixel tables' row order for the clusters: row y = P a + b at index b M + a, so CTA b's rows
    occupy [b M, b M + M) and the permutation is a bijection."""
    for N, M in GEOMETRIES:
        P = N // M
        idx = [(y % P) * (N // P) + y // P for y in range(N)]
        assert sorted(idx) == list(range(N))
        for b in range(P):
            assert sorted(idx[y] for y in range(b, N, P)) == list(range(b * M, b * M + M))


@pytest.mark.parametrize("L,S", [(128, 16), (256, 16), (512, 16), (1024, 16), (512, 64), (1024, 32)])
def test_global_memory_transform_decomposition(L, S):
    """The shared-memory transform of the global-memory kernels: an R-point DFT across the S strided
    subsequences with twiddles W_L^(q n), then an S-point FFT of each subsequence q, output k at position
    q + R k (L = R S; decimation in frequency)."""
    rng = np.random.default_rng(L + S)
    v = rng.standard_normal(L) + 1j * rng.standard_normal(L)
    R = L // S
    w = v.copy()
    for n in range(S):                       # step A: tasks (vector, n)
        a = w[n + S * np.arange(R)]
        A = np.array([np.sum(a * np.exp(-2j * np.pi * np.arange(R) * q / R)) for q in range(R)])
        w[n + S * np.arange(R)] = A * np.exp(-2j * np.pi * np.arange(R) * n / L)
    out = np.empty(L, complex)
    for q in range(R):                       # step C: one S-point transform per thread
        out[q + R * np.arange(S)] = np.fft.fft(w[S * q + np.arange(S)])
    assert np.max(np.abs(out - np.fft.fft(v))) < 1e-9 * L


@pytest.mark.parametrize("L,S", [(1024, 16), (512, 16)])
def test_global_memory_transform_split_step_a(L, S):
    """The same transform when the R-point DFTs of step A are split in two shared-memory passes
    (R = R1 R2, m = m2 + R2 m1, q = q1 + R1 q2): R1-point DFTs over m1 twiddled by w_R^(m2 q1), then
    R2-point DFTs over m2 twiddled by W_L^(q n), as the kernels do when one or two warps would carry
    step A alone."""
    rng = np.random.default_rng(L + 7)
    v = rng.standard_normal(L) + 1j * rng.standard_normal(L)
    R = L // S
    R1, R2 = 8, R // 8
    w = v.copy()
    for n in range(S):                       # A1: tasks (n, m2)
        for m2 in range(R2):
            idx = n + S * (m2 + R2 * np.arange(R1))
            B = np.array([np.sum(w[idx] * np.exp(-2j * np.pi * np.arange(R1) * q1 / R1)) for q1 in range(R1)])
            w[idx] = B * np.exp(-2j * np.pi * m2 * np.arange(R1) / R)
    w2 = w.copy()
    for n in range(S):                       # A2: tasks (n, q1)
        for q1 in range(R1):
            b = w[n + S * (np.arange(R2) + R2 * q1)]
            C = np.array([np.sum(b * np.exp(-2j * np.pi * np.arange(R2) * q2 / R2)) for q2 in range(R2)])
            q = q1 + R1 * np.arange(R2)
            w2[n + S * q] = C * np.exp(-2j * np.pi * q * n / L)
    out = np.empty(L, complex)
    for q in range(R):                       # step C
        out[q + R * np.arange(S)] = np.fft.fft(w2[S * q + np.arange(S)])
    assert np.max(np.abs(out - np.fft.fft(v))) < 1e-9 * L


@pytest.mark.parametrize("N,M", GEOMETRIES)
def test_mode_tables_in_slot_order(N, M):
    """The cluster kernels' mode tables (s-draw coefficients, P): half-spectrum entry (ky, kx) at
    ky L + t with t = (kx mod M) R + kx / M, the slot whose digit-reversed index K(t) = (t mod R) M + t / R
    is kx, and the Nyquist column kx = W/2 at H L + ky; a bijection onto [0, H (W/2 + 1))."""
    H = W = N
    L = W // 2
    R = L // M
    pos = []
    for ky in range(H):
        for kx in range(L + 1):
            if kx < L:
                t = (kx % M) * R + kx // M
                assert (t % R) * M + t // R == kx
                pos.append(ky * L + t)
            else:
                pos.append(H * L + ky)
    assert sorted(pos) == list(range(H * (L + 1)))


def test_row_swizzle_of_the_512_cluster_rows_is_conflict_free():
    """512^2 with 32 rows per CTA (R = 8 threads per row): the slot map s -> s ^ ((s >> 3) & 3) used for the
    staged rows is a bijection, and a half-warp's float2 reads (4 rows x 4 threads of a row, row stride
    L + R/2) fall in 16 distinct bank pairs both in the strided M-point pass (slot R i + h) and in the
    radix-R butterflies (slot R u + j, u = h + R k)."""
    def phys(s):
        return s ^ ((s >> 3) & 3)
    L, R, M = 256, 8, 32
    SP = L + R // 2
    assert sorted(phys(s) for s in range(L)) == list(range(L))
    rows_per_warp = 32 // R
    for i in range(M):
        banks = {(a * SP + phys(R * i + h)) % 16 for a in range(rows_per_warp) for h in range(4)}
        assert len(banks) == 16
    for k in range((M // 2 + 1 + R - 1) // R):
        for j in range(R):
            banks = {(a * SP + phys(R * (h + R * k) + j)) % 16 for a in range(rows_per_warp) for h in range(4)}
            assert len(banks) == 16
