"""CPU models of the data movement of two GPU kernels, checked before they
ran on a GPU and kept as documentation of their index algebra.

1. The tensor-core product (tc_gemm.cu): slices stored as
   [term][k/8][slice][row][8 k]; one 5-D TMA box (8 k, R rows, 7 slices,
   2 k groups, 1 term) copied in box order into shared memory; operands
   read through K-major no-swizzle descriptors (start, LBO = next 8-wide k
   group, SBO = 128 B = next 8-row group); ten MMAs per 16-wide stage, A
   slice s against the consecutive B rows of slices t <= 8 - s into TMEM
   columns 64 (s - 1) + ...  The model checks that these ten products add
   every slice product A_s B_t into accumulator g = s + t (the 28 Ozaki
   products), using the kernel's constants.
2. The two-sided Jacobi leaf solver (svd.cu) in column-only form: kernel 1
   rotates each pair's two columns (angle from g_pp, g_qq, g_pq), kernel 2
   applies every pair's row rotation to each CTA's own columns, the idle
   column of an odd size included.  The model converges to the
   eigendecomposition for even and odd sizes, real and complex.
"""
import numpy as np
import pytest

S, BM, BN, KS = 7, 128, 64, 16


def _to_global(X, rpad, kpad, nbj):
    out = np.zeros(X.size, np.int64)
    for bj in range(nbj):
        for s in range(S):
            for i in range(rpad):
                for k in range(kpad):
                    out[(((bj * (kpad // 8) + k // 8) * S + s) * rpad + i) * 8 + k % 8] = X[bj, s, i, k]
    return out


def _tma_box(G, rpad, kpad, row0, kg0, bj, R):
    sm = np.zeros(8 * R * S * 2, np.int64)
    o = 0
    for d3 in range(2):
        for d2 in range(S):
            for d1 in range(R):
                for d0 in range(8):
                    gi = d0 + 8 * (row0 + d1) + 8 * rpad * d2 + 8 * rpad * S * (kg0 + d3) + 8 * rpad * S * (kpad // 8) * bj
                    sm[o] = G[gi]
                    o += 1
    return sm


def _fetch(sm, start_b, lbo_b, sbo_b, rows, K):
    M = np.zeros((rows, K), np.int64)
    for r in range(rows):
        for k in range(K):
            off = start_b + (r // 8) * sbo_b + (k // 8) * lbo_b + (r % 8) * 16 + (k % 8) * 2
            M[r, k] = sm[off // 2]
    return M


def test_tensor_core_stage_forms_the_28_slice_products():
    rng = np.random.default_rng(0)
    rpadA, rpadB, kpad, nbj = 256, 128, 64, 2
    A = rng.integers(-100, 100, (nbj, S, rpadA, kpad)).astype(np.int64)
    B = rng.integers(-100, 100, (nbj, S, rpadB, kpad)).astype(np.int64)
    GA, GB = _to_global(A, rpadA, kpad, nbj), _to_global(B, rpadB, kpad, nbj)
    m0, n0, k0, bj = 128, 64, 32, 1
    sa = _tma_box(GA, rpadA, kpad, m0, k0 // 8, bj, BM)
    sb = _tma_box(GB, rpadB, kpad, n0, k0 // 8, bj, BN)
    LBO_A, LBO_B = S * BM * 16, S * BN * 16
    acc = np.zeros((BM, 512), np.int64)
    nmma = 0
    for s1 in range(1, S + 1):
        ntot = BN * (8 - s1)
        for c0 in range(0, ntot, 256):
            nn = min(256, ntot - c0)
            Aop = _fetch(sa, (s1 - 1) * BM * 16, LBO_A, 128, BM, KS)
            Bop = _fetch(sb, c0 * 16, LBO_B, 128, nn, KS)
            acc[:, BN * (s1 - 1) + c0: BN * (s1 - 1) + c0 + nn] += Aop @ Bop.T
            nmma += 1
    want = np.zeros((BM, 512), np.int64)
    for s in range(1, S + 1):
        for t in range(1, 9 - s):
            g = s + t
            want[:, 64 * (g - 2): 64 * (g - 1)] += (A[bj, s - 1, m0:m0 + BM, k0:k0 + KS] @
                                                    B[bj, t - 1, n0:n0 + BN, k0:k0 + KS].T)
    assert nmma == 10
    assert np.max(np.nonzero(want.any(0))) == 447  # 7 accumulators x 64 columns
    assert np.array_equal(acc, want)


def _pairs(npad, r):
    out = [(npad - 1, r)]
    for k in range(1, npad // 2):
        out.append(((r + k) % (npad - 1), (r - k + npad - 1) % (npad - 1)))
    return [(min(a, b), max(a, b)) for a, b in out]


def _jacobi_column_form(B, sweeps=30):
    n = B.shape[0]
    B = B.copy()
    V = np.eye(n, dtype=B.dtype)
    npad = n + (n & 1)
    nrm = np.linalg.norm(B)
    for _ in range(sweeps):
        rot = 0
        for r in range(npad - 1):
            cs = {}
            B1 = B.copy()
            for p, q in _pairs(npad, r):  # kernel 1: own columns only
                if q >= n:
                    continue
                g = abs(B[p, q])
                if g <= 2.0 ** -53 * nrm:
                    cs[(p, q)] = (1.0, 0.0, 1.0)
                    continue
                ph = B[p, q] / g
                zeta = (B[q, q].real - B[p, p].real) / (2 * g)
                t = (1.0 if zeta >= 0 else -1.0) / (abs(zeta) + np.sqrt(1 + zeta * zeta))
                c = 1 / np.sqrt(1 + t * t)
                s = c * t
                cs[(p, q)] = (c, s, ph)
                rot += 1
                for M, M1 in ((B, B1), (V, V)):
                    x, y = M[:, p].copy(), M[:, q] * np.conj(ph)
                    M1[:, p] = c * x - s * y
                    M1[:, q] = s * x + c * y
            B2 = B1.copy()
            for p, q in _pairs(npad, r):  # kernel 2: every pair's rows, on this CTA's columns
                for col in [x for x in (p, q) if x < n]:
                    for (i, j), (c, s, ph) in cs.items():
                        x, y = B1[i, col], B1[j, col] * ph
                        B2[i, col] = c * x - s * y
                        B2[j, col] = s * x + c * y
            B = B2
        if rot == 0:
            break
    return np.real(np.diag(B)), V


@pytest.mark.parametrize("n,cplx", [(7, False), (16, False), (9, True), (12, True)])
def test_two_sided_jacobi_column_form_converges(n, cplx):
    rng = np.random.default_rng(n)
    X = rng.standard_normal((n, n)) + (1j * rng.standard_normal((n, n)) if cplx else 0)
    A = X + X.conj().T
    lam, V = _jacobi_column_form(A)
    assert np.max(np.abs(np.sort(lam) - np.linalg.eigvalsh(A))) <= 1e-13 * n
    assert np.linalg.norm(A @ V - V * lam) <= 1e-13 * n
    assert np.linalg.norm(V.conj().T @ V - np.eye(n)) <= 1e-13 * n


# ---- one-CTA shared-memory Jacobi leaf (svd.cu, leaf_smem_kernel): every
# round computes the rotations of its disjoint pairs from G, applies them to
# the columns of G and V, then to the rows of G (three phases separated by
# barriers); a sweep with no rotation ends the iteration.  The model keeps
# the kernel's column-major indexing and round-robin pair order.
def _smem_leaf_model(B, max_sweeps=40):
    n = B.shape[0]
    cplx = np.iscomplexobj(B)
    G = np.array(B, dtype=complex if cplx else float).flatten(order="F")
    W = np.eye(n, dtype=G.dtype).flatten(order="F")
    thr = 2.0 ** -53 * max(np.sqrt(np.sum(np.abs(G) ** 2)), 1e-300)
    npad = n + (n & 1)
    sweeps = 0
    for sweep in range(max_sweeps):
        nrot = 0
        for r in range(npad - 1):
            pairs = []
            for k in range(npad // 2):
                if k == 0:
                    p, q = npad - 1, r
                else:
                    p, q = (r + k) % (npad - 1), (r - k + npad - 1) % (npad - 1)
                if p > q:
                    p, q = q, p
                if q >= n:
                    continue
                gpp, gqq, gpq = G[p + p * n].real, G[q + q * n].real, G[p + q * n]
                g = abs(gpq)
                if not g > thr:
                    continue
                ph = gpq / g
                zeta = (gqq - gpp) / (2.0 * g)
                t = (1.0 if zeta >= 0 else -1.0) / (abs(zeta) + np.sqrt(1.0 + zeta * zeta))
                c = 1.0 / np.sqrt(1.0 + t * t)
                pairs.append((p, q, c, c * t, ph))
                nrot += 1
            for (p, q, c, s, ph) in pairs:  # columns of G and V
                for X in (G, W):
                    x = X[p * n:(p + 1) * n].copy()
                    y = X[q * n:(q + 1) * n] * np.conj(ph)
                    X[p * n:(p + 1) * n] = c * x - s * y
                    X[q * n:(q + 1) * n] = s * x + c * y
            for (p, q, c, s, ph) in pairs:  # rows of G
                x = G[p::n].copy()
                y = G[q::n] * ph
                G[p::n] = c * x - s * y
                G[q::n] = s * x + c * y
        sweeps += 1
        if nrot == 0:
            break
    lam = np.array([G[j + j * n].real for j in range(n)])
    return lam, W.reshape((n, n), order="F"), sweeps


@pytest.mark.parametrize("n,cplx", [(1, False), (2, False), (7, False), (33, True), (64, False), (64, True)])
def test_smem_leaf_model_matches_lapack(n, cplx):
    rng = np.random.default_rng(n + 100 * cplx)
    A = rng.standard_normal((n, n)) + (1j * rng.standard_normal((n, n)) if cplx else 0)
    B = (A + A.conj().T) / 2
    lam, V, sweeps = _smem_leaf_model(B)
    u = 2.0 ** -53
    nb = np.linalg.norm(B)
    assert sweeps < 40
    assert np.max(np.abs(np.sort(lam) - np.linalg.eigvalsh(B))) <= 20 * n * u * max(nb, 1.0)
    assert np.linalg.norm(V.conj().T @ V - np.eye(n)) <= 20 * n * u
    assert np.linalg.norm(B @ V - V * lam) <= 20 * n * u * max(nb, 1.0)
