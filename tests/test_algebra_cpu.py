"""CPU models of the reformulations the CUDA path makes of the paper's computation.

The kernels do not compute Eq. 2's log-determinants and the diagonal of G = A^-1 the textbook
way: they run a blocked Gauss-Jordan sweep written as rank-nb updates M <- mask(M) - F W, skip
the pivot search in the blocks that provably need none, update only the lower triangle of the
symmetric blocks, merge two elimination steps into one K = 2 nb update, refine diag(G) with one
Newton step, read that refinement from the lower triangle alone, and contract in BF16x3.  Each
test below writes one of those reformulations out in a few lines of FP64 numpy (test code
only, sharing nothing with the CUDA sources) and checks it against the plain definition on the
blocks of the paper's ionic Hubbard model (Eq. 1, assembled by the oracle): numpy's inverse and
slogdet, an unblocked partially pivoted LU, the full quadratic form, or an exact closed form.
So a wrong sign, mask, index range or bound in the design fails here, on the CPU.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2311_04435_gb300 import inputs


def block_matrix(L, n, sigma, T=0.1, U=4.0, delta=1.0, mu=0.0, seed=3, scale=1.0):
    """A_{n,sigma} = (i w_n + mu) I - H_sigma(phi) (Eq. 2) for a seeded random field."""
    p = oracle.make_params(L, n + 1, U=U, T=T, delta=delta, mu=mu)
    phi = inputs.random_phi(seed, L * L, scale)
    H = oracle.hamiltonian(p, phi, sigma)
    w = (2 * n + 1) * math.pi * T
    return (1j * w + mu) * np.eye(L * L) - H, w


def lu_pivots_unblocked(A):
    """Textbook LU with partial pivoting (row of largest |z|^2, first on ties): the row chosen
    at every column and ln|det A| = sum ln|u_kk|."""
    M = A.astype(complex).copy()
    N = M.shape[0]
    piv, ld = [], 0.0
    for k in range(N):
        r = k + int(np.argmax(np.abs(M[k:, k]) ** 2))
        piv.append(r)
        M[[k, r]] = M[[r, k]]
        ld += math.log(abs(M[k, k]))
        M[k + 1:, k] /= M[k, k]
        M[k + 1:, k + 1:] -= np.outer(M[k + 1:, k], M[k, k + 1:])
    return piv, ld


def gj_factors(M, k0, kb):
    """F and W of one Gauss-Jordan step over K = [k0, k0 + kb): with T = inv(M_KK),
    F[i] = M[i, K] T outside K and -T inside, W[K, j] = M[K, j] outside K and e_j inside."""
    N = M.shape[0]
    K = slice(k0, k0 + kb)
    T = np.linalg.inv(M[K, K])
    F = M[:, K] @ T
    F[K] = -T
    W = M[K, :].copy()
    W[:, K] = np.eye(kb)
    return F, W


def masked(M, k0, kb):
    """mask(M): the rows and the columns of K set to zero."""
    R = M.copy()
    R[k0:k0 + kb, :] = 0
    R[:, k0:k0 + kb] = 0
    return R


def gj_step(M, k0, kb):
    F, W = gj_factors(M, k0, kb)
    return masked(M, k0, kb) - F @ W


@pytest.mark.parametrize("L,n,nb", [(6, 0, 4), (6, 1, 8), (8, 0, 16), (8, 2, 12)])
def test_pivoted_blocked_gauss_jordan_is_the_inverse_with_the_lu_pivots(L, n, nb):
    """The pivoted path: per step a partially pivoted LU of the nb-wide panel of the Schur
    complement (rows k0..N-1 of the tableau's columns K) picks the interchanges, which are
    applied to whole tableau rows, then one mask(M) - F W sweep over K.  The sweep leaves
    R = (P A)^{-1}, so A^{-1}[i, perm[r]] = R[i, r]; the panel's pivots are those of the
    unblocked LU and sum ln|u_kk| is ln|det A|.  Low frequencies (w_n <= 4|t|), where
    interchanges happen; a ragged last step where nb does not divide N."""
    A, _ = block_matrix(L, n, +1, T=0.02, delta=0.2, scale=0.5)
    N = A.shape[0]
    M = A.copy()
    perm = np.arange(N)
    piv_blocked, ld = [], 0.0
    for k0 in range(0, N, nb):
        kb = min(nb, N - k0)
        P = M[k0:, k0:k0 + kb].copy()  # the panel: Schur complement columns below the swept rows
        for c in range(kb):
            r = c + int(np.argmax(np.abs(P[c:, c]) ** 2))
            piv_blocked.append(k0 + r)
            P[[c, r]] = P[[r, c]]
            M[[k0 + c, k0 + r]] = M[[k0 + r, k0 + c]]
            perm[[k0 + c, k0 + r]] = perm[[k0 + r, k0 + c]]
            ld += math.log(abs(P[c, c]))
            P[c + 1:, c] /= P[c, c]
            P[c + 1:, c + 1:] -= np.outer(P[c + 1:, c], P[c, c + 1:])
        M = gj_step(M, k0, kb)
    X = np.empty_like(M)
    X[:, perm] = M
    piv_ref, ld_ref = lu_pivots_unblocked(A)
    assert piv_blocked == piv_ref
    assert any(p != k for k, p in enumerate(piv_ref))  # the case really interchanges rows
    sign, ld_np = np.linalg.slogdet(A)
    assert ld == pytest.approx(ld_np, rel=1e-13, abs=1e-12)
    assert ld_ref == pytest.approx(ld_np, rel=1e-13, abs=1e-12)
    Ainv = np.linalg.inv(A)
    assert np.max(np.abs(X - Ainv)) <= 1e-12 * np.max(np.abs(Ainv))


@pytest.mark.parametrize("L", [2, 4, 6])
@pytest.mark.parametrize("scale", [0.5, 4.0])
def test_blocks_above_four_t_keep_the_diagonal_pivot(L, scale):
    """Blocks with w_n > 4|t| skip the pivot search.  |A_jj| >= w_n exceeds the off-diagonal
    column sum 4|t| (two bonds of 2t each for L = 2), a strict column dominance that every
    Schur complement keeps, so partial pivoting picks the diagonal at every column, with a
    strict margin, whatever the field and the ionic potential.  The lowest such frequency at
    T = 0.1 (n = 6, w = 4.08) and a far one; fields up to 4 in magnitude."""
    for n in (6, 40):
        A, w = block_matrix(L, n, -1, delta=2.0, scale=scale, seed=11 + L)
        assert w > 4.0
        M = A.copy()
        N = M.shape[0]
        for k in range(N):
            col = np.abs(M[k:, k])
            assert col[0] > np.max(col[1:], initial=0.0) * (1 + 1e-6)
            assert col[0] - np.sum(col[1:]) > 0  # the dominance itself survives
            M[k + 1:, k] /= M[k, k]
            M[k + 1:, k + 1:] -= np.outer(M[k + 1:, k], M[k, k + 1:])
        piv, _ = lu_pivots_unblocked(A)
        assert piv == list(range(N))


@pytest.mark.parametrize("L,nb", [(6, 4), (8, 16), (8, 12)])
def test_symmetric_tableau_sign_rule(L, nb):
    """A_{n,sigma} is complex symmetric and the dominant blocks are never pivoted, so after the
    index set S has been swept the tableau obeys M_ij = e_ij M_ji with e_ij = -1 when exactly
    one of i, j is in S and +1 otherwise.  The update computes the lower tiles only and the
    prep kernels read the strips' other half through this rule."""
    A, _ = block_matrix(L, 7, +1)
    assert np.allclose(A, A.T, rtol=0, atol=0)
    N = A.shape[0]
    M = A.copy()
    swept = np.zeros(N, bool)
    for k0 in range(0, N, nb):
        kb = min(nb, N - k0)
        M = gj_step(M, k0, kb)
        swept[k0:k0 + kb] = True
        e = np.where(swept[:, None] ^ swept[None, :], -1.0, 1.0)
        assert np.max(np.abs(M - e * M.T)) <= 1e-14 * np.max(np.abs(M))
    assert np.max(np.abs(M - np.linalg.inv(A))) <= 1e-13 * np.max(np.abs(M))


@pytest.mark.parametrize("L,kb1,kb2,start", [(8, 16, 16, 16), (8, 16, 12, 36), (6, 8, 8, 0)])
def test_merged_pair_equals_two_sequential_steps(L, kb1, kb2, start):
    """Two adjacent Gauss-Jordan steps K1, K2 as the dominant group runs them: the cross
    launch updates only K2's rows and columns with F1 W1 (under K1's mask), K2's factors come
    from that cross, and the merged launch updates every other entry with [F1 F2][W1; W2]
    (one K = kb1 + kb2 product, under K1's mask) and the cross with F2 W2 (under K2's mask).
    Equal to the two steps in sequence; from the start and from a partly swept tableau."""
    A, _ = block_matrix(L, 9, -1)
    N = A.shape[0]
    M = A.copy()
    for k0 in range(0, start, kb1):  # sweep the blocks before the pair
        M = gj_step(M, k0, min(kb1, start - k0))
    k1, k2 = start, start + kb1
    assert k2 + kb2 <= N
    seq = gj_step(gj_step(M, k1, kb1), k2, kb2)

    F1, W1 = gj_factors(M, k1, kb1)
    cross = np.zeros((N, N), bool)
    cross[k2:k2 + kb2, :] = True
    cross[:, k2:k2 + kb2] = True
    Mc = np.where(cross, masked(M, k1, kb1) - F1 @ W1, np.nan)  # only the cross is formed
    F2, W2 = gj_factors(Mc, k2, kb2)  # reads the cross alone (no NaN may leak in)
    assert np.all(np.isfinite(F2)) and np.all(np.isfinite(W2))
    merged = masked(M, k1, kb1) - np.hstack([F1, F2]) @ np.vstack([W1, W2])
    on_cross = masked(np.nan_to_num(Mc), k2, kb2) - F2 @ W2
    out = np.where(cross, on_cross, merged)
    assert np.max(np.abs(out - seq)) <= 1e-13 * np.max(np.abs(seq))


@pytest.mark.parametrize("eps", [1e-3, 1e-5])
def test_newton_refinement_error_is_minus_delta_a_delta(eps):
    """The refinement G_ii <- 2 X_ii - (X A X)_ii of an approximate inverse X = G + D leaves
    exactly G_ii - (D A D)_ii (G A = A G = I): the error becomes quadratic in the error of the
    float32 inverse, which is what lets float32 blocks give FP64-level gradients."""
    A, _ = block_matrix(6, 3, +1)
    G = np.linalg.inv(A)
    rng = np.random.default_rng(5)
    D = eps * np.max(np.abs(G)) * (rng.standard_normal(G.shape) + 1j * rng.standard_normal(G.shape))
    D = 0.5 * (D + D.T)  # the inverse of a symmetric block is symmetric
    X = G + D
    refined = 2 * np.diag(X) - np.einsum("ij,jk,ki->i", X, A, X)
    predicted = np.diag(G) - np.einsum("ij,jk,ki->i", D, A, D)
    assert np.max(np.abs(refined - predicted)) <= 1e-13 * np.max(np.abs(G))
    assert np.max(np.abs(refined - np.diag(G))) <= 40 * eps ** 2 * np.max(np.abs(G))
    assert np.max(np.abs(np.diag(X) - np.diag(G))) >= 0.1 * eps * np.max(np.abs(G))


def bonds(L):
    """Each site's bonds to its +x and +y neighbours (site j = x L + y, periodic)."""
    N = L * L
    j = np.arange(N)
    x, y = j // L, j % L
    return (np.concatenate([j, j]),
            np.concatenate([((x + 1) % L) * L + y, x * L + (y + 1) % L]))


def boundary_bonds(i, L):
    """The bonds with one end <= i and the other > i, enumerated as the row kernel of the
    lower-triangle refinement does (3L candidates): (j, j+L) for i-L < j <= i off the last
    x row, (i, i+1) off the last y column, the +y wraps (j+1-L, j) for i < j < i+L with
    y_j = L-1, and the +x wraps (j+L-N, j) for j >= N-L; (row end, column end) pairs."""
    N = L * L
    out = []
    for t in range(3 * L):
        if t < L:
            j = i - t
            if j >= 0 and j // L != L - 1 and j + L > i:
                out.append((j, j + L))
        elif t == L:
            if i % L != L - 1 and i + 1 < N:
                out.append((i, i + 1))
        elif t < 2 * L:
            j = i + t - L
            if j < N and j % L == L - 1 and j + 1 - L <= i:
                out.append((j + 1 - L, j))
        else:
            j = N - 3 * L + t
            if j > i and j + L - N <= i:
                out.append((j + L - N, j))
    return out


@pytest.mark.parametrize("L", [2, 4, 6, 8, 12, 16])
def test_boundary_bond_enumeration_is_exact(L):
    """For every row i the enumeration yields each bond that crosses i exactly once (as a
    multiset, so L = 2's doubled bonds count twice), with its row end <= i < its column end,
    and at most 2L + 2 of them."""
    bj, bk = bonds(L)
    lo, hi = np.minimum(bj, bk), np.maximum(bj, bk)
    for i in range(L * L):
        want = sorted(zip(lo[(lo <= i) & (hi > i)].tolist(), hi[(lo <= i) & (hi > i)].tolist()))
        got = boundary_bonds(i, L)
        assert sorted(got) == want, i
        assert all(r <= i < c for r, c in got)
        assert len(got) <= 2 * L + 2


@pytest.mark.parametrize("L", [2, 4, 8, 12])
def test_lower_triangle_split_of_the_refinement_form(L):
    """q_i = Re(x^T A x), x = row i of the symmetric inverse, as the sum of a_j Re x_j^2 -
    2 w Re x_j Im x_j over sites and 2t Re(x_j x_k) over bonds, split into the row part
    (sites j <= i, bonds with both ends <= i, read from row i), the column part (sites j > i,
    bonds with both ends > i, read down column i) and the boundary bonds (row end from row i,
    column end from column i).  The upper triangle of the stored inverse is NaN, so a read of
    it would show; the split equals the full quadratic form."""
    A, w = block_matrix(L, 8, -1)
    N = L * L
    t = 1.0  # A's off-diagonal entries are +t per bond
    a = A.diagonal().real
    assert np.allclose(A.diagonal().imag, w)
    X = np.linalg.inv(A)
    S = np.where(np.tril(np.ones((N, N), bool)), X, np.nan)  # only the lower triangle stored
    bj, bk = bonds(L)
    for i in range(N):
        row = S[i, :i + 1]  # x_j, j <= i
        col = S[i + 1:, i]  # x_j, j > i
        site = lambda x, aj: aj * (x.real ** 2 - x.imag ** 2) - 2 * w * x.real * x.imag
        lo, hi = np.minimum(bj, bk), np.maximum(bj, bk)
        inr, inc = hi <= i, lo > i
        q_row = np.sum(site(row, a[:i + 1])) + 2 * t * np.sum((row[lo[inr]] * row[hi[inr]]).real)
        q_col = (np.sum(site(col, a[i + 1:]))
                 + 2 * t * np.sum((col[lo[inc] - i - 1] * col[hi[inc] - i - 1]).real))
        q_bnd = 2 * t * sum((S[i, r] * S[c, i]).real for r, c in boundary_bonds(i, L))
        q = q_row + q_col + q_bnd
        assert np.isfinite(q), i
        x = X[i]
        q_ref = (x @ A @ x).real
        assert q == pytest.approx(q_ref, rel=1e-13, abs=1e-13)


def test_float32_vote_bound():
    """The float32 shortcut of the refinement: every site term obeys |e_j| <= C m^2 with
    C = 2 max|a_j| + 2w + 4|2t| and m the largest |Re|, |Im| among the site's entry and its
    two bond partners, so a group with m^2 <= small / C stays under the per-term bound."""
    rng = np.random.default_rng(17)
    for _ in range(2000):
        v = rng.standard_normal(6) * 10.0 ** rng.uniform(-8, 2)
        aj, w, t = rng.uniform(-6, 6), rng.uniform(0.3, 60), rng.choice([1.0, -1.0, 0.5])
        amax = abs(aj) * rng.uniform(1, 3)
        ar, ai, xr, xi, yr, yi = v
        e = aj * (ar * ar - ai * ai) - 2 * w * ar * ai + 2 * t * (ar * xr - ai * xi + ar * yr - ai * yi)
        m = np.max(np.abs(v))
        C = 2 * amax + 2 * w + 4 * abs(2 * t)
        assert abs(e) <= C * m * m * (1 + 1e-12)


def bf16_rn(x):
    """Round float32 values to the nearest bfloat16 (ties to even), returned as float32."""
    b = np.asarray(x, np.float32).view(np.uint32).astype(np.uint64)
    r = (b + 0x7FFF + ((b >> 16) & 1)) & 0xFFFF0000
    return r.astype(np.uint32).view(np.float32)


def test_bf16x3_split_product_error():
    """BF16x3: v = hi + lo with hi = RN_bf16(v), lo = RN_bf16(v - hi) keeps about 17
    significant bits (|v - hi - lo| <= 2^-17 |v|), and hi*hi' + hi*lo' + lo*hi' (the dropped
    lo*lo' term and the representation errors), accumulated in float32 over K = 256 terms,
    stays within a few 2^-16 of sum |a||b| against the FP64 dot product."""
    rng = np.random.default_rng(23)
    v = rng.standard_normal(100000).astype(np.float32) * np.float32(10.0) ** rng.integers(-3, 3, 100000).astype(np.float32)
    hi = bf16_rn(v)
    lo = bf16_rn(v - hi)
    rel = np.abs(v.astype(np.float64) - hi - lo) / np.abs(v)
    assert rel.max() <= 2.0 ** -17
    for _ in range(50):
        a = rng.standard_normal(256).astype(np.float32)
        b = rng.standard_normal(256).astype(np.float32)
        ah, bh = bf16_rn(a), bf16_rn(b)
        al, bl = bf16_rn(a - ah), bf16_rn(b - bh)
        acc = np.float32(0)
        for k in range(256):  # float32 accumulation of the three bf16 products
            acc = np.float32(acc + np.float32(ah[k] * bh[k]))
            acc = np.float32(acc + np.float32(ah[k] * bl[k]))
            acc = np.float32(acc + np.float32(al[k] * bh[k]))
        exact = float(np.dot(a.astype(np.float64), b.astype(np.float64)))
        scale = float(np.sum(np.abs(a.astype(np.float64) * b)))
        assert abs(float(acc) - exact) <= 4 * 2.0 ** -16 * scale
