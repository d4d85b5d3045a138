"""Pins for the CPU oracle: each check compares it with something other than
itself — the paper's printed matrices, the triple-product property, closed-form
operation counts, per-bit brute force, a library integer matmul, and algebraic
identities of the products. A plausible slip (a dropped term, a wrong index,
a transposed operand) fails at least one of them."""
import itertools

import numpy as np
import pytest

import oracle as O
from bitgen import fill_cpu

VARIANTS = {"sw": O.SW, "self_inverse": O.SELF_INVERSE, "chaining": O.CHAINING}
rng = np.random.default_rng(1909)


def rand_bits(rows, cols, p=0.5):
    return (rng.random((rows, cols)) < p).astype(np.uint8)


def gf2(M):
    return (np.asarray(M, dtype=np.int64) % 2).astype(np.uint8)


# ------------------------------------------------------------ golden matrices
def _triple_ok(zeta, xi, eta):
    """Eq. triple-prod with <2,2,2>_7: sum_h zeta[i'k',h] xi[h,ij] eta[h,j'k] == [i=i',j=j',k=k']."""
    for i, j, jp, k, ip, kp in itertools.product(range(2), repeat=6):
        s = sum(int(zeta[2 * ip + kp, h]) * int(xi[h, 2 * i + j]) * int(eta[h, 2 * jp + k])
                for h in range(7)) % 2
        if s != int(i == ip and j == jp and k == kp):
            return False
    return True


def test_golden_triple_product_sw(decomp):
    assert _triple_ok(decomp["sw", "zeta"], decomp["sw", "xi"], decomp["sw", "eta"])


@pytest.mark.parametrize("variant", ["self_inverse", "chaining"])
def test_golden_triple_product_alt_basis(decomp, variant):
    """(chi gamma | alpha phi, beta psi) has the triple product property (Sec. 2.8)."""
    phi, chi = decomp[variant, "phi"], decomp[variant, "chi"]
    al, be, ga = decomp[variant, "alpha"], decomp[variant, "beta"], decomp[variant, "gamma"]
    assert _triple_ok(gf2(chi @ ga), gf2(al @ phi), gf2(be @ phi))


def test_golden_triple_product_detects_a_slip(decomp):
    ga = decomp["self_inverse", "gamma"].copy()
    ga[3, 6] ^= 1
    phi, chi = decomp["self_inverse", "phi"], decomp["self_inverse", "chi"]
    al, be = decomp["self_inverse", "alpha"], decomp["self_inverse", "beta"]
    assert not _triple_ok(gf2(chi @ ga), gf2(al @ phi), gf2(be @ phi))


def test_golden_basis_properties(decomp):
    I = np.eye(4, dtype=np.uint8)
    phi, chi = decomp["self_inverse", "phi"], decomp["self_inverse", "chi"]
    assert (gf2(phi @ phi) == I).all() and (gf2(chi @ chi) == I).all()  # self-inverse
    assert (phi == chi.T).all()  # phi = psi = chi^T
    phi2, chi2 = decomp["chaining", "phi"], decomp["chaining", "chi"]
    assert (gf2(chi2 @ phi2) == I).all()  # chi = phi^{-1}: chaining (Thm. 2)
    assert not (gf2(phi2 @ phi2) == I).all()


def test_golden_weight_distributions(decomp):
    """Thm. 1: weights 1,1,1,1,2,2,2; Thm. 2: 1,1,1,1,2,2,2 (operands) and 1,1,1,1,2,3,3 (products)."""
    for v in ("self_inverse", "chaining"):
        for name in ("alpha", "beta"):
            assert sorted(decomp[v, name].sum(axis=1)) == [1, 1, 1, 1, 2, 2, 2]
    assert sorted(decomp["self_inverse", "gamma"].sum(axis=0)) == [1, 1, 1, 1, 2, 2, 2]
    assert sorted(decomp["chaining", "gamma"].sum(axis=0)) == [1, 1, 1, 1, 2, 3, 3]


# ------------------------------------------------------------ oracle programs vs golden
@pytest.mark.parametrize("variant", ["self_inverse", "chaining"])
def test_oracle_straight_line_programs_match_paper(decomp, variant):
    v = VARIANTS[variant]
    assert (O.level_matrix(v, O.PHI) == decomp[variant, "phi"]).all()
    assert (O.level_matrix(v, O.PSI) == decomp[variant, "phi"]).all()
    assert (O.level_matrix(v, O.CHI) == decomp[variant, "chi"]).all()
    assert (O.level_matrix(v, O.ALPHA) == decomp[variant, "alpha"]).all()
    assert (O.level_matrix(v, O.BETA) == decomp[variant, "beta"]).all()
    assert (O.level_matrix(v, O.GAMMA) == decomp[variant, "gamma"]).all()


def test_oracle_sw_programs_match_paper(decomp):
    assert (O.level_matrix(O.SW, O.ALPHA) == decomp["sw", "xi"]).all()
    assert (O.level_matrix(O.SW, O.BETA) == decomp["sw", "eta"]).all()
    assert (O.level_matrix(O.SW, O.GAMMA) == decomp["sw", "zeta"]).all()
    assert (O.level_matrix(O.SW, O.PHI) == np.eye(4, dtype=np.uint8)).all()


# ------------------------------------------------------------ cubic product
@pytest.mark.parametrize("op", [O.GF2, O.BOOL])
@pytest.mark.parametrize("m,k,n,p", [(64, 64, 64, 0.5), (128, 64, 192, 0.5), (64, 192, 128, 0.1),
                                     (192, 128, 64, 0.03)])
def test_cubic_matches_per_bit_brute_force(op, m, k, n, p):
    if m * k * n > 64 * 192 * 128 and op == O.BOOL:
        pytest.skip("keep the pure-Python loop small")
    Ab, Bb = rand_bits(m, k, p), rand_bits(k, n, p)
    C = O.cubic(op, O.pack(Ab), O.pack(Bb), m, k, n)
    ref = O.brute_force(op, Ab[:64, :], Bb) if m * k * n > 2e6 else O.brute_force(op, Ab, Bb)
    assert (O.unpack(C, m, n)[: ref.shape[0]] == ref).all()


@pytest.mark.parametrize("m,k,n", [(256, 512, 320), (1024, 1024, 1024), (64, 2048, 128)])
def test_cubic_matches_integer_matmul(m, k, n):
    """Library special case: GF(2) = (Z-product mod 2), Boolean = (Z-product > 0)."""
    Ab, Bb = rand_bits(m, k), rand_bits(k, n, 2.0 / k ** 0.5)
    Z = Ab.astype(np.int64) @ Bb.astype(np.int64)
    A, B = O.pack(Ab), O.pack(Bb)
    assert (O.unpack(O.cubic(O.GF2, A, B, m, k, n), m, n) == (Z % 2)).all()
    assert (O.unpack(O.cubic(O.BOOL, A, B, m, k, n), m, n) == (Z > 0)).all()


def test_cubic_identity_and_zero():
    n = 256
    I = O.pack(np.eye(n, dtype=np.uint8))
    A = O.pack(rand_bits(n, n))
    Z = np.zeros_like(A)
    for op in (O.GF2, O.BOOL):
        assert (O.cubic(op, A, I, n, n, n) == A).all()
        assert (O.cubic(op, I, A, n, n, n) == A).all()
        assert (O.cubic(op, A, Z, n, n, n) == 0).all()
        assert (O.cubic(op, Z, A, n, n, n) == 0).all()


def test_cubic_counts_closed_form():
    """Row i of A has its first c_i bits set and B is all ones, so every entry of
    row i of the integer product is c_i: GF(2) gives c_i mod 2, Boolean gives c_i > 0."""
    m, k, n = 256, 192, 128
    c = np.array([(7 * i) % (k + 1) for i in range(m)])
    Ab = (np.arange(k)[None, :] < c[:, None]).astype(np.uint8)
    Bb = np.ones((k, n), dtype=np.uint8)
    g = O.unpack(O.cubic(O.GF2, O.pack(Ab), O.pack(Bb), m, k, n), m, n)
    b = O.unpack(O.cubic(O.BOOL, O.pack(Ab), O.pack(Bb), m, k, n), m, n)
    assert (g == (c % 2)[:, None]).all()
    assert (b == (c > 0)[:, None]).all()


@pytest.mark.parametrize("op", [O.GF2, O.BOOL])
def test_cubic_transpose_identity(op):
    """(AB)^T = B^T A^T, with an independent bit transpose."""
    m, k, n = 192, 320, 128
    A, B = O.pack(rand_bits(m, k, 0.3)), O.pack(rand_bits(k, n, 0.3))
    C = O.cubic(op, A, B, m, k, n)
    Ct = O.cubic(op, O.transpose(B, k, n), O.transpose(A, m, k), n, k, m)
    assert (O.transpose(C, m, n) == Ct).all()
    assert (O.unpack(O.transpose(A, m, k), k, m) == O.unpack(A, m, k).T).all()


@pytest.mark.parametrize("op", [O.GF2, O.BOOL])
def test_cubic_associativity(op):
    m, k, n, r = 128, 192, 64, 256
    p = 0.5 if op == O.GF2 else 0.05
    A, B, C = (O.pack(rand_bits(m, k, p)), O.pack(rand_bits(k, n, p)),
               O.pack(rand_bits(n, r, p)))
    left = O.cubic(op, O.cubic(op, A, B, m, k, n), C, m, n, r)
    right = O.cubic(op, A, O.cubic(op, B, C, k, n, r), m, k, r)
    assert (left == right).all()


def test_gf2_linearity_and_boolean_monotonicity():
    m, k, n = 128, 256, 192
    A1, A2, B = O.pack(rand_bits(m, k)), O.pack(rand_bits(m, k)), O.pack(rand_bits(k, n))
    lhs = O.cubic(O.GF2, A1 ^ A2, B, m, k, n)
    assert (lhs == (O.cubic(O.GF2, A1, B, m, k, n) ^ O.cubic(O.GF2, A2, B, m, k, n))).all()
    As = O.pack(rand_bits(m, k, 0.02))
    Abig = As | O.pack(rand_bits(m, k, 0.01))
    Bs = O.pack(rand_bits(k, n, 0.02))
    small, big = O.cubic(O.BOOL, As, Bs, m, k, n), O.cubic(O.BOOL, Abig, Bs, m, k, n)
    assert ((small & ~big) == 0).all()
    assert (O.cubic(O.BOOL, A1 | A2, B, m, k, n) ==
            (O.cubic(O.BOOL, A1, B, m, k, n) | O.cubic(O.BOOL, A2, B, m, k, n))).all()


def test_rows_columns_and_freivalds_helpers():
    m, k, n = 256, 320, 192
    A, B = O.pack(rand_bits(m, k)), O.pack(rand_bits(k, n))
    for op in (O.GF2, O.BOOL):
        C = O.cubic(op, A, B, m, k, n)
        sel = [0, 17, 255]
        assert (O.rows(op, A[sel], B, k, n) == C[sel]).all()
        for j in (0, 63, 64, 191):
            assert (O.column(op, A, B, j, m, k, n) == O.unpack(C, m, n)[:, j]).all()
    C = O.cubic(O.GF2, A, B, m, k, n)
    x = O.pack(rand_bits(1, n))[0]
    lhs = O.matvec_gf2(C, x, m, n)
    rhs = O.matvec_gf2(A, O.matvec_gf2(B, x, k, n), m, k)
    assert (lhs == rhs).all()
    bad = C.copy()
    bad[3, 1] ^= np.uint64(1 << 5)
    # one flipped bit is caught by at least one of a few random vectors
    caught = False
    for _ in range(8):
        x = O.pack(rand_bits(1, n))[0]
        caught |= not (O.matvec_gf2(bad, x, m, n) ==
                       O.matvec_gf2(A, O.matvec_gf2(B, x, k, n), m, k)).all()
    assert caught


# ------------------------------------------------------------ Strassen model
@pytest.mark.parametrize("variant", ["sw", "self_inverse", "chaining"])
@pytest.mark.parametrize("depth,m,k,n", [(1, 128, 128, 128), (2, 256, 512, 256),
                                         (3, 512, 512, 512), (2, 768, 256, 1024)])
def test_strassen_equals_cubic(variant, depth, m, k, n):
    A, B = O.pack(rand_bits(m, k)), O.pack(rand_bits(k, n))
    C, _ = O.strassen_gf2(VARIANTS[variant], A, B, m, k, n, depth)
    assert (C == O.cubic(O.GF2, A, B, m, k, n)).all()


@pytest.mark.parametrize("variant", ["sw", "self_inverse", "chaining"])
@pytest.mark.parametrize("depth", [1, 2, 3])
def test_strassen_counts_match_closed_forms(variant, depth):
    """Sec. 2.7, Eqs. diag-basis-change-cost and diag-linear-comb-cost with blocks of
    b x b bits at the leaves: basis changes (P^chi+P^phi+P^psi) s^(2(d-1)) d b^2,
    linear combinations (P^gamma+P^alpha+P^beta) (r^d - s^(2d))/(r - s^2) b^2 and
    r^d leaf products of 2 b^3 - b^2 bit operations each (r = 7, s = 2).
    At b = 1 these give 5 n^lg7 - 4 n^2 (alternative basis) and 6 n^lg7 - 5 n^2
    (Strassen-Winograd) plus n^2 lg n / 2 per basis change (Sec. 1)."""
    b = 64
    n = b << depth
    A, B = O.pack(rand_bits(n, n)), O.pack(rand_bits(n, n))
    _, cnt = O.strassen_gf2(VARIANTS[variant], A, B, n, n, n, depth)
    P_lin = 15 if variant == "sw" else 12
    P_basis = 0 if variant == "sw" else 6
    assert cnt["basis_bitops"] == P_basis * 4 ** (depth - 1) * depth * b * b
    assert cnt["lincomb_bitops"] == P_lin * (7 ** depth - 4 ** depth) // 3 * b * b
    assert cnt["leaf_products"] == 7 ** depth
    assert cnt["mult_bitops"] == 7 ** depth * (2 * b ** 3 - b ** 2)
    # the b = 1 specialisation of the same formulas is the paper's headline count
    nn = 2 ** depth
    total_b1 = P_lin * (7 ** depth - 4 ** depth) // 3 + 7 ** depth
    want = (6 * 7 ** depth - 5 * nn * nn) if variant == "sw" else (5 * 7 ** depth - 4 * nn * nn)
    assert total_b1 == want


@pytest.mark.parametrize("variant", ["self_inverse", "chaining"])
def test_basis_change_round_trips(variant):
    v = VARIANTS[variant]
    n, d = 512, 3
    X = O.pack(rand_bits(n, n))
    Y, ops = O.basis_change(v, False, X, n, n, d)
    assert ops == d * n * n // 2  # Sec. 1: (1/2) n^2 per level
    assert not (Y == X).all()
    if variant == "self_inverse":
        Z, _ = O.basis_change(v, False, Y, n, n, d)  # phi is its own inverse (Eq. mb-basis)
        assert (Z == X).all()
    Z, _ = O.basis_change(v, True, Y, n, n, d)
    if variant == "chaining":
        assert (Z == X).all()  # chi = phi^{-1} (Eq. ab-basis)


@pytest.mark.parametrize("depth", [1, 2])
def test_alternative_basis_product_in_the_basis(depth):
    """Before the output basis change, the recursion yields chi^{-1} applied to AB.
    Chaining (Thm. 2, chi = phi^{-1}): the product of phi(A) and phi(B) is phi(AB),
    so products chain in the alternative basis. Self-inverse (Thm. 1, chi = chi^{-1}):
    it is chi(AB)."""
    n = 128 << depth
    A, B = O.pack(rand_bits(n, n)), O.pack(rand_bits(n, n))
    C = O.cubic(O.GF2, A, B, n, n, n)
    for v in (O.CHAINING, O.SELF_INVERSE):
        Ah, _ = O.basis_change(v, False, A, n, n, depth)
        Bh, _ = O.basis_change(v, False, B, n, n, depth)
        Ch = O.alt_product(v, Ah, Bh, n, n, n, depth)
        if v == O.CHAINING:
            want, _ = O.basis_change(v, False, C, n, n, depth)
        else:
            want, _ = O.basis_change(v, True, C, n, n, depth)
        assert (Ch == want).all()
    # chaining: a second product straight from the alternative basis
    D = O.pack(rand_bits(n, n))
    Dh, _ = O.basis_change(O.CHAINING, False, D, n, n, depth)
    Ch = O.alt_product(O.CHAINING, *[O.basis_change(O.CHAINING, False, X, n, n, depth)[0]
                                     for X in (A, B)], n, n, n, depth)
    CDh = O.alt_product(O.CHAINING, Ch, Dh, n, n, n, depth)
    back, _ = O.basis_change(O.CHAINING, True, CDh, n, n, depth)
    assert (back == O.cubic(O.GF2, C, D, n, n, n)).all()


def test_strassen_rejects_bad_sizes():
    A = np.zeros((64, 2), dtype=np.uint64)
    with pytest.raises(ValueError):
        O.strassen_gf2(O.SELF_INVERSE, A, np.zeros((128, 1), dtype=np.uint64), 64, 128, 64, 1)


def test_oracle_on_generated_inputs_is_deterministic():
    A1 = fill_cpu(128, 256, 1, 0)
    A2 = fill_cpu(128, 256, 1, 0)
    assert (A1 == A2).all()
