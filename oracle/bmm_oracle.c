/*
 * CPU oracle for bit-matrix products — TEST INFRASTRUCTURE ONLY.
 *
 * Only the tests, the smoke check and the bench's CPU-baseline leg load this
 * library. The GPU product path never calls it, and it shares no code with
 * the GPU path (the two meet only in the seeded input generator, bitgen/).
 *
 * What it computes (Karppa & Kaski, arXiv:1909.01554):
 *   - Boolean product  C_ij = OR_k  (A_ik AND B_kj)  over (0,1,v,^)   (Sec. 1, Sec. 3.18)
 *   - binary product   C_ij = XOR_k (A_ik AND B_kj)  over GF(2)        (Sec. 2.4 product
 *     definition; Eq. c-equals-ab with "+" read as XOR)
 *   - the same binary product through 2x2 block recursions on packed quadrants:
 *       variant 0: Strassen–Winograd, standard basis   (Eqs. sw-input, sw-mul, sw-output)
 *       variant 1: alternative basis, self-inverse     (Sec. 2.2, Eqs. mb-*)
 *       variant 2: alternative basis, chaining         (Sec. 2.3, Eqs. ab-*)
 *     instrumented to count bit operations (Sec. 2.7 cost formulas).
 *
 * Layout (Sec. 3.4 linearisation: the least significant index lives in the
 * bits of a word): row-major, cols a multiple of 64, bit j of row i is bit
 * (j % 64) of word i*(cols/64) + j/64.
 *
 * Plain loops only: the cubic product is written as the definition row by
 * row (row i of C is the XOR/OR of the rows of B selected by row i of A),
 * threaded over rows of C.
 */
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OP_GF2 0
#define OP_BOOL 1

static int bit_of(const uint64_t *row, int64_t j) { return (int)((row[j >> 6] >> (j & 63)) & 1u); }

/* ------------------------------------------------------------------ cubic */
typedef struct {
    int op;
    const uint64_t *A, *B;
    uint64_t *C;
    int64_t k, n, lo, hi;
} cubic_job;

static void *cubic_worker(void *p) {
    cubic_job *j = (cubic_job *)p;
    int64_t kw = j->k / 64, nw = j->n / 64;
    for (int64_t i = j->lo; i < j->hi; i++) {
        const uint64_t *a = j->A + i * kw;
        uint64_t *c = j->C + i * nw;
        for (int64_t w = 0; w < nw; w++) c[w] = 0;
        for (int64_t kk = 0; kk < j->k; kk++) {
            if (!bit_of(a, kk)) continue; /* A_ik AND B_kj is 0 for every j */
            const uint64_t *b = j->B + kk * nw;
            if (j->op == OP_GF2)
                for (int64_t w = 0; w < nw; w++) c[w] ^= b[w];
            else
                for (int64_t w = 0; w < nw; w++) c[w] |= b[w];
        }
    }
    return NULL;
}

static void run_rows(void *(*fn)(void *), void *jobs, size_t job_size, int nthreads) {
    pthread_t *th = (pthread_t *)malloc(sizeof(pthread_t) * (size_t)nthreads);
    for (int t = 0; t < nthreads; t++) pthread_create(&th[t], NULL, fn, (char *)jobs + job_size * t);
    for (int t = 0; t < nthreads; t++) pthread_join(th[t], NULL);
    free(th);
}

/* C (m x n) = A (m x k) * B (k x n) over GF(2) (op 0) or the Boolean algebra (op 1). */
void oracle_cubic(int op, const uint64_t *A, const uint64_t *B, uint64_t *C, int64_t m,
                  int64_t k, int64_t n, int nthreads) {
    if (nthreads < 1) nthreads = 1;
    if (nthreads > m) nthreads = (int)(m > 0 ? m : 1);
    cubic_job *jobs = (cubic_job *)malloc(sizeof(cubic_job) * (size_t)nthreads);
    for (int t = 0; t < nthreads; t++) {
        cubic_job j = {op, A, B, C, k, n, m * t / nthreads, m * (t + 1) / nthreads};
        jobs[t] = j;
    }
    run_rows(cubic_worker, jobs, sizeof(cubic_job), nthreads);
    free(jobs);
}

/* Selected rows of C: Arows holds the nrows requested rows of A (nrows x k),
 * Crows receives the same rows of C (nrows x n). */
void oracle_rows(int op, const uint64_t *Arows, const uint64_t *B, uint64_t *Crows, int64_t nrows,
                 int64_t k, int64_t n, int nthreads) {
    oracle_cubic(op, Arows, B, Crows, nrows, k, n, nthreads);
}

/* Column j of B as a packed k-vector: out[kk] = B[kk][j]. */
void oracle_extract_column(const uint64_t *B, int64_t k, int64_t n, int64_t j, uint64_t *out) {
    int64_t nw = n / 64;
    for (int64_t w = 0; w < k / 64; w++) out[w] = 0;
    for (int64_t kk = 0; kk < k; kk++)
        if (bit_of(B + kk * nw, j)) out[kk >> 6] |= 1ULL << (kk & 63);
}

/* Column of C from one packed column of B: out[i] = OR/XOR_kk A[i][kk] AND bcol[kk]. */
void oracle_column(int op, const uint64_t *A, const uint64_t *bcol, uint8_t *out, int64_t m,
                   int64_t k) {
    int64_t kw = k / 64;
    for (int64_t i = 0; i < m; i++) {
        int acc = 0;
        for (int64_t w = 0; w < kw; w++) {
            uint64_t x = A[i * kw + w] & bcol[w];
            if (op == OP_GF2)
                acc ^= __builtin_parityll(x);
            else
                acc |= (x != 0);
        }
        out[i] = (uint8_t)acc;
    }
}

/* y = M x over GF(2) for a packed rows x cols matrix M and packed x (cols bits);
 * y is packed (rows bits). Used by Freivalds checks C x == A (B x). */
void oracle_matvec_gf2(const uint64_t *M, const uint64_t *x, uint64_t *y, int64_t rows,
                       int64_t cols) {
    int64_t cw = cols / 64;
    for (int64_t w = 0; w < (rows + 63) / 64; w++) y[w] = 0;
    for (int64_t i = 0; i < rows; i++) {
        uint64_t acc = 0;
        for (int64_t w = 0; w < cw; w++) acc ^= M[i * cw + w] & x[w];
        if (__builtin_parityll(acc)) y[i >> 6] |= 1ULL << (i & 63);
    }
}

/* ------------------------------------------------------------------ block views */
typedef struct {
    uint64_t *p;
    int64_t rows, wcols, stride; /* wcols, stride in 64-bit words */
} view;

typedef struct {
    uint64_t basis_bitops;   /* phi, psi, chi (Eq. mb-basis-change-cost) */
    uint64_t lincomb_bitops; /* alpha, beta, gamma or xi, eta, zeta (Eq. mb-linear-comb-cost) */
    uint64_t mult_bitops;    /* leaf cubic products: 2 m k n - m n each */
    uint64_t leaf_products;
} oracle_counts;

static view quad(view x, int r, int c) {
    view q = {x.p + (int64_t)r * (x.rows / 2) * x.stride + (int64_t)c * (x.wcols / 2), x.rows / 2,
              x.wcols / 2, x.stride};
    return q;
}

static view alloc_view(int64_t rows, int64_t wcols) {
    view v = {(uint64_t *)calloc((size_t)(rows * wcols), 8), rows, wcols, wcols};
    return v;
}

/* d = a + b over GF(2) (d may alias a or b); counts rows * cols bit additions. */
static void vxor(view d, view a, view b, uint64_t *cnt) {
    for (int64_t i = 0; i < d.rows; i++)
        for (int64_t w = 0; w < d.wcols; w++)
            d.p[i * d.stride + w] = a.p[i * a.stride + w] ^ b.p[i * b.stride + w];
    if (cnt) *cnt += (uint64_t)(d.rows * d.wcols * 64);
}

static void vcopy(view d, view a) {
    for (int64_t i = 0; i < d.rows; i++)
        for (int64_t w = 0; w < d.wcols; w++) d.p[i * d.stride + w] = a.p[i * a.stride + w];
}

/* --------------------------------------------------- one-level straight-line programs
 * X[0..3] are the blocks X00, X01, X10, X11 (quadrant (r,c) is X[2r+c],
 * Eq. ab). Products are indexed h = 0..6 as in the paper. */

/* Input linear combinations T_h from A-blocks. */
static void slp_alpha(int variant, view *a, view *t, uint64_t *cnt) {
    switch (variant) {
    case 0: /* Eq. sw-input, T side */
        vxor(t[0], a[2], a[3], cnt);  /* T0 = A10 + A11 */
        vcopy(t[1], a[1]);            /* T1 = A01       */
        vxor(t[2], a[1], a[3], cnt);  /* T2 = A01 + A11 */
        vxor(t[3], a[2], t[2], cnt);  /* T3 = A10 + T2  */
        vxor(t[4], a[0], t[3], cnt);  /* T4 = A00 + T3  */
        vcopy(t[5], a[2]);            /* T5 = A10       */
        vcopy(t[6], a[0]);            /* T6 = A00       */
        break;
    case 1: /* Eq. mb-tsrecurrence, T side */
        vcopy(t[0], a[0]);
        vcopy(t[1], a[1]);
        vcopy(t[2], a[2]);
        vcopy(t[3], a[3]);
        vxor(t[4], a[0], a[3], cnt); /* T4 = A00 + A11 */
        vxor(t[5], a[1], a[3], cnt); /* T5 = A01 + A11 */
        vxor(t[6], a[2], a[3], cnt); /* T6 = A10 + A11 */
        break;
    default: /* Eq. ab-tsrecurrence, T side */
        vcopy(t[0], a[0]);
        vcopy(t[1], a[1]);
        vcopy(t[2], a[2]);
        vcopy(t[3], a[3]);
        vxor(t[4], a[0], a[2], cnt); /* T4 = A00 + A10 */
        vxor(t[5], a[1], a[2], cnt); /* T5 = A01 + A10 */
        vxor(t[6], a[2], a[3], cnt); /* T6 = A10 + A11 */
        break;
    }
}

/* Input linear combinations S_h from B-blocks. */
static void slp_beta(int variant, view *b, view *s, uint64_t *cnt) {
    switch (variant) {
    case 0: /* Eq. sw-input, S side */
        vxor(s[0], b[2], b[3], cnt);  /* S0 = B10 + B11 */
        vcopy(s[1], b[2]);            /* S1 = B10       */
        vxor(s[2], b[1], b[3], cnt);  /* S2 = B01 + B11 */
        vxor(s[3], b[2], s[2], cnt);  /* S3 = B10 + S2  */
        vcopy(s[4], b[1]);            /* S4 = B01       */
        vxor(s[5], b[0], s[3], cnt);  /* S5 = B00 + S3  */
        vcopy(s[6], b[0]);            /* S6 = B00       */
        break;
    case 1: /* Eq. mb-tsrecurrence, S side */
        vcopy(s[0], b[0]);            /* S0 = B00       */
        vcopy(s[1], b[2]);            /* S1 = B10       */
        vxor(s[2], b[0], b[3], cnt);  /* S2 = B00 + B11 */
        vcopy(s[3], b[3]);            /* S3 = B11       */
        vcopy(s[4], b[1]);            /* S4 = B01       */
        vxor(s[5], b[1], b[3], cnt);  /* S5 = B01 + B11 */
        vxor(s[6], b[2], b[3], cnt);  /* S6 = B10 + B11 */
        break;
    default: /* Eq. ab-tsrecurrence, S side */
        vcopy(s[0], b[0]);            /* S0 = B00       */
        vxor(s[1], b[2], b[3], cnt);  /* S1 = B10 + B11 */
        vcopy(s[2], b[2]);            /* S2 = B10       */
        vcopy(s[3], b[3]);            /* S3 = B11       */
        vcopy(s[4], b[1]);            /* S4 = B01       */
        vxor(s[5], b[1], b[2], cnt);  /* S5 = B01 + B10 */
        vxor(s[6], b[0], b[2], cnt);  /* S6 = B00 + B10 */
        break;
    }
}

/* Output linear combinations: C-blocks from the seven products Q_h.
 * u[0..2] is scratch of the C-block shape (variant 0 uses U0..U2, variant 2 uses R). */
static void slp_gamma(int variant, view *q, view *c, view *u, uint64_t *cnt) {
    switch (variant) {
    case 0: /* Eq. sw-output */
        vxor(u[0], q[1], q[3], cnt);  /* U0 = Q1 + Q3 */
        vxor(u[1], q[2], u[0], cnt);  /* U1 = Q2 + U0 */
        vxor(u[2], q[4], u[0], cnt);  /* U2 = Q4 + U0 */
        vxor(c[0], q[1], q[6], cnt);  /* C00 = Q1 + Q6 */
        vxor(c[1], q[0], u[2], cnt);  /* C01 = Q0 + U2 */
        vxor(c[2], q[5], u[1], cnt);  /* C10 = Q5 + U1 */
        vxor(c[3], q[0], u[1], cnt);  /* C11 = Q0 + U1 */
        break;
    case 1: /* Eq. mb-qrecurrence */
        vxor(c[0], q[0], q[1], cnt);  /* C00 = Q0 + Q1 */
        vxor(c[1], q[4], q[6], cnt);  /* C01 = Q4 + Q6 */
        vxor(c[2], q[2], q[5], cnt);  /* C10 = Q2 + Q5 */
        vxor(c[3], q[1], q[3], cnt);  /* C11 = Q1 + Q3 + Q5 + Q6 */
        vxor(c[3], c[3], q[5], cnt);
        vxor(c[3], c[3], q[6], cnt);
        break;
    default: /* Eq. ab-qrecurrence */
        vxor(u[0], q[1], q[2], cnt);  /* R = Q1 + Q2 + Q4 */
        vxor(u[0], u[0], q[4], cnt);
        vxor(c[0], q[0], q[1], cnt);  /* C00 = Q0 + Q1 */
        vxor(c[1], u[0], q[5], cnt);  /* C01 = R + Q5 */
        vxor(c[2], u[0], q[6], cnt);  /* C10 = R + Q6 */
        vxor(c[3], q[3], q[4], cnt);  /* C11 = Q3 + Q4 */
        break;
    }
}

/* Forward basis change on the four blocks, in place (phi for A, psi for B;
 * the paper uses phi = psi for both alternative-basis variants). */
static void slp_phi(int variant, view *x, uint64_t *cnt) {
    switch (variant) {
    case 0: /* standard basis: identity */
        break;
    case 1: /* Eq. mb-fwdbasisrecurrence: X11 <- X01 + X10 + X11 */
        vxor(x[3], x[3], x[1], cnt);
        vxor(x[3], x[3], x[2], cnt);
        break;
    default: /* Eq. ab-fwdbasisrecurrence: X11 <- X01 + X11, then X10 <- X11^ + X10 */
        vxor(x[3], x[1], x[3], cnt);
        vxor(x[2], x[3], x[2], cnt);
        break;
    }
}

/* Inverse basis change chi on C-blocks, in place. */
static void slp_chi(int variant, view *x, uint64_t *cnt) {
    switch (variant) {
    case 0:
        break;
    case 1: /* Eq. mb-revbasisrecurrence: C01 <- C01 + C11, C10 <- C10 + C11 */
        vxor(x[1], x[1], x[3], cnt);
        vxor(x[2], x[2], x[3], cnt);
        break;
    default: /* Eq. ab-revbasisrecurrence: X10 <- X10 + X11, then X11 <- X01 + X11 */
        vxor(x[2], x[2], x[3], cnt);
        vxor(x[3], x[1], x[3], cnt);
        break;
    }
}

#define WHICH_PHI 0
#define WHICH_PSI 1
#define WHICH_CHI 2
#define WHICH_ALPHA 3
#define WHICH_BETA 4
#define WHICH_GAMMA 5

/* Apply one level's straight-line program to single 64-bit words (64
 * independent instances side by side). in/out: 4 or 7 words. Lets tests read
 * off the matrix each program implements, by feeding unit vectors. */
void oracle_level_probe(int variant, int which, const uint64_t *in, uint64_t *out) {
    uint64_t buf_in[7], buf_out[7], buf_u[3];
    view vin[7], vout[7], vu[3];
    int n_in = (which == WHICH_GAMMA) ? 7 : 4;
    for (int h = 0; h < 7; h++) {
        buf_in[h] = h < n_in ? in[h] : 0;
        buf_out[h] = 0;
        view a = {&buf_in[h], 1, 1, 1}, b = {&buf_out[h], 1, 1, 1};
        vin[h] = a;
        vout[h] = b;
    }
    for (int h = 0; h < 3; h++) {
        buf_u[h] = 0;
        view u = {&buf_u[h], 1, 1, 1};
        vu[h] = u;
    }
    switch (which) {
    case WHICH_PHI:
    case WHICH_PSI:
        slp_phi(variant, vin, NULL);
        for (int h = 0; h < 4; h++) out[h] = buf_in[h];
        break;
    case WHICH_CHI:
        slp_chi(variant, vin, NULL);
        for (int h = 0; h < 4; h++) out[h] = buf_in[h];
        break;
    case WHICH_ALPHA:
        slp_alpha(variant, vin, vout, NULL);
        for (int h = 0; h < 7; h++) out[h] = buf_out[h];
        break;
    case WHICH_BETA:
        slp_beta(variant, vin, vout, NULL);
        for (int h = 0; h < 7; h++) out[h] = buf_out[h];
        break;
    default:
        slp_gamma(variant, vin, vout, vu, NULL);
        for (int h = 0; h < 4; h++) out[h] = buf_out[h];
        break;
    }
}

/* ------------------------------------------------------------------ recursion */
static void leaf_product(view A, view B, view C, int64_t k, oracle_counts *cnt) {
    /* C = A B over GF(2), by the definition, on strided views. */
    int64_t m = A.rows, nw = C.wcols;
    for (int64_t i = 0; i < m; i++) {
        uint64_t *c = C.p + i * C.stride;
        for (int64_t w = 0; w < nw; w++) c[w] = 0;
        const uint64_t *a = A.p + i * A.stride;
        for (int64_t kk = 0; kk < k; kk++) {
            if (!bit_of(a, kk)) continue;
            const uint64_t *b = B.p + kk * B.stride;
            for (int64_t w = 0; w < nw; w++) c[w] ^= b[w];
        }
    }
    int64_t n = nw * 64;
    cnt->mult_bitops += (uint64_t)(2 * m * k * n - m * n);
    cnt->leaf_products += 1;
}

/* Hat C = product of Hat A and Hat B in the (alternative) basis over `depth`
 * levels: T = alpha(A-blocks), S = beta(B-blocks), Q_h = recurse(T_h, S_h),
 * C-blocks = gamma(Q) (Eqs. mb-tsrecurrence, mb-qmul, mb-qrecurrence and the
 * Kronecker closure of Sec. 2.5, applied one level at a time as in Eq. yates). */
static void rec_mul(int variant, view A, view B, view C, int depth, oracle_counts *cnt) {
    if (depth == 0) {
        leaf_product(A, B, C, A.wcols * 64, cnt);
        return;
    }
    view a[4], b[4], c[4], t[7], s[7], q[7], u[3];
    for (int i = 0; i < 4; i++) {
        a[i] = quad(A, i >> 1, i & 1);
        b[i] = quad(B, i >> 1, i & 1);
        c[i] = quad(C, i >> 1, i & 1);
    }
    for (int h = 0; h < 7; h++) {
        t[h] = alloc_view(a[0].rows, a[0].wcols);
        s[h] = alloc_view(b[0].rows, b[0].wcols);
        q[h] = alloc_view(c[0].rows, c[0].wcols);
    }
    for (int h = 0; h < 3; h++) u[h] = alloc_view(c[0].rows, c[0].wcols);
    slp_alpha(variant, a, t, &cnt->lincomb_bitops);
    slp_beta(variant, b, s, &cnt->lincomb_bitops);
    for (int h = 0; h < 7; h++) rec_mul(variant, t[h], s[h], q[h], depth - 1, cnt);
    slp_gamma(variant, q, c, u, &cnt->lincomb_bitops);
    for (int h = 0; h < 7; h++) {
        free(t[h].p);
        free(s[h].p);
        free(q[h].p);
    }
    for (int h = 0; h < 3; h++) free(u[h].p);
}

/* Basis change over `depth` levels (Yates, Eq. yates): the one-level program
 * on the four quadrants, then the same on each quadrant recursively. */
static void rec_basis(int variant, int inverse, view X, int depth, uint64_t *cnt) {
    if (depth == 0) return;
    view x[4];
    for (int i = 0; i < 4; i++) x[i] = quad(X, i >> 1, i & 1);
    if (inverse)
        slp_chi(variant, x, cnt);
    else
        slp_phi(variant, x, cnt);
    for (int i = 0; i < 4; i++) rec_basis(variant, inverse, x[i], depth - 1, cnt);
}

/* In-place basis change of an rows x cols matrix over `depth` levels:
 * inverse = 0 applies phi (= psi), inverse = 1 applies chi. */
void oracle_basis_change(int variant, int inverse, uint64_t *X, int64_t rows, int64_t cols,
                         int depth, uint64_t *bitops) {
    view v = {X, rows, cols / 64, cols / 64};
    uint64_t c = 0;
    rec_basis(variant, inverse, v, depth, &c);
    if (bitops) *bitops = c;
}

/* C = A B over GF(2) through `depth` levels of the chosen 2x2 recursion:
 * change basis (phi on A, psi on B), recurse, change basis back (chi).
 * Requires m, k, n divisible by 64 * 2^depth. Returns 0, or -1 on bad sizes. */
int oracle_strassen_gf2(int variant, const uint64_t *A, const uint64_t *B, uint64_t *C, int64_t m,
                        int64_t k, int64_t n, int depth, oracle_counts *counts) {
    int64_t unit = 64LL << depth;
    if (m % (1LL << depth) || k % unit || n % unit) return -1;
    oracle_counts cnt = {0, 0, 0, 0};
    view Ah = alloc_view(m, k / 64), Bh = alloc_view(k, n / 64), Ch = alloc_view(m, n / 64);
    memcpy(Ah.p, A, (size_t)(m * k / 64) * 8);
    memcpy(Bh.p, B, (size_t)(k * n / 64) * 8);
    rec_basis(variant, 0, Ah, depth, &cnt.basis_bitops); /* Eq. mb-mm-input-basis */
    rec_basis(variant, 0, Bh, depth, &cnt.basis_bitops);
    rec_mul(variant, Ah, Bh, Ch, depth, &cnt);
    rec_basis(variant, 1, Ch, depth, &cnt.basis_bitops); /* Eq. mb-mm-output-basis */
    memcpy(C, Ch.p, (size_t)(m * n / 64) * 8);
    free(Ah.p);
    free(Bh.p);
    free(Ch.p);
    if (counts) *counts = cnt;
    return 0;
}

/* Hat C from Hat A and Hat B, both already in the alternative basis: the
 * recursion alone, without the input or output basis changes. */
int oracle_alt_product(int variant, const uint64_t *Ah, const uint64_t *Bh, uint64_t *Ch,
                       int64_t m, int64_t k, int64_t n, int depth) {
    int64_t unit = 64LL << depth;
    if (m % (1LL << depth) || k % unit || n % unit) return -1;
    oracle_counts cnt = {0, 0, 0, 0};
    view a = {(uint64_t *)Ah, m, k / 64, k / 64}, b = {(uint64_t *)Bh, k, n / 64, n / 64};
    view c = {Ch, m, n / 64, n / 64};
    rec_mul(variant, a, b, c, depth, &cnt);
    return 0;
}

/* Packed bit transpose: out (cols x rows) = in^T (in is rows x cols). */
void oracle_transpose(const uint64_t *in, uint64_t *out, int64_t rows, int64_t cols) {
    int64_t iw = cols / 64, ow = rows / 64;
    for (int64_t w = 0; w < cols * ow; w++) out[w] = 0;
    for (int64_t i = 0; i < rows; i++)
        for (int64_t j = 0; j < cols; j++)
            if (bit_of(in + i * iw, j)) out[j * ow + (i >> 6)] |= 1ULL << (i & 63);
}
