/*
 * oracle.c -- plain CPU reference for the Schroedinger-style state-vector path
 * of Pednault et al., "Leveraging Secondary Storage to Simulate Deep 54-qubit
 * Sycamore Circuits" (arXiv:1910.09534).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * bench's CPU-baseline leg may load this file's library.  The product path
 * (the CUDA library) shares no code with it and never calls it.
 *
 * What it computes: the plain definition that the paper's method (gate
 * aggregation, slicing, qubit reorganisation, secondary storage) reaches up to
 * rounding: psi = U_G ... U_1 |0...0>, each gate applied one at a time to the
 * full state vector (the "Schroedinger approach", Sect. 2), in complex128.
 * For contraction deferral (Sect. 2; Appendix, EI and E2Q) it also builds the two
 * subcircuit tensors with their entanglement indices, index by index from the
 * Appendix's equations, and the contraction that removes those indices.
 *
 * Conventions: qubit q is bit q of the amplitude index (little-endian).  A
 * k-qubit matrix is 2^k x 2^k, row-major; bit j of its row/column index is the
 * value of targets[j].  Gate kinds: 0 sqrt(X), 1 sqrt(Y), 2 sqrt(W), 3 fSim.
 *
 * Every function below is pinned by the tests against closed forms, invariants
 * or brute force (full 2^n x 2^n operator products); none is "parity unpinned".
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef double complex cplx;

void orc_set_threads(int t)
{
#ifdef _OPENMP
    if (t > 0) omp_set_num_threads(t);
#else
    (void)t;
#endif
}

int orc_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/*
 * Gate matrices.
 *
 * Single-qubit gates (Sect. 3 names sqrt(X), sqrt(Y), sqrt(W) without matrices):
 * read as sqrt(P) = (I - i P) / sqrt(2) for P in {X, Y, W}, W = (X + Y)/sqrt(2).
 * fSim (Sect. 3, Eq. 1) including the detuning terms D+ (dp), D- (dm) and
 * D-,off (dmoff); basis index = b(q0) + 2 b(q1).
 * Returns the matrix dimension (2 or 4), or 0 for an unknown kind.
 */
int orc_gate_matrix(int kind, double theta, double phi, double dp, double dm,
                    double dmoff, cplx *out)
{
    const double h = 1.0 / sqrt(2.0);
    cplx p01, p10; /* off-diagonal entries of the Pauli P */
    switch (kind) {
    case 0: p01 = 1.0; p10 = 1.0; break;                        /* X */
    case 1: p01 = -I; p10 = I; break;                           /* Y */
    case 2: p01 = (1.0 - I) * h; p10 = (1.0 + I) * h; break;    /* W = (X+Y)/sqrt2 */
    case 3: {
        for (int i = 0; i < 16; i++) out[i] = 0.0;
        out[0 * 4 + 0] = 1.0;
        out[1 * 4 + 1] = cexp(I * (dp + dm)) * cos(theta);
        out[1 * 4 + 2] = -I * cexp(I * (dp - dmoff)) * sin(theta);
        out[2 * 4 + 1] = -I * cexp(I * (dp + dmoff)) * sin(theta);
        out[2 * 4 + 2] = cexp(I * (dp - dm)) * cos(theta);
        out[3 * 4 + 3] = cexp(I * (2.0 * dp - phi));
        return 4;
    }
    default: return 0;
    }
    /* (I - i P) / sqrt 2 */
    out[0] = h;
    out[1] = -I * p01 * h;
    out[2] = -I * p10 * h;
    out[3] = h;
    return 2;
}

/* One single-qubit gate: for every index i with bit q clear, the pair
 * (psi[i], psi[i + 2^q]) is multiplied by the 2x2 matrix u. */
void orc_apply_1q(cplx *psi, int n, int q, const cplx *u)
{
    const int64_t dim = (int64_t)1 << n, s = (int64_t)1 << q;
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < dim; i++) {
        if (i & s) continue;
        cplx a0 = psi[i], a1 = psi[i + s];
        psi[i] = u[0] * a0 + u[1] * a1;
        psi[i + s] = u[2] * a0 + u[3] * a1;
    }
}

/* One two-qubit gate on (q0, q1): for every index i with both bits clear, the
 * four amplitudes indexed by b0 + 2 b1 are multiplied by the 4x4 matrix u. */
void orc_apply_2q(cplx *psi, int n, int q0, int q1, const cplx *u)
{
    const int64_t dim = (int64_t)1 << n;
    const int64_t s0 = (int64_t)1 << q0, s1 = (int64_t)1 << q1;
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < dim; i++) {
        if ((i & s0) || (i & s1)) continue;
        int64_t idx[4] = {i, i + s0, i + s1, i + s0 + s1};
        cplx a[4], b[4];
        for (int c = 0; c < 4; c++) a[c] = psi[idx[c]];
        for (int r = 0; r < 4; r++) {
            b[r] = 0.0;
            for (int c = 0; c < 4; c++) b[r] += u[r * 4 + c] * a[c];
        }
        for (int r = 0; r < 4; r++) psi[idx[r]] = b[r];
    }
}

/* A k-qubit block (the paper's aggregated gate, Sect. 5): for every index i
 * whose target bits are all clear, the 2^k amplitudes i + sum_j b_j 2^t_j are
 * multiplied by the 2^k x 2^k matrix u.  Returns 0, or -1 on bad arguments. */
int orc_apply_kq(cplx *psi, int n, int k, const int *t, const cplx *u)
{
    if (k < 1 || k > 10 || k > n) return -1;
    int64_t tmask = 0;
    for (int j = 0; j < k; j++) {
        if (t[j] < 0 || t[j] >= n || (tmask >> t[j]) & 1) return -1;
        tmask |= (int64_t)1 << t[j];
    }
    const int64_t dim = (int64_t)1 << n, d = (int64_t)1 << k;
    int64_t *off = malloc(sizeof(int64_t) * d);
    for (int64_t r = 0; r < d; r++) {
        off[r] = 0;
        for (int j = 0; j < k; j++)
            if ((r >> j) & 1) off[r] += (int64_t)1 << t[j];
    }
#pragma omp parallel
    {
        cplx *a = malloc(sizeof(cplx) * d), *b = malloc(sizeof(cplx) * d);
#pragma omp for schedule(static)
        for (int64_t i = 0; i < dim; i++) {
            if (i & tmask) continue;
            for (int64_t c = 0; c < d; c++) a[c] = psi[i + off[c]];
            for (int64_t r = 0; r < d; r++) {
                cplx acc = 0.0;
                for (int64_t c = 0; c < d; c++) acc += u[r * d + c] * a[c];
                b[r] = acc;
            }
            for (int64_t r = 0; r < d; r++) psi[i + off[r]] = b[r];
        }
        free(a);
        free(b);
    }
    free(off);
    return 0;
}

/* Set psi to the computational basis state |basis>. */
void orc_basis_state(cplx *psi, int n, uint64_t basis)
{
    const int64_t dim = (int64_t)1 << n;
    memset(psi, 0, sizeof(cplx) * dim);
    psi[basis & (dim - 1)] = 1.0;
}

/* Apply a gate list in order to psi (Sect. 3 circuits; q1 ignored for the
 * single-qubit kinds).  dp, dm, dmoff: per-gate fSim detunings D+, D-, D-,off
 * of Eq. 1 (Sect. 3: the two-qubit unitaries vary with location and depth);
 * NULL means 0 for every gate.  Returns 0, or -(1 + index) of the first bad
 * gate. */
int orc_apply_gates(cplx *psi, int n, int ngates, const int *kind, const int *q0,
                    const int *q1, const double *theta, const double *phi,
                    const double *dp, const double *dm, const double *dmoff)
{
    cplx u[16];
    for (int g = 0; g < ngates; g++) {
        int d = orc_gate_matrix(kind[g], theta[g], phi[g], dp ? dp[g] : 0.0, dm ? dm[g] : 0.0,
                                dmoff ? dmoff[g] : 0.0, u);
        if (d == 2) {
            if (q0[g] < 0 || q0[g] >= n) return -(1 + g);
            orc_apply_1q(psi, n, q0[g], u);
        } else if (d == 4) {
            if (q0[g] < 0 || q0[g] >= n || q1[g] < 0 || q1[g] >= n || q0[g] == q1[g])
                return -(1 + g);
            orc_apply_2q(psi, n, q0[g], q1[g], u);
        } else {
            return -(1 + g);
        }
    }
    return 0;
}

/* Qubit-bit permutation (Sect. 4: reorganising which qubits are local/global):
 * out[pi(i)] = in[i], where pi moves bit q of i to bit perm[q].  Elements are
 * opaque `esize`-byte words, so the map is checked bit-exactly on any dtype.
 * Returns 0, or -1 if perm is not a bijection on 0..n-1. */
int orc_permute(const void *in, void *out, int n, const int *perm, int esize)
{
    int seen[64] = {0};
    for (int q = 0; q < n; q++) {
        if (perm[q] < 0 || perm[q] >= n || seen[perm[q]]) return -1;
        seen[perm[q]] = 1;
    }
    const int64_t dim = (int64_t)1 << n;
    const char *src = in;
    char *dst = out;
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < dim; i++) {
        int64_t j = 0;
        for (int q = 0; q < n; q++)
            if ((i >> q) & 1) j |= (int64_t)1 << perm[q];
        memcpy(dst + j * esize, src + i * esize, esize);
    }
    return 0;
}

/* Slice gather for secondary storage (Sect. 4, logical files indexed by the
 * sliced qubits): out[j] = in[i], where i has bits sliced[0..s-1] equal to the
 * bits of `value` and its other bits, in increasing order, equal to the bits of j.
 * scatter=1 performs the inverse move in[i] = out[j].  Opaque esize-byte words. */
int orc_slice_move(void *full, void *slice, int n, int s, const int *sliced,
                   uint64_t value, int esize, int scatter)
{
    int is_sliced[64] = {0};
    for (int j = 0; j < s; j++) {
        if (sliced[j] < 0 || sliced[j] >= n || is_sliced[sliced[j]]) return -1;
        is_sliced[sliced[j]] = 1;
    }
    int64_t fixed = 0;
    for (int j = 0; j < s; j++)
        if ((value >> j) & 1) fixed |= (int64_t)1 << sliced[j];
    const int64_t count = (int64_t)1 << (n - s);
    char *f = full, *sl = slice;
#pragma omp parallel for schedule(static)
    for (int64_t j = 0; j < count; j++) {
        int64_t i = fixed;
        int b = 0;
        for (int q = 0; q < n; q++) {
            if (is_sliced[q]) continue;
            if ((j >> b) & 1) i |= (int64_t)1 << q;
            b++;
        }
        if (scatter) memcpy(f + i * esize, sl + j * esize, esize);
        else memcpy(sl + j * esize, f + i * esize, esize);
    }
    return 0;
}

/* Reductions over p_i = |psi_i|^2: norm = sum p, sum_p2_scaled = 2^n sum p^2
 * (about 2 for Porter-Thomas statistics), xeb = 2^n sum p^2 - 1 (linear
 * cross-entropy benchmark of the ideal distribution). */
void orc_reduce(const cplx *psi, int n, double *norm, double *sum_p2_scaled, double *xeb)
{
    const int64_t dim = (int64_t)1 << n;
    double s1 = 0.0, s2 = 0.0;
#pragma omp parallel for reduction(+ : s1, s2) schedule(static)
    for (int64_t i = 0; i < dim; i++) {
        double p = creal(psi[i]) * creal(psi[i]) + cimag(psi[i]) * cimag(psi[i]);
        s1 += p;
        s2 += p * p;
    }
    *norm = s1;
    *sum_p2_scaled = ldexp(s2, n);
    *xeb = *sum_p2_scaled - 1.0;
}

/*
 * Contraction deferral (Sect. 2) with the synthesized operations EI and E2Q
 * defined in the Appendix.
 *
 * side[q] = 0 puts qubit q in tensor 1, side[q] = 1 in tensor 2.  Each tensor
 * starts as |0..0> over its own qubits, qubit positions 0.. in increasing qubit
 * order.  Gates are taken in list order.  A gate whose qubits are all on one
 * side acts on that side's tensor at its qubits' positions (orc_apply_1q /
 * orc_apply_2q).  A two-qubit gate G that bridges qubit a (side 0) and qubit b
 * (side 1) is the j-th bridging gate: it appends two indices to each tensor, at
 * positions m and m + 1 where m is the tensor's index count before the gate, and
 *   EI  (tensor 1): T1'[.., a'' at p(a), a' at m, a at m+1]
 *                     = delta(a'', a') T1[.., a at p(a)]
 *   E2Q (tensor 2): T2'[.., b'' at p(b), a' at m, a at m+1]
 *                     = sum_b G[a', b''; a, b] T2[.., b at p(b)]
 * where G[x'', y''; x, y] is the gate's matrix element from input (x, y) to
 * output (x'', y'') with x the value of qubit a and y that of qubit b (the gate's
 * own index is b(q0) + 2 b(q1), whichever of a, b is q0).  Qubit a keeps position
 * p(a) for its new index a''.  So tensor 1 ends with its n1 qubits at positions
 * 0..n1-1 and pair j's (a', a) at n1 + 2j, n1 + 2j + 1; tensor 2 likewise.
 *
 * t1, t2: room for 2^(n1 + 2c) and 2^(n2 + 2c) amplitudes, c = number of
 * bridging gates; with t1 == NULL only c is computed.  dp, dm, dmoff (fSim
 * detunings) may be NULL for zero.  Returns c, or -(1 + g) for a bad gate g, or
 * -1000000 for a bad side vector.
 */
static int64_t put_bit(int64_t i, int p, int v)
{
    return (i & ~((int64_t)1 << p)) | ((int64_t)v << p);
}

int orc_split_tensors(int n, int ngates, const int *kind, const int *q0, const int *q1,
                      const double *theta, const double *phi, const double *dp,
                      const double *dm, const double *dmoff, const int *side, cplx *t1,
                      cplx *t2)
{
    int pos[64], bits[2] = {0, 0}, c = 0;
    if (n < 1 || n > 62) return -1000000;
    for (int q = 0; q < n; q++) {
        if (side[q] != 0 && side[q] != 1) return -1000000;
        pos[q] = bits[side[q]]++;
    }
    if (bits[0] == 0 || bits[1] == 0) return -1000000;
    for (int g = 0; g < ngates; g++) { /* validate and count the bridging gates first */
        cplx u[16];
        int d = orc_gate_matrix(kind[g], theta[g], phi[g], 0.0, 0.0, 0.0, u);
        if (d == 0 || q0[g] < 0 || q0[g] >= n) return -(1 + g);
        if (d == 4) {
            if (q1[g] < 0 || q1[g] >= n || q1[g] == q0[g]) return -(1 + g);
            if (side[q0[g]] != side[q1[g]]) c++;
        }
    }
    if (!t1) return c;
    cplx *T[2] = {t1, t2};
    for (int s = 0; s < 2; s++) {
        memset(T[s], 0, sizeof(cplx) << bits[s]);
        T[s][0] = 1.0;
    }
    cplx *tmp = NULL;
    for (int g = 0; g < ngates; g++) {
        cplx u[16];
        int d = orc_gate_matrix(kind[g], theta[g], phi[g], dp ? dp[g] : 0.0, dm ? dm[g] : 0.0,
                                dmoff ? dmoff[g] : 0.0, u);
        if (d == 2) {
            int s = side[q0[g]];
            orc_apply_1q(T[s], bits[s], pos[q0[g]], u);
            continue;
        }
        int sa = side[q0[g]], sb = side[q1[g]];
        if (sa == sb) {
            orc_apply_2q(T[sa], bits[sa], pos[q0[g]], pos[q1[g]], u);
            continue;
        }
        const int a_is_q0 = sa == 0;
        const int a = a_is_q0 ? q0[g] : q1[g], b = a_is_q0 ? q1[g] : q0[g];
        /* EI on tensor 1 */
        {
            const int m = bits[0], pa = pos[a];
            const int64_t dim = (int64_t)1 << (m + 2);
            tmp = (cplx *)realloc(tmp, sizeof(cplx) * (size_t)dim);
            if (!tmp) return -2000000;
            for (int64_t i = 0; i < dim; i++) {
                const int64_t low = i & (((int64_t)1 << m) - 1);
                const int app = (int)((low >> pa) & 1); /* a'' */
                const int ap = (int)((i >> m) & 1);     /* a'  */
                const int av = (int)((i >> (m + 1)) & 1); /* a */
                tmp[i] = app == ap ? T[0][put_bit(low, pa, av)] : 0.0;
            }
            memcpy(T[0], tmp, sizeof(cplx) * (size_t)dim);
            bits[0] = m + 2;
        }
        /* E2Q on tensor 2 */
        {
            const int m = bits[1], pb = pos[b];
            const int64_t dim = (int64_t)1 << (m + 2);
            tmp = (cplx *)realloc(tmp, sizeof(cplx) * (size_t)dim);
            if (!tmp) return -2000000;
            for (int64_t i = 0; i < dim; i++) {
                const int64_t low = i & (((int64_t)1 << m) - 1);
                const int bpp = (int)((low >> pb) & 1); /* b'' */
                const int ap = (int)((i >> m) & 1);     /* a'  */
                const int av = (int)((i >> (m + 1)) & 1); /* a */
                const int row = a_is_q0 ? ap + 2 * bpp : bpp + 2 * ap;
                cplx acc = 0.0;
                for (int bv = 0; bv < 2; bv++) {
                    const int col = a_is_q0 ? av + 2 * bv : bv + 2 * av;
                    acc += u[row * 4 + col] * T[1][put_bit(low, pb, bv)];
                }
                tmp[i] = acc;
            }
            memcpy(T[1], tmp, sizeof(cplx) * (size_t)dim);
            bits[1] = m + 2;
        }
    }
    free(tmp);
    return c;
}

/*
 * The contraction that removes the entanglement indices (Appendix: the sum over
 * every pair's (a', a) of the product of the two tensors).  t1 holds n1 qubit
 * indices at positions 0..n1-1 followed by e entanglement bits, t2 likewise with
 * n2 qubits and the same e bits in the same order.  qa[i] / qb[j] name the qubit
 * at position i of t1 / j of t2.  Writes psi (n1 + n2 qubits, logical order):
 *   psi[sum_i x_i 2^qa[i] + sum_j y_j 2^qb[j]] = sum_k t1[x + k 2^n1] t2[y + k 2^n2].
 */
void orc_contract(const cplx *t1, int n1, const cplx *t2, int n2, int e, const int *qa,
                  const int *qb, cplx *psi)
{
    const int64_t X = (int64_t)1 << n1, Y = (int64_t)1 << n2, E = (int64_t)1 << e;
#pragma omp parallel for schedule(static)
    for (int64_t y = 0; y < Y; y++) {
        int64_t ly = 0;
        for (int j = 0; j < n2; j++)
            if ((y >> j) & 1) ly |= (int64_t)1 << qb[j];
        for (int64_t x = 0; x < X; x++) {
            int64_t lx = 0;
            for (int i = 0; i < n1; i++)
                if ((x >> i) & 1) lx |= (int64_t)1 << qa[i];
            cplx acc = 0.0;
            for (int64_t k = 0; k < E; k++) acc += t1[x + k * X] * t2[y + k * Y];
            psi[lx | ly] = acc;
        }
    }
}
