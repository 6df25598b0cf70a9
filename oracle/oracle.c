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
 * single-qubit kinds).  Returns 0, or -(1 + index) of the first bad gate. */
int orc_apply_gates(cplx *psi, int n, int ngates, const int *kind, const int *q0,
                    const int *q1, const double *theta, const double *phi)
{
    cplx u[16];
    for (int g = 0; g < ngates; g++) {
        int d = orc_gate_matrix(kind[g], theta[g], phi[g], 0.0, 0.0, 0.0, u);
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
