/*
 * sqd_oracle.c -- plain CPU oracle for the SQD Hamiltonian on a selected
 * alpha x beta determinant subspace.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the CPU
 * baseline leg of the benchmark load this library.  The product path (the
 * CUDA library and its Python binding) never calls it, and the two share no
 * code, header, table or constant.
 *
 * What it computes (arXiv 2601.16169, Sections I-II): the lowest eigenpairs
 * of P H P, where P projects onto span{|I_a I_b>} over sampled alpha strings
 * I_a and beta strings I_b, and H is the electronic Hamiltonian given by
 * one-electron integrals h_pq and two-electron integrals (pq|rs) through the
 * Slater-Condon rules (the paper's Hij / ZeroExcite / OneExcite / TwoExcite,
 * Section II, Table I; rules after Knowles-Handy, cited in Section IV).
 *
 * Readings where the paper is silent:
 *  - H = E_core + sum_{pq,s} h_pq a+_{ps} a_{qs}
 *        + 1/2 sum_{pqrs,st} (pq|rs) a+_{ps} a+_{rt} a_{st} a_{qs}
 *    with spatial orbitals and chemist-notation integrals.
 *  - A determinant is the 2*norb spin-orbital occupation with the alpha block
 *    first: spin-orbital k < norb is alpha orbital k, spin-orbital norb + k is
 *    beta orbital k, and |n> = prod_{k ascending} (a+_k)^{n_k} |0>.  So
 *    a_k|n> = (-1)^{sum_{j<k} n_j} n_k |n - e_k>.
 *  - Every matrix element is computed from that operator definition: the
 *    sign by applying the creation/annihilation operators one at a time, the
 *    value from the rules below written for arbitrary real (not necessarily
 *    symmetric) integrals, so that an index transposition cannot hide behind
 *    integral symmetry.
 *
 * Nothing here uses the alpha/beta factorisation of the GPU path: every
 * H_IJ is the generic spin-orbital element of two full determinants.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef unsigned __int128 u128;

/* ---------------------------------------------------------------- bits -- */

static inline int popc128(u128 x) {
    return __builtin_popcountll((uint64_t)x) + __builtin_popcountll((uint64_t)(x >> 64));
}

static inline int occ(u128 d, int k) { return (int)((d >> k) & 1u); }

/* number of occupied spin-orbitals with index strictly below k */
static inline int count_below(u128 d, int k) {
    u128 mask = (k == 0) ? (u128)0 : ((((u128)1) << k) - 1);
    return popc128(d & mask);
}

static inline u128 det_of(uint64_t a, uint64_t b, int norb) {
    return (u128)a | ((u128)b << norb);
}

/* Apply a_k to *d.  Returns the sign (+1/-1) or 0 if orbital k is empty. */
static int apply_annihilate(u128 *d, int k) {
    if (!occ(*d, k)) return 0;
    int s = (count_below(*d, k) & 1) ? -1 : 1;
    *d &= ~(((u128)1) << k);
    return s;
}

/* Apply a+_k to *d.  Returns the sign or 0 if orbital k is already filled. */
static int apply_create(u128 *d, int k) {
    if (occ(*d, k)) return 0;
    int s = (count_below(*d, k) & 1) ? -1 : 1;
    *d |= (((u128)1) << k);
    return s;
}

/* lowest set bit index of a nonzero 128-bit word */
static int lowest_bit(u128 x) {
    uint64_t lo = (uint64_t)x;
    if (lo) return __builtin_ctzll(lo);
    return 64 + __builtin_ctzll((uint64_t)(x >> 64));
}

/* ---------------------------------------------------- spin-orbital ints -- */

typedef struct {
    int norb;
    const double *h; /* norb*norb, h[p*norb+q] = h_pq */
    const double *V; /* norb^4, V[((p*norb+q)*norb+r)*norb+s] = (pq|rs) */
    double ecore;
} ham_t;

static inline int spin_of(const ham_t *H, int k) { return k >= H->norb; }
static inline int spat(const ham_t *H, int k) { return k >= H->norb ? k - H->norb : k; }

/* h in the spin-orbital basis: zero unless both spin-orbitals have one spin */
static inline double h_so(const ham_t *H, int k, int l) {
    if (spin_of(H, k) != spin_of(H, l)) return 0.0;
    int n = H->norb;
    return H->h[spat(H, k) * n + spat(H, l)];
}

/* (kl|mn) in the spin-orbital basis */
static inline double v_so(const ham_t *H, int k, int l, int m, int nn) {
    if (spin_of(H, k) != spin_of(H, l) || spin_of(H, m) != spin_of(H, nn)) return 0.0;
    int n = H->norb;
    size_t idx = (((size_t)spat(H, k) * n + spat(H, l)) * n + spat(H, m)) * n + spat(H, nn);
    return H->V[idx];
}

/* ------------------------------------------------------ Slater-Condon --- */

/*
 * <I|H|J> for two determinants (bra I, ket J) given as 2*norb-bit
 * occupations.  Rules (Slater-Condon, Knowles-Handy; the paper's
 * ZeroExcite / OneExcite / TwoExcite):
 *   I == J : E_core + sum_k h_kk + 1/2 sum_{k,l in I} [(kk|ll) - (kl|lk)]
 *   single, x in I\J, y in J\I :
 *        <I|a+_x a_y|J> * ( h_xy + sum_{k in I&J} 1/2[(xy|kk) + (kk|xy)
 *                                                   - (xk|ky) - (ky|xk)] )
 *   double, x1<x2 in I\J, y1<y2 in J\I :
 *        <I|a+_x1 a+_x2 a_y2 a_y1|J> * 1/2[(x1y1|x2y2) + (x2y2|x1y1)
 *                                         - (x1y2|x2y1) - (x2y1|x1y2)]
 *   otherwise 0.
 * Each rule is the sum of the terms of H that connect J to I, written out
 * for arbitrary real integrals.
 */
static double hij_det(const ham_t *H, u128 I, u128 J) {
    int nso = 2 * H->norb;
    u128 D = I ^ J;
    int nd = popc128(D);
    if (nd == 0) {
        double e = H->ecore;
        for (int k = 0; k < nso; k++) {
            if (!occ(I, k)) continue;
            e += h_so(H, k, k);
            for (int l = 0; l < nso; l++) {
                if (!occ(I, l)) continue;
                e += 0.5 * (v_so(H, k, k, l, l) - v_so(H, k, l, l, k));
            }
        }
        return e;
    }
    if (nd == 2) {
        int x = lowest_bit(I & D);
        int y = lowest_bit(J & D);
        u128 t = J;
        int s = apply_annihilate(&t, y);
        s *= apply_create(&t, x);
        if (s == 0 || t != I) return 0.0; /* cannot happen for nd == 2 */
        double v = h_so(H, x, y);
        u128 common = I & J;
        for (int k = 0; k < nso; k++) {
            if (!occ(common, k)) continue;
            v += 0.5 * (v_so(H, x, y, k, k) + v_so(H, k, k, x, y)
                        - v_so(H, x, k, k, y) - v_so(H, k, y, x, k));
        }
        return s * v;
    }
    if (nd == 4) {
        u128 a = I & D, b = J & D;
        int x1 = lowest_bit(a);
        int x2 = lowest_bit(a & ~(((u128)1) << x1));
        int y1 = lowest_bit(b);
        int y2 = lowest_bit(b & ~(((u128)1) << y1));
        u128 t = J;
        int s = apply_annihilate(&t, y1);
        s *= apply_annihilate(&t, y2);
        s *= apply_create(&t, x2);
        s *= apply_create(&t, x1);
        if (s == 0 || t != I) return 0.0;
        double v = 0.5 * (v_so(H, x1, y1, x2, y2) + v_so(H, x2, y2, x1, y1)
                          - v_so(H, x1, y2, x2, y1) - v_so(H, x2, y1, x1, y2));
        return s * v;
    }
    return 0.0;
}

/* <I_a I_b | H | J_a J_b> */
double oracle_hij(int norb, const double *h, const double *V, double ecore,
                  uint64_t ia, uint64_t ib, uint64_t ja, uint64_t jb) {
    ham_t H = {norb, h, V, ecore};
    return hij_det(&H, det_of(ia, ib, norb), det_of(ja, jb, norb));
}

/* ------------------------------------------------------------ dense H --- */

/*
 * Dense P H P, determinant index I = ia * nb + ib (C stored as an
 * |I_a| x |I_b| row-major matrix).  out is N*N row-major, out[I*N+J] = <I|H|J>.
 */
int oracle_dense_h(int norb, const double *h, const double *V, double ecore,
                   const uint64_t *sa, int64_t na, const uint64_t *sb, int64_t nb,
                   double *out) {
    ham_t H = {norb, h, V, ecore};
    int64_t N = na * nb;
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t I = 0; I < N; I++) {
        u128 dI = det_of(sa[I / nb], sb[I % nb], norb);
        for (int64_t J = 0; J < N; J++) {
            u128 dJ = det_of(sa[J / nb], sb[J % nb], norb);
            out[I * N + J] = hij_det(&H, dI, dJ);
        }
    }
    return 0;
}

/* --------------------------------------------------------- neighbours --- */

/*
 * For each string s[i], the indices j (ascending) with popcount(s[i]^s[j])
 * in {0, 2, 4}: the strings reachable by at most a double excitation.
 * Brute-force scan over all pairs.  Two passes: with idx == NULL only the
 * offsets off[0..n] are written.
 */
int oracle_neighbours(const uint64_t *s, int64_t n, int64_t *off, int32_t *idx) {
    if (!idx) {
        off[0] = 0;
        for (int64_t i = 0; i < n; i++) {
            int64_t c = 0;
            for (int64_t j = 0; j < n; j++) {
                int d = __builtin_popcountll(s[i] ^ s[j]);
                if (d <= 4) c++;
            }
            off[i + 1] = off[i] + c;
        }
        return 0;
    }
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t i = 0; i < n; i++) {
        int64_t o = off[i];
        for (int64_t j = 0; j < n; j++) {
            int d = __builtin_popcountll(s[i] ^ s[j]);
            if (d <= 4) idx[o++] = (int32_t)j;
        }
    }
    return 0;
}

static int64_t *nbr_off(const uint64_t *s, int64_t n, int32_t **idx_out) {
    int64_t *off = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n + 1));
    if (!off) return NULL;
    /* count in parallel */
    int64_t *cnt = (int64_t *)calloc((size_t)n, sizeof(int64_t));
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t i = 0; i < n; i++) {
        int64_t c = 0;
        for (int64_t j = 0; j < n; j++)
            if (__builtin_popcountll(s[i] ^ s[j]) <= 4) c++;
        cnt[i] = c;
    }
    off[0] = 0;
    for (int64_t i = 0; i < n; i++) off[i + 1] = off[i] + cnt[i];
    free(cnt);
    int32_t *idx = (int32_t *)malloc(sizeof(int32_t) * (size_t)(off[n] ? off[n] : 1));
    oracle_neighbours(s, n, off, idx);
    *idx_out = idx;
    return off;
}

/* --------------------------------------------------------- sigma = HC --- */

/*
 * Matrix-free sigma = (P H P) C for nvec vectors, C and sigma laid out as
 * [nvec][na][nb].  If rows != NULL only the nrows listed determinant rows
 * are computed and sigma is [nvec][nrows] (row-sample mode).
 *
 * For row I = (I_a, I_b) every candidate J = (J_a, J_b) is taken from the
 * brute-force neighbour lists of I_a and I_b, kept if the total number of
 * differing spin-orbitals is at most 4, and contributes <I|H|J> C_J with the
 * generic element above.
 */
int oracle_sigma(int norb, const double *h, const double *V, double ecore,
                 const uint64_t *sa, int64_t na, const uint64_t *sb, int64_t nb,
                 const double *C, int nvec, double *sigma,
                 const int64_t *rows, int64_t nrows) {
    ham_t H = {norb, h, V, ecore};
    int32_t *ia_idx = NULL, *ib_idx = NULL;
    int64_t *ia_off = nbr_off(sa, na, &ia_idx);
    int64_t *ib_off = (sa == sb && na == nb) ? ia_off : nbr_off(sb, nb, &ib_idx);
    if (sa == sb && na == nb) ib_idx = ia_idx;
    if (!ia_off || !ib_off) return -2;
    if (nvec < 1 || nvec > 64) return -1;
    int64_t N = na * nb;
    int64_t R = rows ? nrows : N;
#pragma omp parallel for schedule(dynamic, 32)
    for (int64_t r = 0; r < R; r++) {
        int64_t I = rows ? rows[r] : r;
        int64_t ia = I / nb, ib = I % nb;
        u128 dI = det_of(sa[ia], sb[ib], norb);
        double acc[64];
        int nv = nvec;
        for (int v = 0; v < nv; v++) acc[v] = 0.0;
        for (int64_t x = ia_off[ia]; x < ia_off[ia + 1]; x++) {
            int64_t ja = ia_idx[x];
            int da = __builtin_popcountll(sa[ia] ^ sa[ja]);
            for (int64_t y = ib_off[ib]; y < ib_off[ib + 1]; y++) {
                int64_t jb = ib_idx[y];
                int db = __builtin_popcountll(sb[ib] ^ sb[jb]);
                if (da + db > 4) continue;
                double hv = hij_det(&H, dI, det_of(sa[ja], sb[jb], norb));
                if (hv == 0.0) continue;
                int64_t J = ja * nb + jb;
                for (int v = 0; v < nv; v++) acc[v] += hv * C[(int64_t)v * N + J];
            }
        }
        for (int v = 0; v < nv; v++) sigma[(int64_t)v * R + r] = acc[v];
    }
    if (ib_off != ia_off) { free(ib_off); free(ib_idx); }
    free(ia_off); free(ia_idx);
    return 0;
}

/* diagonal H_II for all determinants, [na][nb] */
int oracle_diag(int norb, const double *h, const double *V, double ecore,
                const uint64_t *sa, int64_t na, const uint64_t *sb, int64_t nb,
                double *out) {
    ham_t H = {norb, h, V, ecore};
#pragma omp parallel for schedule(static)
    for (int64_t I = 0; I < na * nb; I++) {
        u128 d = det_of(sa[I / nb], sb[I % nb], norb);
        out[I] = hij_det(&H, d, d);
    }
    return 0;
}

/* ------------------------------------------------- excitation tables --- */

/*
 * Same-spin excitation tables by brute force: for every string I (row) and
 * every string J of the set (ascending index) that differs from I in exactly
 * one orbital (kind 1) or two orbitals (kind 2), one entry.
 *
 * kind 1 entry: target J, p = the orbital in J not in I, q = the orbital in I
 *   not in J, sign = <J| a+_p a_q |I>.
 * kind 2 entry: target J, i < j the orbitals in I not in J, a < b the
 *   orbitals in J not in I, sign = <J| a+_a a+_b a_j a_i |I>.
 * val = <I|H_s|J>, the element of the one-spin Hamiltonian (h plus the
 *   same-spin two-electron part), computed by the generic element on the
 *   determinants (I, empty) and (J, empty).
 *
 * With tgt == NULL only the row offsets off[0..n] are written.
 * orb receives 2 (kind 1: p, q) or 4 (kind 2: i, j, a, b) bytes per entry.
 */
int oracle_excitations(int norb, const double *h, const double *V, int kind,
                       const uint64_t *s, int64_t n, int64_t *off, int32_t *tgt,
                       uint8_t *orb, int8_t *sign, double *val) {
    ham_t H = {norb, h, V, 0.0};
    int want = 2 * kind;
    if (!tgt) {
        off[0] = 0;
        for (int64_t i = 0; i < n; i++) {
            int64_t c = 0;
            for (int64_t j = 0; j < n; j++)
                if (__builtin_popcountll(s[i] ^ s[j]) == want) c++;
            off[i + 1] = off[i] + c;
        }
        return 0;
    }
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t i = 0; i < n; i++) {
        int64_t o = off[i];
        for (int64_t j = 0; j < n; j++) {
            uint64_t d = s[i] ^ s[j];
            if (__builtin_popcountll(d) != want) continue;
            uint64_t gone = s[i] & d, new_ = s[j] & d;
            u128 t = (u128)s[i];
            int sg;
            if (kind == 1) {
                int p = __builtin_ctzll(new_), q = __builtin_ctzll(gone);
                sg = apply_annihilate(&t, q);
                sg *= apply_create(&t, p);
                orb[2 * o] = (uint8_t)p;
                orb[2 * o + 1] = (uint8_t)q;
            } else {
                int ii = __builtin_ctzll(gone);
                int jj = __builtin_ctzll(gone & (gone - 1));
                int aa = __builtin_ctzll(new_);
                int bb = __builtin_ctzll(new_ & (new_ - 1));
                sg = apply_annihilate(&t, ii);
                sg *= apply_annihilate(&t, jj);
                sg *= apply_create(&t, bb);
                sg *= apply_create(&t, aa);
                orb[4 * o] = (uint8_t)ii;
                orb[4 * o + 1] = (uint8_t)jj;
                orb[4 * o + 2] = (uint8_t)aa;
                orb[4 * o + 3] = (uint8_t)bb;
            }
            tgt[o] = (int32_t)j;
            sign[o] = (int8_t)sg;
            val[o] = hij_det(&H, (u128)s[i], (u128)s[j]);
            o++;
        }
    }
    return 0;
}

/* one-spin diagonal energies E_s(I) = <I,empty|H|I,empty> without E_core */
int oracle_string_energy(int norb, const double *h, const double *V,
                         const uint64_t *s, int64_t n, double *out) {
    ham_t H = {norb, h, V, 0.0};
    for (int64_t i = 0; i < n; i++) out[i] = hij_det(&H, (u128)s[i], (u128)s[i]);
    return 0;
}

/* --------------------------------------------------------------- RDMs --- */

static int64_t find_str(const uint64_t *s, int64_t n, uint64_t x) {
    int64_t lo = 0, hi = n - 1;
    while (lo <= hi) {
        int64_t mid = (lo + hi) / 2;
        if (s[mid] == x) return mid;
        if (s[mid] < x) lo = mid + 1; else hi = mid - 1;
    }
    return -1;
}

/* Look up a determinant in the product subspace; -1 if outside. */
static int64_t find_det(int norb, const uint64_t *sa, int64_t na,
                        const uint64_t *sb, int64_t nb, u128 d) {
    uint64_t mask = (norb == 64) ? ~0ull : ((1ull << norb) - 1);
    uint64_t a = (uint64_t)d & mask;
    uint64_t b = (uint64_t)(d >> norb) & mask;
    int64_t ia = find_str(sa, na, a);
    if (ia < 0) return -1;
    int64_t ib = find_str(sb, nb, b);
    if (ib < 0) return -1;
    return ia * nb + ib;
}

/*
 * Expectation values of operator strings in the state C (one vector, [na][nb]):
 *   nops == 2 : <C| a+_k a_l |C>                 (ops = {k, l})
 *   nops == 4 : <C| a+_k a+_l a_m a_n |C>        (ops = {k, l, m, n})
 * with spin-orbital indices k, l, m, n.  Each entry e of the nent requested
 * is sum_J sum_K C_K C_J <K|op|J>, the operator applied right to left to
 * every determinant J and the result looked up in the subspace (the RDM of
 * the state projected on the subspace, which is the state itself).
 */
int oracle_expect(int norb, const uint64_t *sa, int64_t na, const uint64_t *sb,
                  int64_t nb, const double *C, int nops, const int32_t *ops,
                  int64_t nent, double *out) {
    int64_t N = na * nb;
    for (int64_t e = 0; e < nent; e++) {
        const int32_t *o = ops + e * nops;
        double acc = 0.0;
#pragma omp parallel for reduction(+ : acc) schedule(static)
        for (int64_t J = 0; J < N; J++) {
            double cj = C[J];
            if (cj == 0.0) continue;
            u128 d = det_of(sa[J / nb], sb[J % nb], norb);
            int s = 1;
            if (nops == 2) {
                s *= apply_annihilate(&d, o[1]);
                if (!s) continue;
                s *= apply_create(&d, o[0]);
            } else {
                s *= apply_annihilate(&d, o[3]);
                if (!s) continue;
                s *= apply_annihilate(&d, o[2]);
                if (!s) continue;
                s *= apply_create(&d, o[1]);
                if (!s) continue;
                s *= apply_create(&d, o[0]);
            }
            if (!s) continue;
            int64_t K = find_det(norb, sa, na, sb, nb, d);
            if (K < 0) continue;
            acc += s * C[K] * cj;
        }
        out[e] = acc;
    }
    return 0;
}
