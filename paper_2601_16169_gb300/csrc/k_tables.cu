// Excitation tables of a string set (singles, doubles), one-spin string
// terms and the determinant diagonal.
//
// Construction follows the paper's GenerateExcitation step (Section II,
// Table I) restated for one 64-bit word per string: every candidate
// I - q + p (or I - i - j + a + b) is looked up in the sorted set by binary
// search; hits are counted (pass 1), offsets come from a scan, hits are
// written as 64-bit keys (row << 32 | target) (pass 2) and a global sort of
// the keys puts every row's entries in ascending target order, which makes
// the table independent of the enumeration order.  Orbitals, signs and
// Slater-Condon values are then derived from (row, target) alone.
#include "sqd_internal.cuh"

__device__ __forceinline__ int64_t find_string(const uint64_t *__restrict__ s, int64_t n,
                                               uint64_t x) {
    int64_t lo = 0, hi = n;
    while (lo < hi) {
        int64_t mid = (lo + hi) >> 1;
        uint64_t v = __ldg(s + mid);
        if (v < x) lo = mid + 1; else hi = mid;
    }
    return (lo < n && __ldg(s + lo) == x) ? lo : -1;
}

// mask of orbitals strictly between x and y
__device__ __forceinline__ uint64_t between_mask(int x, int y) {
    int lo = min(x, y), hi = max(x, y);
    uint64_t below_hi = (hi >= 64) ? ~0ull : ((1ull << hi) - 1);
    uint64_t upto_lo = (lo >= 63) ? ~0ull : ((1ull << (lo + 1)) - 1);
    return below_hi & ~upto_lo;
}

// sign of a+_p a_q acting on X (q occupied, p empty)
__device__ __forceinline__ int single_sign(uint64_t X, int p, int q) {
    return (__popcll(X & between_mask(p, q)) & 1) ? -1 : 1;
}

// One warp per string.  Lanes take occupied orbitals (kind 1) or occupied
// pairs (kind 2); the inner loops run over empty orbitals / pairs.
template <bool FILL>
__global__ void k_excitations(const uint64_t *__restrict__ s, int64_t n, int norb, int kind,
                              int64_t *__restrict__ counts, const int64_t *__restrict__ off,
                              int64_t *__restrict__ cursor, uint64_t *__restrict__ keys) {
    int64_t row = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    int lane = threadIdx.x & 31;
    if (row >= n) return;
    uint64_t I = s[row];
    uint64_t full = (norb == 64) ? ~0ull : ((1ull << norb) - 1);
    uint64_t empty = full & ~I;
    int ne = __popcll(I);
    int64_t cnt = 0;
    if (kind == 1) {
        for (int t = lane; t < ne; t += 32) {
            // t-th occupied orbital
            uint64_t m = I;
            for (int k = 0; k < t; k++) m &= m - 1;
            int q = __ffsll((long long)m) - 1;
            uint64_t e = empty;
            while (e) {
                int p = __ffsll((long long)e) - 1;
                e &= e - 1;
                uint64_t J = I ^ (1ull << q) ^ (1ull << p);
                int64_t j = find_string(s, n, J);
                if (j >= 0) {
                    if (FILL) {
                        int64_t slot = atomicAdd((unsigned long long *)&cursor[row], 1ull);
                        keys[slot] = ((uint64_t)row << 32) | (uint64_t)j;
                    }
                    cnt++;
                }
            }
        }
    } else {
        int npairs = ne * (ne - 1) / 2;
        for (int t = lane; t < npairs; t += 32) {
            // t-th pair (i<j) of occupied orbitals in lexicographic order
            int a_idx = 0, rem = t;
            while (rem >= ne - 1 - a_idx) {
                rem -= ne - 1 - a_idx;
                a_idx++;
            }
            int b_idx = a_idx + 1 + rem;
            uint64_t m = I;
            for (int k = 0; k < a_idx; k++) m &= m - 1;
            int oi = __ffsll((long long)m) - 1;
            for (int k = a_idx; k < b_idx; k++) m &= m - 1;
            int oj = __ffsll((long long)m) - 1;
            uint64_t base = I ^ (1ull << oi) ^ (1ull << oj);
            uint64_t e1 = empty;
            while (e1) {
                int va = __ffsll((long long)e1) - 1;
                e1 &= e1 - 1;
                uint64_t e2 = e1;
                while (e2) {
                    int vb = __ffsll((long long)e2) - 1;
                    e2 &= e2 - 1;
                    uint64_t J = base | (1ull << va) | (1ull << vb);
                    int64_t j = find_string(s, n, J);
                    if (j >= 0) {
                        if (FILL) {
                            int64_t slot = atomicAdd((unsigned long long *)&cursor[row], 1ull);
                            keys[slot] = ((uint64_t)row << 32) | (uint64_t)j;
                        }
                        cnt++;
                    }
                }
            }
        }
    }
    if (!FILL) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) cnt += __shfl_down_sync(0xffffffffu, cnt, o);
        if (lane == 0) counts[row] = cnt;
    }
}

int launch_count_excitations(sqd_ctx *ctx, const uint64_t *s, int64_t n, int norb, int kind,
                             int64_t *counts) {
    if (n == 0) return SQD_OK;
    k_excitations<false><<<grid_1d(n * 32, 256), 256, 0, ctx->stream>>>(
        s, n, norb, kind, counts, nullptr, nullptr, nullptr);
    SQD_LAUNCHED(ctx);
    return SQD_OK;
}

int launch_fill_excitations(sqd_ctx *ctx, const uint64_t *s, int64_t n, int norb, int kind,
                            const int64_t *off, int64_t *cursor, uint64_t *keys) {
    if (n == 0) return SQD_OK;
    SQD_CUDA(ctx, cudaMemcpyAsync(cursor, off, sizeof(int64_t) * n, cudaMemcpyDeviceToDevice,
                                  ctx->stream));
    k_excitations<true><<<grid_1d(n * 32, 256), 256, 0, ctx->stream>>>(
        s, n, norb, kind, nullptr, off, cursor, keys);
    SQD_LAUNCHED(ctx);
    return SQD_OK;
}

__device__ __forceinline__ double Vat(const double *__restrict__ V, int norb, int p, int q,
                                      int r, int s_) {
    return __ldg(V + ((((int64_t)p * norb + q) * norb + r) * norb + s_));
}

// Single I -> J: p = orbital of J not in I (created), q = orbital of I not in
// J (annihilated).  <I|H_s|J> = sign * (h_qp + sum_{k in I&J} [(qp|kk) - (qk|kp)]).
__global__ void k_finalize_singles(const uint64_t *__restrict__ s, int norb,
                                   const uint64_t *__restrict__ keys, int64_t nnz,
                                   const double *__restrict__ h, const double *__restrict__ V,
                                   int32_t *__restrict__ tgt, uint16_t *__restrict__ pq,
                                   int8_t *__restrict__ sgn, double *__restrict__ val) {
    int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= nnz) return;
    uint64_t key = keys[e];
    int64_t row = (int64_t)(key >> 32), j = (int64_t)(key & 0xffffffffu);
    uint64_t I = s[row], J = s[j];
    int p = __ffsll((long long)(J & ~I)) - 1;
    int q = __ffsll((long long)(I & ~J)) - 1;
    int sg = single_sign(I, p, q);
    double v = __ldg(h + (int64_t)q * norb + p);
    uint64_t common = I & J;
    while (common) {
        int k = __ffsll((long long)common) - 1;
        common &= common - 1;
        v += Vat(V, norb, q, p, k, k) - Vat(V, norb, q, k, k, p);
    }
    tgt[e] = (int32_t)j;
    pq[e] = (uint16_t)(p * norb + q);
    sgn[e] = (int8_t)sg;
    val[e] = sg * v;
}

// Double I -> J: i<j of I not in J, a<b of J not in I.
// sign = <J|a+_a a+_b a_j a_i|I> = s(I; i->a) * s(I-i+a; j->b), since
// a+_a a+_b a_j a_i = (a+_b a_j)(a+_a a_i).  <I|H_s|J> = sign*[(ia|jb)-(ib|ja)].
__global__ void k_finalize_doubles(const uint64_t *__restrict__ s, int norb,
                                   const uint64_t *__restrict__ keys, int64_t nnz,
                                   const double *__restrict__ V, int32_t *__restrict__ tgt,
                                   uint32_t *__restrict__ orb, int8_t *__restrict__ sgn,
                                   double *__restrict__ val) {
    int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= nnz) return;
    uint64_t key = keys[e];
    int64_t row = (int64_t)(key >> 32), jj = (int64_t)(key & 0xffffffffu);
    uint64_t I = s[row], J = s[jj];
    uint64_t gone = I & ~J, add = J & ~I;
    int i = __ffsll((long long)gone) - 1;
    int j = __ffsll((long long)(gone & (gone - 1))) - 1;
    int a = __ffsll((long long)add) - 1;
    int b = __ffsll((long long)(add & (add - 1))) - 1;
    int s1 = single_sign(I, a, i);
    uint64_t K = I ^ (1ull << i) ^ (1ull << a);
    int s2 = single_sign(K, b, j);
    int sg = s1 * s2;
    double v = Vat(V, norb, i, a, j, b) - Vat(V, norb, i, b, j, a);
    tgt[e] = (int32_t)jj;
    orb[e] = (uint32_t)i | ((uint32_t)j << 8) | ((uint32_t)a << 16) | ((uint32_t)b << 24);
    sgn[e] = (int8_t)sg;
    val[e] = sg * v;
}

int launch_finalize_singles(sqd_ctx *ctx, const uint64_t *s, int norb, const uint64_t *keys,
                            int64_t nnz, const double *h, const double *V, int32_t *tgt,
                            uint16_t *pq, int8_t *sgn, double *val) {
    if (nnz == 0) return SQD_OK;
    k_finalize_singles<<<grid_1d(nnz, 256), 256, 0, ctx->stream>>>(s, norb, keys, nnz, h, V,
                                                                    tgt, pq, sgn, val);
    SQD_LAUNCHED(ctx);
    return SQD_OK;
}

int launch_finalize_doubles(sqd_ctx *ctx, const uint64_t *s, int norb, const uint64_t *keys,
                            int64_t nnz, const double *V, int32_t *tgt, uint32_t *orb,
                            int8_t *sgn, double *val) {
    if (nnz == 0) return SQD_OK;
    k_finalize_doubles<<<grid_1d(nnz, 256), 256, 0, ctx->stream>>>(s, norb, keys, nnz, V, tgt,
                                                                    orb, sgn, val);
    SQD_LAUNCHED(ctx);
    return SQD_OK;
}

// E_s(I) = sum_{k in I} h_kk + 1/2 sum_{k,l in I} [(kk|ll) - (kl|lk)]
__global__ void k_string_energy(const uint64_t *__restrict__ s, int64_t n, int norb,
                                const double *__restrict__ h, const double *__restrict__ V,
                                double *__restrict__ energy) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    uint64_t I = s[i];
    double e1 = 0.0, e2 = 0.0;
    uint64_t m = I;
    while (m) {
        int k = __ffsll((long long)m) - 1;
        m &= m - 1;
        e1 += __ldg(h + (int64_t)k * norb + k);
        uint64_t m2 = I;
        while (m2) {
            int l = __ffsll((long long)m2) - 1;
            m2 &= m2 - 1;
            e2 += Vat(V, norb, k, k, l, l) - Vat(V, norb, k, l, l, k);
        }
    }
    energy[i] = e1 + 0.5 * e2;
}

// W[pq][I] = sum_{l in I} (pq|ll): the coupling of an excitation E_pq of one
// spin with the occupations of a string of the other spin.
__global__ void k_string_W(const uint64_t *__restrict__ s, int64_t n, int norb,
                           const double *__restrict__ V, double *__restrict__ W) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int64_t pq = blockIdx.y;
    if (i >= n) return;
    uint64_t I = s[i];
    const double *row = V + pq * norb * norb;
    double w = 0.0;
    while (I) {
        int l = __ffsll((long long)I) - 1;
        I &= I - 1;
        w += __ldg(row + (int64_t)l * norb + l);
    }
    W[pq * n + i] = w;
}

int launch_string_terms(sqd_ctx *ctx, const uint64_t *s, int64_t n, int norb, const double *h,
                        const double *V, double *energy, double *W, double *u) {
    (void)u;
    if (n == 0) return SQD_OK;
    k_string_energy<<<grid_1d(n, 128), 128, 0, ctx->stream>>>(s, n, norb, h, V, energy);
    SQD_LAUNCHED(ctx);
    dim3 g(grid_1d(n, 256), (unsigned)(norb * norb));
    k_string_W<<<g, 256, 0, ctx->stream>>>(s, n, norb, V, W);
    SQD_LAUNCHED(ctx);
    return SQD_OK;
}

// H_II = E_core + E_a(I_a) + E_b(I_b) + sum_{k in I_a} W_b[kk][I_b]
__global__ void k_diagonal(int64_t na, int64_t nb, int norb, double ecore,
                           const uint64_t *__restrict__ sa, const double *__restrict__ Ea,
                           const double *__restrict__ Eb, const double *__restrict__ Wb,
                           double *__restrict__ diag) {
    int64_t ib = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (ib >= nb) return;
    for (int64_t ia = blockIdx.y; ia < na; ia += gridDim.y) {
        uint64_t I = sa[ia];
        double c = 0.0;
        while (I) {
            int k = __ffsll((long long)I) - 1;
            I &= I - 1;
            c += Wb[(int64_t)(k * norb + k) * nb + ib];
        }
        diag[ia * nb + ib] = ecore + Ea[ia] + Eb[ib] + c;
    }
}

int launch_diagonal(sqd_ctx *ctx, const spin_tables *a, const spin_tables *b, int norb,
                    double ecore, const uint64_t *sa, double *diag) {
    if (a->n == 0 || b->n == 0) return SQD_OK;
    dim3 g(grid_1d(b->n, 256), (unsigned)(a->n < 65535 ? a->n : 65535));
    k_diagonal<<<g, 256, 0, ctx->stream>>>(a->n, b->n, norb, ecore, sa, a->energy, b->energy,
                                           b->W, diag);
    SQD_LAUNCHED(ctx);
    return SQD_OK;
}
