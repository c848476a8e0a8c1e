// Spin-summed reduced density matrices of a state C on the alpha x beta
// subspace:  gamma_pq = sum_s <a+_ps a_qs>,
//            Gamma_pqrs = sum_{s,t} <a+_ps a+_rt a_st a_qs>.
// With C an eigenvector of P H P they are dE/dh and 2 dE/dV element-wise
// (Hellmann-Feynman).  The paper has no adjoint; the decomposition below
// mirrors the three kinds of excitation pairs of its sigma (Section IV).
//
// For a pair (bra J, ket I) of one spin the table entry of row I with target
// J carries <J|op|I>; with D(I,J) = sum over the other spin of C(I,.) C(J,.):
//  singles (p created, q annihilated, sign s):      gamma_pq += s D and, for
//    every spectator k of I and J, Gamma_pqkk += s D, Gamma_kkpq += s D,
//    Gamma_pkkq -= s D, Gamma_kqpk -= s D;
//  doubles (i<j annihilated, a<b created, sign s): Gamma_aibj += s D,
//    Gamma_biaj -= s D, Gamma_ajbi -= s D, Gamma_bjai += s D;
//  diagonal (w = |C(I,.)|^2): gamma_kk += w; Gamma_kkll += w and
//    Gamma_kllk -= w for k != l in I.
// The alpha-beta part Gamma_{pq,rs} += Gamma^ab_{pq,rs} + Gamma^ab_{rs,pq}
// with Gamma^ab_{pq,rs} = <E^a_pq E^b_rs> summed over pairs of "extended"
// singles (in-set singles plus the occupation terms E_kk of each string):
//   Gamma^ab_{p_a q_a, p_e q_e} += s_a s_e C(J_a, Ib_e) C(I_a, Jb_e).
#include <vector>

#include "sqd_internal.cuh"

// ------------------------------------------------------------ same spin --
// One warp per table entry (kind 1 or 2) or per row (kind 0: diagonal).
// X is the n x m matrix whose rows are indexed by this spin's strings.
__global__ void k_rdm_same_spin(int kind, int64_t n, int64_t m, int norb,
                                const double *__restrict__ X, const uint64_t *__restrict__ str,
                                const int64_t *__restrict__ off, const int32_t *__restrict__ tgt,
                                const uint16_t *__restrict__ pq1, const uint32_t *__restrict__ orb2,
                                const int8_t *__restrict__ sgn, int64_t nnz,
                                double *__restrict__ g1, double *__restrict__ g2) {
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    const int64_t nitems = (kind == 0) ? n : nnz;
    if (warp >= nitems) return;
    int64_t I, J;
    if (kind == 0) {
        I = J = warp;
    } else {
        // row of entry `warp`: upper bound in off
        int64_t lo = 0, hi = n;  // off[lo] <= e < off[hi]
        while (hi - lo > 1) {
            int64_t mid = (lo + hi) >> 1;
            if (off[mid] <= warp) lo = mid; else hi = mid;
        }
        I = lo;
        J = tgt[warp];
    }
    const double *xi = X + I * m, *xj = X + J * m;
    double d = 0.0;
    for (int64_t c = lane; c < m; c += 32) d = fma(xi[c], xj[c], d);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) d += __shfl_down_sync(0xffffffffu, d, o);
    if (lane != 0 || d == 0.0) return;
    const int64_t n2 = (int64_t)norb * norb;
    auto G = [&](int p, int q, int r, int s_) -> double * {
        return g2 + (((int64_t)p * norb + q) * norb + r) * norb + s_;
    };
    if (kind == 0) {
        uint64_t occ = str[I];
        for (uint64_t a = occ; a; a &= a - 1) {
            int k = __ffsll((long long)a) - 1;
            atomicAdd(g1 + (int64_t)k * norb + k, d);
            if (!g2) continue;
            for (uint64_t b = occ; b; b &= b - 1) {
                int l = __ffsll((long long)b) - 1;
                if (l == k) continue;
                atomicAdd(G(k, k, l, l), d);
                atomicAdd(G(k, l, l, k), -d);
            }
        }
        (void)n2;
    } else if (kind == 1) {
        int p = pq1[warp] / norb, q = pq1[warp] % norb;
        double v = sgn[warp] * d;
        atomicAdd(g1 + (int64_t)p * norb + q, v);
        if (!g2) return;
        uint64_t common = str[I] & str[J];
        for (uint64_t a = common; a; a &= a - 1) {
            int k = __ffsll((long long)a) - 1;
            atomicAdd(G(p, q, k, k), v);
            atomicAdd(G(k, k, p, q), v);
            atomicAdd(G(p, k, k, q), -v);
            atomicAdd(G(k, q, p, k), -v);
        }
    } else {
        if (!g2) return;
        uint32_t o = orb2[warp];
        int i = o & 0xff, j = (o >> 8) & 0xff, a = (o >> 16) & 0xff, b = (o >> 24) & 0xff;
        double v = sgn[warp] * d;
        atomicAdd(G(a, i, b, j), v);
        atomicAdd(G(b, i, a, j), -v);
        atomicAdd(G(a, j, b, i), -v);
        atomicAdd(G(b, j, a, i), v);
    }
}

static int rdm_same_spin(sqd_ctx *ctx, const spin_tables *s, int norb, const double *X,
                         int64_t m, double *g1, double *g2) {
    const int threads = 256, wpb = threads / 32;
    auto grid = [&](int64_t items) { return grid_1d(items, wpb); };
    if (s->n > 0) {
        k_rdm_same_spin<<<grid(s->n), threads, 0, ctx->stream>>>(
            0, s->n, m, norb, X, s->str, nullptr, nullptr, nullptr, nullptr, nullptr, 0, g1, g2);
        SQD_LAUNCHED(ctx);
    }
    if (s->nnz1 > 0) {
        k_rdm_same_spin<<<grid(s->nnz1), threads, 0, ctx->stream>>>(
            1, s->n, m, norb, X, s->str, s->off1, s->tgt1, s->pq1, nullptr, s->sgn1, s->nnz1, g1,
            g2);
        SQD_LAUNCHED(ctx);
    }
    if (s->nnz2 > 0 && g2) {
        k_rdm_same_spin<<<grid(s->nnz2), threads, 0, ctx->stream>>>(
            2, s->n, m, norb, X, s->str, s->off2, s->tgt2, nullptr, s->orb2, s->sgn2, s->nnz2,
            g1, g2);
        SQD_LAUNCHED(ctx);
    }
    return SQD_OK;
}

// ----------------------------------------------------------- alpha-beta --
// Extended alpha items (singles and occupations) sorted by their pq index;
// a block owns a range of beta rows Y (their extended entries in registers)
// and a contiguous range of items.  For every item it stages the slab
// C(I_a, Y) (ket rows) in shared memory, gathers C(J_a, Ib_e) and
// accumulates per entry until the item's pq changes, then flushes into
// Gamma[pq_a][pq_e] and Gamma[pq_e][pq_a] with atomics.

#define RDM_THREADS 256
#define RDM_EPT 16
#define RDM_ECAP (RDM_THREADS * RDM_EPT)
#define RDM_YW 256
#define RDM_NA 16

__global__ void k_items_keys(int64_t nnz1, int64_t n, int ne, int norb,
                             const uint16_t *__restrict__ pq1, const uint64_t *__restrict__ str,
                             uint64_t *__restrict__ keys) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int64_t total = nnz1 + n * (int64_t)ne;
    if (i >= total) return;
    uint64_t pq;
    if (i < nnz1) {
        pq = pq1[i];
    } else {
        int64_t d = i - nnz1, row = d / ne;
        int t = (int)(d % ne);
        uint64_t m = str[row];
        for (int k = 0; k < t; k++) m &= m - 1;
        int k = __ffsll((long long)m) - 1;
        pq = (uint64_t)(k * norb + k);
    }
    keys[i] = (pq << 44) | (uint64_t)i;
}

// items: ket row I (int32), bra row J (int32), pq | sign << 15 (uint32)
__global__ void k_items_fill(const uint64_t *__restrict__ keys, int64_t total, int64_t nnz1,
                             int ne, const int64_t *__restrict__ off1,
                             const int32_t *__restrict__ tgt1, const int8_t *__restrict__ sgn1,
                             int64_t n, int32_t *__restrict__ iket, int32_t *__restrict__ ibra,
                             uint32_t *__restrict__ ipq) {
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= total) return;
    uint64_t key = keys[t];
    int64_t i = (int64_t)(key & ((1ull << 44) - 1));
    uint32_t pq = (uint32_t)(key >> 44);
    if (i < nnz1) {
        int64_t lo = 0, hi = n;
        while (hi - lo > 1) {
            int64_t mid = (lo + hi) >> 1;
            if (off1[mid] <= i) lo = mid; else hi = mid;
        }
        iket[t] = (int32_t)lo;
        ibra[t] = tgt1[i];
        ipq[t] = pq | ((sgn1[i] < 0) ? 0x80000000u : 0u);
    } else {
        int64_t row = (i - nnz1) / ne;
        iket[t] = (int32_t)row;
        ibra[t] = (int32_t)row;
        ipq[t] = pq;
    }
}

__device__ __forceinline__ void rdm_cp_async8(void *smem, const void *gmem) {
    unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(s), "l"(gmem));
}

__global__ void __launch_bounds__(RDM_THREADS, 2)
    k_rdm_alpha_beta(int64_t nb, int norb, int ne_b, const uint64_t *__restrict__ b_str,
                     const int64_t *__restrict__ b_off, const int32_t *__restrict__ b_tgt,
                     const uint16_t *__restrict__ b_pq, const int8_t *__restrict__ b_sgn,
                     const int64_t *__restrict__ chunk_rows, const int64_t *__restrict__ item_grp,
                     const int32_t *__restrict__ iket, const int32_t *__restrict__ ibra,
                     const uint32_t *__restrict__ ipq, const double *__restrict__ C,
                     double *__restrict__ g2) {
    extern __shared__ double rdm_dyn[];
    double(*slab)[RDM_NA][RDM_YW] = reinterpret_cast<double(*)[RDM_NA][RDM_YW]>(rdm_dyn);
    __shared__ int32_t sh_bra[2][RDM_NA];
    __shared__ uint32_t sh_pq[2][RDM_NA];
    __shared__ int64_t sh_off[RDM_YW + 1];

    const int tid = threadIdx.x;
    const int64_t y0 = chunk_rows[blockIdx.x], y1 = chunk_rows[blockIdx.x + 1];
    const int width = (int)(y1 - y0);
    for (int t = tid; t <= width; t += RDM_THREADS) sh_off[t] = b_off[y0 + t];
    __syncthreads();
    const int64_t e0 = sh_off[0], nsing = sh_off[width] - e0;
    const int64_t nent = nsing + (int64_t)ne_b * width;
    const int64_t n2 = (int64_t)norb * norb;

    int32_t ib[RDM_EPT];
    uint32_t info[RDM_EPT];  // pq_e | jloc << 12 | sign << 31
    double acc[RDM_EPT];
#pragma unroll
    for (int k = 0; k < RDM_EPT; k++) {
        int64_t idx = tid + (int64_t)k * RDM_THREADS;
        ib[k] = -1;
        info[k] = 0;
        acc[k] = 0.0;
        if (idx < nsing) {
            int64_t e = e0 + idx;
            int lo = 0, hi = width;
            while (hi - lo > 1) {
                int mid = (lo + hi) >> 1;
                if (sh_off[mid] <= e) lo = mid; else hi = mid;
            }
            ib[k] = b_tgt[e];
            info[k] = (uint32_t)b_pq[e] | ((uint32_t)lo << 12) | ((b_sgn[e] < 0) ? 0x80000000u : 0u);
        } else if (idx < nent) {
            int64_t d = idx - nsing;
            int j = (int)(d / ne_b), t = (int)(d % ne_b);
            uint64_t m = b_str[y0 + j];
            for (int q = 0; q < t; q++) m &= m - 1;
            int l = __ffsll((long long)m) - 1;
            ib[k] = (int32_t)(y0 + j);
            info[k] = (uint32_t)(l * norb + l) | ((uint32_t)j << 12);
        }
    }

    const int64_t i0 = item_grp[blockIdx.y], i1 = item_grp[blockIdx.y + 1];
    auto stage = [&](int64_t b, int buf) {
        const int nbat = (int)min((int64_t)RDM_NA, i1 - b);
        if (tid < nbat) {
            sh_bra[buf][tid] = ibra[b + tid];
            sh_pq[buf][tid] = ipq[b + tid];
        }
        for (int idx = tid; idx < nbat * width; idx += RDM_THREADS) {
            int a = idx / width, j = idx - a * width;
            rdm_cp_async8(&slab[buf][a][j], C + (int64_t)iket[b + a] * nb + y0 + j);
        }
        asm volatile("cp.async.commit_group;\n" ::);
    };
    int64_t cur_pq = -1;
    auto flush = [&]() {
        if (cur_pq >= 0) {
#pragma unroll
            for (int k = 0; k < RDM_EPT; k++) {
                if (ib[k] >= 0 && acc[k] != 0.0) {
                    double v = (info[k] & 0x80000000u) ? -acc[k] : acc[k];
                    int64_t pe = info[k] & 0xfffu;
                    atomicAdd(g2 + cur_pq * n2 + pe, v);
                    atomicAdd(g2 + pe * n2 + cur_pq, v);
                }
                acc[k] = 0.0;
            }
        }
    };
    int buf = 0;
    if (i0 < i1) stage(i0, 0);
    for (int64_t b = i0; b < i1; b += RDM_NA) {
        if (b + RDM_NA < i1) stage(b + RDM_NA, buf ^ 1);
        else asm volatile("cp.async.commit_group;\n" ::);
        asm volatile("cp.async.wait_group 1;\n" ::);
        __syncthreads();
        const int nbat = (int)min((int64_t)RDM_NA, i1 - b);
        for (int a = 0; a < nbat; a++) {
            const uint32_t pqa = sh_pq[buf][a];
            const int64_t pq = pqa & 0xfffu;
            if (pq != cur_pq) {  // uniform across the block
                flush();
                cur_pq = pq;
            }
            const double *brow = C + (int64_t)sh_bra[buf][a] * nb;
            const uint32_t sa = pqa & 0x80000000u;
            const double *sl = slab[buf][a];
#pragma unroll
            for (int k = 0; k < RDM_EPT; k++) {
                if (ib[k] < 0) continue;
                double x = __ldg(brow + ib[k]);
                unsigned long long bits = (unsigned long long)__double_as_longlong(x) ^
                                          ((unsigned long long)sa << 32);
                acc[k] = fma(__longlong_as_double((long long)bits), sl[(info[k] >> 12) & 0x1ffu],
                             acc[k]);
            }
        }
        __syncthreads();
        buf ^= 1;
    }
    flush();
    asm volatile("cp.async.wait_group 0;\n" ::);
}

// build (once per table object) the sorted alpha items and both schedules
static int rdm_prepare(sqd_ctx *ctx, sqd_tables *t) {
    if (t->rdm_ready) return SQD_OK;
    const spin_tables *A = &t->a, *B = t->b;
    const int norb = t->norb;
    const int64_t total = A->nnz1 + A->n * (int64_t)A->ne;
    t->rdm_items = total;
    int64_t P = 1;
    while (P < total) P <<= 1;
    uint64_t *keys = nullptr;
    SQD_CUDA(ctx, cudaMallocAsync((void **)&keys, sizeof(uint64_t) * P, ctx->stream));
    SQD_TRY(launch_fill_u64(ctx, keys, P, ~0ull));
    if (total > 0) {
        k_items_keys<<<grid_1d(total, 256), 256, 0, ctx->stream>>>(A->nnz1, A->n, A->ne, norb,
                                                                   A->pq1, A->str, keys);
        SQD_LAUNCHED(ctx);
    }
    SQD_TRY(launch_bitonic_sort_u64(ctx, keys, P));
    SQD_CUDA(ctx, cudaMalloc((void **)&t->rdm_iket, sizeof(int32_t) * (total + 1)));
    SQD_CUDA(ctx, cudaMalloc((void **)&t->rdm_ibra, sizeof(int32_t) * (total + 1)));
    SQD_CUDA(ctx, cudaMalloc((void **)&t->rdm_ipq, sizeof(uint32_t) * (total + 1)));
    t->bytes += 12 * (total + 1);
    if (total > 0) {
        k_items_fill<<<grid_1d(total, 256), 256, 0, ctx->stream>>>(
            keys, total, A->nnz1, A->ne, A->off1, A->tgt1, A->sgn1, A->n, t->rdm_iket,
            t->rdm_ibra, t->rdm_ipq);
        SQD_LAUNCHED(ctx);
    }
    SQD_CUDA(ctx, cudaFreeAsync(keys, ctx->stream));
    // beta chunks: rows with (singles + ne * rows) <= RDM_ECAP, <= RDM_YW rows
    std::vector<int64_t> chunks{0};
    const std::vector<int64_t> &bo = B->h_off1;
    int64_t y = 0;
    while (y < B->n) {
        int64_t ye = y;
        while (ye < B->n && ye - y < RDM_YW &&
               (bo[ye + 1] - bo[y]) + (int64_t)B->ne * (ye + 1 - y) <= RDM_ECAP)
            ye++;
        if (ye == y) ye = y + 1;
        chunks.push_back(ye);
        y = ye;
    }
    int nch = (int)chunks.size() - 1;
    int64_t G = (16LL * ctx->sm_count + nch - 1) / nch;
    if (G > total) G = total;
    if (G < 1) G = 1;
    if (G > 65535) G = 65535;
    std::vector<int64_t> grp;
    for (int64_t g = 0; g <= G; g++) grp.push_back(total * g / G);
    t->rdm_nchunks = nch;
    t->rdm_ngroups = (int)G;
    SQD_CUDA(ctx, cudaMalloc((void **)&t->rdm_chunks, sizeof(int64_t) * chunks.size()));
    SQD_CUDA(ctx, cudaMalloc((void **)&t->rdm_groups, sizeof(int64_t) * grp.size()));
    SQD_CUDA(ctx, cudaMemcpy(t->rdm_chunks, chunks.data(), sizeof(int64_t) * chunks.size(),
                             cudaMemcpyHostToDevice));
    SQD_CUDA(ctx, cudaMemcpy(t->rdm_groups, grp.data(), sizeof(int64_t) * grp.size(),
                             cudaMemcpyHostToDevice));
    t->rdm_ready = true;
    return SQD_OK;
}

int launch_rdm(sqd_ctx *ctx, const sqd_tables *tc, const double *C, double *rdm1, double *rdm2) {
    sqd_tables *t = const_cast<sqd_tables *>(tc);
    const int norb = t->norb;
    const int64_t na = t->a.n, nb = t->b->n, n2 = (int64_t)norb * norb;
    if (!t->scratch_t) {
        SQD_CUDA(ctx, cudaMalloc((void **)&t->scratch_t, sizeof(double) * na * nb));
        t->bytes += 8 * na * nb;
    }
    SQD_TRY(rdm_prepare(ctx, t));
    prof_begin(ctx, PROF_RDM);
    SQD_CUDA(ctx, cudaMemsetAsync(rdm1, 0, sizeof(double) * n2, ctx->stream));
    if (rdm2) SQD_CUDA(ctx, cudaMemsetAsync(rdm2, 0, sizeof(double) * n2 * n2, ctx->stream));
    // alpha same-spin on C, beta same-spin on C^T
    SQD_TRY(rdm_same_spin(ctx, &t->a, norb, C, nb, rdm1, rdm2));
    SQD_TRY(launch_transpose(ctx, C, t->scratch_t, na, nb, false));
    SQD_TRY(rdm_same_spin(ctx, t->b, norb, t->scratch_t, na, rdm1, rdm2));
    if (rdm2 && t->rdm_items > 0) {
        const size_t shm = sizeof(double) * 2 * RDM_NA * RDM_YW;
        SQD_CUDA(ctx, cudaFuncSetAttribute(k_rdm_alpha_beta,
                                           cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm));
        dim3 g((unsigned)t->rdm_nchunks, (unsigned)t->rdm_ngroups);
        const spin_tables *B = t->b;
        k_rdm_alpha_beta<<<g, RDM_THREADS, shm, ctx->stream>>>(
            nb, norb, B->ne, B->str, B->off1, B->tgt1, B->pq1, B->sgn1, t->rdm_chunks,
            t->rdm_groups, t->rdm_iket, t->rdm_ibra, t->rdm_ipq, C, rdm2);
        SQD_LAUNCHED(ctx);
    }
    const double f = 2.0 * ((double)(t->a.nnz1 + t->a.nnz2 + na) * nb +
                            (double)(t->b->nnz1 + t->b->nnz2 + nb) * na +
                            (rdm2 ? (double)t->rdm_items * (double)(t->b->nnz1 + nb * t->b->ne)
                                  : 0.0));
    prof_end(ctx, f, 8.0 * na * nb * 3);
    return SQD_OK;
}

// ------------------------------------------------------ orbital gradient --
// g_pq = dE/dkappa_pq at kappa = 0 for orbitals rotated by U = exp(kappa):
// g_pq = 2 (F_pq - F_qp), F_pq = sum_r h_pr gamma_qr + sum_rst (pr|st) Gamma_qrst
// (generalized Fock matrix).  One thread per (p, q).
__global__ void k_gen_fock(int norb, const double *__restrict__ h, const double *__restrict__ V,
                           const double *__restrict__ g1, const double *__restrict__ g2,
                           double *__restrict__ F) {
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= norb * norb) return;
    int p = t / norb, q = t % norb;
    const int64_t n = norb, n2 = n * n, n3 = n2 * n;
    double f = 0.0;
    for (int r = 0; r < norb; r++) {
        f = fma(h[p * n + r], g1[q * n + r], f);
        const double *vr = V + (p * n + r) * n2;      // (pr|st) over st
        const double *gr = g2 + q * n3 + r * n2;      // Gamma_qrst over st
        for (int64_t st = 0; st < n2; st++) f = fma(vr[st], gr[st], f);
    }
    F[t] = f;
}

__global__ void k_antisym(int norb, const double *__restrict__ F, double *__restrict__ g) {
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= norb * norb) return;
    int p = t / norb, q = t % norb;
    g[t] = 2.0 * (F[p * norb + q] - F[q * norb + p]);
}

int launch_orbital_gradient(sqd_ctx *ctx, const sqd_tables *t, const double *g1,
                            const double *g2, double *grad) {
    const int n2 = t->norb * t->norb;
    double *F = nullptr;
    SQD_CUDA(ctx, cudaMallocAsync((void **)&F, sizeof(double) * n2, ctx->stream));
    k_gen_fock<<<grid_1d(n2, 128), 128, 0, ctx->stream>>>(t->norb, t->h, t->V, g1, g2, F);
    SQD_LAUNCHED(ctx);
    k_antisym<<<grid_1d(n2, 128), 128, 0, ctx->stream>>>(t->norb, F, grad);
    SQD_LAUNCHED(ctx);
    SQD_CUDA(ctx, cudaFreeAsync(F, ctx->stream));
    return SQD_OK;
}
