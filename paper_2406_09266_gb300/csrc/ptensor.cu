// Partially symmetric sparse tensors (Sec. 2.1, Def. "Partial Symmetry"): the
// modes are split into consecutive parts; the tensor is unchanged by any
// permutation that moves positions only inside their part.  The canonical
// triangle keeps the indices non-decreasing inside every part (Sec. 2.1, Def.
// "Canonical"), and one stored entry stands for every distinct arrangement
// obtained by permuting inside parts (the unique symmetry group S_T|E of
// Sec. 4.1, per part).
//
// Canonicalisation: sort inside parts, range check against each part's
// dimension, pack into a key (per-mode bit widths, first mode most
// significant), radix sort, duplicate policy, exact counts.  Device layout:
// the canonical entries as SoA int32 indices (mode q at idx + q * ld) and
// FP32 values, in lexicographic order.
//
// MTTKRP for the factor of part P (Sec. 5.2.6 generalised from one shared
// factor to one factor per part).  The sum over arrangements factorises over
// parts: a part Q != P contributes E(c_Q) * prod_{t in c_Q} F_Q[t, :] (E = the
// number of distinct arrangements of its multiset, every arrangement giving
// the same product), and the output part contributes, for each distinct value
// u of c_P, W_u * prod_{t in c_P minus one copy of u} F_P[t, :] with
// W_u = (s_P - 1)! m_u / prod_t m_t! arrangements that put u first.  So per
// canonical entry and per distinct u:
//   M[u, :] += v * W_u * prod_{c_P minus u} F_P * prod_{Q != P} E(c_Q) prod F_Q.
#include <algorithm>
#include <new>
#include <string.h>

#include "common.cuh"

struct sym_ptensor_s;

namespace symgpu {

namespace {

constexpr int PT = 256;

struct PartDesc {
    int order;
    int nparts;
    int part_of[5];  // mode -> part
    int first[5];    // part -> first mode
    int size[5];     // part -> number of modes
    int bits[5];     // mode -> key bits
    int shift[5];    // mode -> key bit offset (mode 0 most significant)
    int total_bits;
    int64_t dim[5];  // part -> index range
};

struct PCounters {
    unsigned long long range_bad;
    unsigned long long dup_seen;
    unsigned long long dup_mismatch;
    unsigned long long kept;
    unsigned long long expanded;
    double normsq;
};

// a / b for small integers when b divides a (arrangement counts): the
// correctly rounded reciprocal times a is within a few ulps of the integer
// quotient, so rounding to the nearest integer gives it exactly, without the
// integer-division routine a run-time divisor needs.
__device__ __forceinline__ float exact_quot(int a, int b) { return rintf((float)a * __frcp_rn((float)b)); }

__host__ __device__ __forceinline__ int fact_small(int k) {
    const int f[6] = {1, 1, 2, 6, 24, 120};
    return f[k];
}

template <int N>
__device__ __forceinline__ void sort_parts(int32_t* c, const PartDesc& D) {
#pragma unroll
    for (int a = 1; a < N; ++a)
#pragma unroll
        for (int b = a; b > 0; --b)
            if (D.part_of[b] == D.part_of[b - 1]) {  // compare-exchange only inside a part
                const int32_t x = c[b - 1], y = c[b];
                c[b - 1] = min(x, y);
                c[b] = max(x, y);
            }
}

// prod over parts of the distinct arrangements of each part's (sorted) multiset
template <int N>
__device__ __forceinline__ unsigned arrangements(const int32_t* c, const PartDesc& D) {
    unsigned e = 1;
    for (int p = 0; p < D.nparts; ++p) {
        const int f = D.first[p], s = D.size[p];
        int den = 1, run = 1;
        for (int j = 1; j < s; ++j) {
            if (c[f + j] == c[f + j - 1]) {
                ++run;
            } else {
                den *= fact_small(run);
                run = 1;
            }
        }
        den *= fact_small(run);
        e *= (unsigned)(fact_small(s) / den);
    }
    return e;
}

template <int N>
__device__ __forceinline__ unsigned __int128 ppack(const int32_t* c, const PartDesc& D) {
    unsigned __int128 k = 0;
#pragma unroll
    for (int q = 0; q < N; ++q) k |= (unsigned __int128)(uint32_t)c[q] << D.shift[q];
    return k;
}

template <int N>
__device__ __forceinline__ void punpack(unsigned __int128 k, const PartDesc& D, int32_t* c) {
#pragma unroll
    for (int q = 0; q < N; ++q) c[q] = (int32_t)(uint64_t)((k >> D.shift[q]) & ((((unsigned __int128)1) << D.bits[q]) - 1));
}

template <int N>
__global__ void k_ppack(PartDesc D, const int32_t* __restrict__ idx, int64_t ld, int64_t nnz,
                        uint64_t* __restrict__ klo, uint64_t* __restrict__ khi, uint32_t* __restrict__ pay,
                        PCounters* cnt) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    bool bad = false;
    if (e < nnz) {
        int32_t c[N];
#pragma unroll
        for (int q = 0; q < N; ++q) {
            c[q] = idx[(int64_t)q * ld + e];
            if (c[q] < 0 || (int64_t)c[q] >= D.dim[D.part_of[q]]) {
                bad = true;
                c[q] = 0;
            }
        }
        sort_parts<N>(c, D);
        const unsigned __int128 k = ppack<N>(c, D);
        klo[e] = (uint64_t)k;
        if (khi) khi[e] = (uint64_t)(k >> 64);
        pay[e] = (uint32_t)e;
    }
    const unsigned m = __ballot_sync(0xffffffffu, bad);
    if (m && (threadIdx.x & 31) == 0) atomicAdd(&cnt->range_bad, (unsigned long long)__popc(m));
}

// keep[p] = 1 for the first entry of each run of equal keys; counts.
template <int N>
__global__ void __launch_bounds__(PT) k_pmark(PartDesc D, const uint64_t* __restrict__ klo,
                                              const uint64_t* __restrict__ khi, const uint32_t* __restrict__ pay,
                                              const float* __restrict__ val, int64_t nnz, int policy,
                                              uint32_t* __restrict__ keep, PCounters* cnt) {
    __shared__ double s_norm[PT / 32];
    const int64_t p = (int64_t)blockIdx.x * PT + threadIdx.x;
    bool dup = false, mismatch = false, kept = false;
    unsigned ex = 0;
    double nrm = 0.0;
    if (p < nnz) {
        const uint64_t lo = klo[p], hi = khi ? khi[p] : 0ull;
        if (p > 0) {
            dup = klo[p - 1] == lo && (khi ? khi[p - 1] : 0ull) == hi;
            if (dup && policy == SYM_DUP_KEEP_EQUAL)
                mismatch = __float_as_uint(val[pay[p]]) != __float_as_uint(val[pay[p - 1]]);
        }
        kept = !dup;
        keep[p] = kept ? 1u : 0u;
        if (kept) {
            int32_t c[N];
            punpack<N>(((unsigned __int128)hi << 64) | lo, D, c);
            ex = arrangements<N>(c, D);
            const double v = (double)val[pay[p]];
            nrm = (double)ex * v * v;
        }
    }
    const unsigned full = 0xffffffffu;
    const unsigned long long ex_sum = (unsigned long long)__reduce_add_sync(full, ex);
    const int n_keep = __popc(__ballot_sync(full, kept));
    const int n_dup = __popc(__ballot_sync(full, dup));
    const int n_mis = __popc(__ballot_sync(full, mismatch));
    if ((threadIdx.x & 31) == 0) {
        if (ex_sum) atomicAdd(&cnt->expanded, ex_sum);
        if (n_keep) atomicAdd(&cnt->kept, (unsigned long long)n_keep);
        if (n_dup) atomicAdd(&cnt->dup_seen, (unsigned long long)n_dup);
        if (n_mis) atomicAdd(&cnt->dup_mismatch, (unsigned long long)n_mis);
    }
    nrm = warp_sum(nrm);
    if ((threadIdx.x & 31) == 0) s_norm[threadIdx.x >> 5] = nrm;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < PT / 32; ++w) t += s_norm[w];  // fixed order inside the block
        atomicAdd(&cnt->normsq, t);
    }
}

template <int N>
__global__ void k_pcompact(PartDesc D, const uint64_t* __restrict__ klo, const uint64_t* __restrict__ khi,
                           const uint32_t* __restrict__ pay, const float* __restrict__ val, int64_t nnz,
                           const uint32_t* __restrict__ keep, const uint32_t* __restrict__ pos,
                           int32_t* __restrict__ out_idx, int64_t ld, float* __restrict__ out_val) {
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= nnz || !keep[p]) return;
    int32_t c[N];
    punpack<N>(((unsigned __int128)(khi ? khi[p] : 0ull) << 64) | klo[p], D, c);
    const int64_t dst = pos[p];
#pragma unroll
    for (int q = 0; q < N; ++q) out_idx[(int64_t)q * ld + dst] = c[q];
    out_val[dst] = val[pay[p]];
}

__global__ void k_pexport(const int32_t* __restrict__ idx, int64_t ld, const float* __restrict__ val, int order,
                          int64_t nnz, int32_t* __restrict__ out, int64_t ld_out, float* __restrict__ out_val) {
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= nnz) return;
    for (int q = 0; q < order; ++q) out[(int64_t)q * ld_out + p] = idx[(int64_t)q * ld + p];
    out_val[p] = val[p];
}

// Per-mode view of the partition and the factors for one MTTKRP call
// (resolved on the host so the kernel indexes it only at compile time).
struct ModeArgs {
    const void* F[5];  // factor of the mode's part
    int64_t ld[5];
    int pos[5];        // position of the mode inside its part
    int inP[5];        // 1 when the mode belongs to the output part
    int s;             // size of the output part
};

// One entry per group of GP lanes (GP = rank / 4 rounded up to a power of
// two); lane j of the group owns columns [4j, 4j + 4).  Every loop runs over
// modes at compile time with the partition tested at run time, so the tuple
// and the factor rows stay in registers.
template <int N, bool BF16>
__global__ void __launch_bounds__(256) k_pmttkrp(ModeArgs A, const int32_t* __restrict__ idx, int64_t ld,
                                                 const float* __restrict__ val, int64_t nnz, int R, int GP,
                                                 float* __restrict__ M, int64_t ldm) {
    const int lane = threadIdx.x & 31;
    const int col = 4 * (lane & (GP - 1));
    const int per_warp = 32 / GP;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t e0 = warp * per_warp; e0 < nnz; e0 += nwarps * per_warp) {
        const int64_t e = e0 + lane / GP;
        if (e >= nnz || col >= R) continue;
        int32_t c[N];
        float4 row[N];
#pragma unroll
        for (int q = 0; q < N; ++q) {
            c[q] = idx[(int64_t)q * ld + e];
            row[q] = load_row4<BF16>(A.F[q], c[q], A.ld[q], col);
        }
        // run position of each mode inside its part: the product over a part is prod_t m_t!
        bool same[N];
        int runpos[N];
#pragma unroll
        for (int q = 0; q < N; ++q) {
            same[q] = q > 0 && A.pos[q] > 0 && c[q] == c[q > 0 ? q - 1 : 0];
            runpos[q] = same[q] ? runpos[q > 0 ? q - 1 : 0] + 1 : 1;
        }
        // parts other than P: E(c_Q) = s_Q! / prod m!, times the product of their rows
        float4 prod = make_float4(1.f, 1.f, 1.f, 1.f);
        int num = 1, den = 1, denP = 1;
#pragma unroll
        for (int q = 0; q < N; ++q) {
            if (A.inP[q]) {
                denP *= runpos[q];
            } else {
                prod = f4_mul(prod, row[q]);
                num *= A.pos[q] + 1;
                den *= runpos[q];
            }
        }
        const float base = val[e] * exact_quot(num, den);
        // one update per distinct value u of part P, at the first mode of its run
#pragma unroll
        for (int q = 0; q < N; ++q) {
            if (!A.inP[q] || same[q]) continue;
            int m = 0;
            float4 t = prod;
#pragma unroll
            for (int k = 0; k < N; ++k) {
                if (!A.inP[k]) continue;
                if (c[k] == c[q]) ++m;
                if (k != q) t = f4_mul(t, row[k]);
            }
            const float W = exact_quot(fact_small(A.s - 1) * m, denP);
            red_add_f4(M + (int64_t)c[q] * ldm + col, f4_scale(t, base * W));
        }
    }
}

// Arrangement count of each canonical entry (for the expansion offsets).
template <int N>
__global__ void k_pcount(PartDesc D, const int32_t* __restrict__ idx, int64_t ld, int64_t nnz,
                         int64_t* __restrict__ cnt) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= nnz) return;
    int32_t c[N];
#pragma unroll
    for (int q = 0; q < N; ++q) c[q] = idx[(int64_t)q * ld + e];
    cnt[e] = (int64_t)arrangements<N>(c, D);
}

// Writes every inside-part arrangement of entry e at off[e] ...: each part
// steps through the distinct permutations of its multiset (next permutation
// in lexicographic order), the last part fastest.
template <int N>
__global__ void k_pexpand(PartDesc D, const int32_t* __restrict__ idx, int64_t ld, const float* __restrict__ val,
                          int64_t nnz, const int64_t* __restrict__ off, int32_t* __restrict__ out, int64_t ld_out,
                          float* __restrict__ out_val) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= nnz) return;
    int32_t c[N];
    for (int q = 0; q < N; ++q) c[q] = idx[(int64_t)q * ld + e];
    const float v = val[e];
    int64_t w = off[e];
    for (;;) {
        for (int q = 0; q < N; ++q) out[(int64_t)q * ld_out + w] = c[q];
        out_val[w] = v;
        ++w;
        bool advanced = false;
        for (int p = D.nparts - 1; p >= 0 && !advanced; --p) {
            const int f = D.first[p], s = D.size[p];
            int i = s - 2;
            while (i >= 0 && c[f + i] >= c[f + i + 1]) --i;
            if (i >= 0) {
                int j = s - 1;
                while (c[f + j] <= c[f + i]) --j;
                int32_t t = c[f + i];
                c[f + i] = c[f + j];
                c[f + j] = t;
                for (int a = i + 1, b = s - 1; a < b; ++a, --b) {
                    t = c[f + a];
                    c[f + a] = c[f + b];
                    c[f + b] = t;
                }
                advanced = true;
            } else {
                for (int a = 0, b = s - 1; a < b; ++a, --b) {  // back to ascending, carry to the part before
                    const int32_t t = c[f + a];
                    c[f + a] = c[f + b];
                    c[f + b] = t;
                }
            }
        }
        if (!advanced) break;
    }
}

// The same update when the output part starts at mode 0: the canonical entries
// are sorted by c_0, so each warp takes a contiguous chunk of entries and each
// lane group a strided, still sorted, subsequence of it; the update of row
// c_0 is summed in registers along each run of equal c_0 and reduced once per
// run (F_P[c_0] loaded once per run too).  The other distinct values of the
// output part still take one reduction per entry.
template <int N, bool BF16>
__global__ void __launch_bounds__(256) k_pmttkrp_root(ModeArgs A, const int32_t* __restrict__ idx, int64_t ld,
                                                      const float* __restrict__ val, int64_t nnz, int R, int GP,
                                                      float* __restrict__ M, int64_t ldm, int64_t chunk) {
    const int lane = threadIdx.x & 31;
    const int col = 4 * (lane & (GP - 1));
    const int per_warp = 32 / GP;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t start = warp * chunk, end = min(start + chunk, nnz);
    if (start >= end || col >= R) return;
    int32_t cur = -1;
    float4 acc = f4_zero(), row0 = f4_zero();
    for (int64_t e = start + lane / GP; e < end; e += per_warp) {
        int32_t c[N];
        float4 row[N];
#pragma unroll
        for (int q = 0; q < N; ++q) c[q] = idx[(int64_t)q * ld + e];
        if (c[0] != cur) {
            if (cur >= 0) red_add_f4(M + (int64_t)cur * ldm + col, acc);
            cur = c[0];
            acc = f4_zero();
            row0 = load_row4<BF16>(A.F[0], c[0], A.ld[0], col);
        }
        row[0] = row0;
#pragma unroll
        for (int q = 1; q < N; ++q) row[q] = load_row4<BF16>(A.F[q], c[q], A.ld[q], col);
        bool same[N];
        int runpos[N];
#pragma unroll
        for (int q = 0; q < N; ++q) {
            same[q] = q > 0 && A.pos[q] > 0 && c[q] == c[q > 0 ? q - 1 : 0];
            runpos[q] = same[q] ? runpos[q > 0 ? q - 1 : 0] + 1 : 1;
        }
        float4 prod = make_float4(1.f, 1.f, 1.f, 1.f);
        int num = 1, den = 1, denP = 1;
#pragma unroll
        for (int q = 0; q < N; ++q) {
            if (A.inP[q]) {
                denP *= runpos[q];
            } else {
                prod = f4_mul(prod, row[q]);
                num *= A.pos[q] + 1;
                den *= runpos[q];
            }
        }
        const float base = val[e] * exact_quot(num, den);
#pragma unroll
        for (int q = 0; q < N; ++q) {
            if (!A.inP[q] || same[q]) continue;
            int m = 0;
            float4 t = prod;
#pragma unroll
            for (int k = 0; k < N; ++k) {
                if (!A.inP[k]) continue;
                if (c[k] == c[q]) ++m;
                if (k != q) t = f4_mul(t, row[k]);
            }
            const float W = exact_quot(fact_small(A.s - 1) * m, denP);
            t = f4_scale(t, base * W);
            if (q == 0) {
                acc = make_float4(acc.x + t.x, acc.y + t.y, acc.z + t.z, acc.w + t.w);  // row c_0: summed along the run
            } else {
                red_add_f4(M + (int64_t)c[q] * ldm + col, t);
            }
        }
    }
    if (cur >= 0) red_add_f4(M + (int64_t)cur * ldm + col, acc);
}

// Mode-1 TTM of a partially symmetric order-3 tensor (the TTM of Sec. 4.2 with
// the symmetry of Def. "Partial Symmetry"): C[j, l, :] = sum_k A[k, j, l] B[k, :]
// over the full tensor.  One lane group per canonical entry (sorted inside
// parts); each distinct inside-part arrangement (a1, a2, a3) of it adds
// v B[a1, :] to output position (a2, a3).  Packed layout (modes 2 and 3 in one
// part, so C is symmetric in (j, l)): only arrangements with a2 <= a3 are
// applied, at the canonical position a2 d - a2 (a2 - 1) / 2 + (a3 - a2); the
// mirrored arrangement holds the same value and is not stored.
template <bool BF16, bool PACKED>
__global__ void __launch_bounds__(256) k_pttm3(PartDesc D, const int32_t* __restrict__ idx, int64_t ld,
                                               const float* __restrict__ val, int64_t nnz, const void* __restrict__ B,
                                               int64_t ldb, int R, int GP, float* __restrict__ C, int64_t d3) {
    // the six permutations of three positions
    const int perm[6][3] = {{0, 1, 2}, {0, 2, 1}, {1, 0, 2}, {1, 2, 0}, {2, 0, 1}, {2, 1, 0}};
    const int lane = threadIdx.x & 31;
    const int col = 4 * (lane & (GP - 1));
    const int per_warp = 32 / GP;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t e0 = warp * per_warp; e0 < nnz; e0 += nwarps * per_warp) {
        const int64_t e = e0 + lane / GP;
        if (e >= nnz || col >= R) continue;
        int32_t c[3];
#pragma unroll
        for (int q = 0; q < 3; ++q) c[q] = idx[(int64_t)q * ld + e];
        const float v = val[e];
        int32_t seen[6][3];
        int ns = 0;
#pragma unroll
        for (int k = 0; k < 6; ++k) {
            // only permutations inside parts
            bool inside = true;
#pragma unroll
            for (int q = 0; q < 3; ++q) inside = inside && D.part_of[perm[k][q]] == D.part_of[q];
            if (!inside) continue;
            const int32_t a1 = c[perm[k][0]], a2 = c[perm[k][1]], a3 = c[perm[k][2]];
            bool dup = false;  // the same arrangement from an earlier permutation (repeated indices)
            for (int t = 0; t < ns; ++t) dup = dup || (seen[t][0] == a1 && seen[t][1] == a2 && seen[t][2] == a3);
            if (dup) continue;
            seen[ns][0] = a1;
            seen[ns][1] = a2;
            seen[ns][2] = a3;
            ++ns;
            if (PACKED && a2 > a3) continue;
            const int64_t pos = PACKED ? (int64_t)a2 * d3 - (int64_t)a2 * (a2 - 1) / 2 + (a3 - a2)
                                       : (int64_t)a2 * d3 + a3;
            red_add_f4(C + pos * R + col, f4_scale(load_row4<BF16>(B, a1, ldb, col), v));
        }
    }
}

__global__ void k_zero_rows(float* __restrict__ M, int64_t rows, int R, int64_t ldm) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t tot = rows * (int64_t)R;
    if (i < tot) M[(i / R) * ldm + i % R] = 0.f;
}

int bits_for_dim(int64_t n) {
    int b = 0;
    while ((1ll << b) < n) ++b;
    return b < 1 ? 1 : b;
}

sym_status make_desc(int order, int nparts, const int32_t* part, const int64_t* dim, PartDesc* D) {
    if (order < 1 || order > 5 || nparts < 1 || nparts > order || !part || !dim) return SYM_E_INVALID;
    memset(D, 0, sizeof(*D));
    D->order = order;
    D->nparts = nparts;
    int q = 0;
    for (int p = 0; p < nparts; ++p) {
        if (part[p] < 1 || dim[p] < 1 || dim[p] > 0x7fffffffLL) return SYM_E_INVALID;
        D->first[p] = q;
        D->size[p] = part[p];
        D->dim[p] = dim[p];
        for (int t = 0; t < part[p]; ++t) {
            if (q >= order) return SYM_E_INVALID;
            D->part_of[q] = p;
            D->bits[q] = bits_for_dim(dim[p]);
            ++q;
        }
    }
    if (q != order) return SYM_E_INVALID;
    int sh = 0;
    for (int m = order - 1; m >= 0; --m) {
        D->shift[m] = sh;
        sh += D->bits[m];
    }
    D->total_bits = sh;
    if (sh > 128) return SYM_E_UNSUPPORTED;
    return SYM_OK;
}

template <typename C>
void layout_pws(C& c, int64_t nnz, int kw, uint64_t** lo0, uint64_t** hi0, uint32_t** p0, uint64_t** lo1,
                uint64_t** hi1, uint32_t** p1, uint32_t** keep, uint32_t** pos, PCounters** cnt, void** radix,
                void** scan) {
    const size_t m = nnz > 0 ? (size_t)nnz : 1;
    *lo0 = c.template take<uint64_t>(m);
    *hi0 = kw == 2 ? c.template take<uint64_t>(m) : nullptr;
    *p0 = c.template take<uint32_t>(m);
    *lo1 = c.template take<uint64_t>(m);
    *hi1 = kw == 2 ? c.template take<uint64_t>(m) : nullptr;
    *p1 = c.template take<uint32_t>(m);
    *keep = c.template take<uint32_t>(m);
    *pos = c.template take<uint32_t>(m);
    *cnt = c.template take<PCounters>(1);
    *radix = c.template take<char>(radix_ws_bytes((int64_t)m, kw));
    *scan = c.template take<char>(scan_ws_bytes((int64_t)m));
}

template <typename C>
void layout_parena(C& c, int64_t nnz, int order, int32_t** idx, float** val) {
    const size_t m = nnz > 0 ? (size_t)nnz : 1;
    *idx = c.template take<int32_t>(m * (size_t)order);
    *val = c.template take<float>(m);
}

struct SizeOnly {
    Sizer s;
    template <typename T>
    T* take(size_t n) {
        s.take<T>(n);
        return nullptr;
    }
};

template <int N>
sym_status run_pcreate(const PartDesc& D, int kw, const int32_t* idx, int64_t ld, const float* val, int64_t nnz,
                       int policy, uint64_t* lo0, uint64_t* hi0, uint32_t* p0, uint64_t* lo1, uint64_t* hi1,
                       uint32_t* p1, uint32_t* keep, uint32_t* pos, PCounters* cnt, void* radix, void* scan,
                       int32_t* out_idx, int64_t out_ld, float* out_val, cudaStream_t s) {
    const unsigned g = (unsigned)((nnz + PT - 1) / PT);
    k_ppack<N><<<g, PT, 0, s>>>(D, idx, ld, nnz, lo0, kw == 2 ? hi0 : nullptr, p0, cnt);
    SYM_CHECK_LAUNCH();
    uint64_t *slo, *shi;
    uint32_t* sp;
    sym_status st = radix_sort_pairs(kw, lo0, hi0, p0, lo1, hi1, p1, nnz, D.total_bits, radix, s, &slo, &shi, &sp);
    if (st != SYM_OK) return st;
    k_pmark<N><<<g, PT, 0, s>>>(D, slo, kw == 2 ? shi : nullptr, sp, val, nnz, policy, keep, cnt);
    SYM_CHECK_LAUNCH();
    st = exclusive_scan_u32(keep, pos, nnz, scan, s);
    if (st != SYM_OK) return st;
    k_pcompact<N><<<g, PT, 0, s>>>(D, slo, kw == 2 ? shi : nullptr, sp, val, nnz, keep, pos, out_idx, out_ld,
                                   out_val);
    SYM_CHECK_LAUNCH();
    return SYM_OK;
}

}  // namespace

}  // namespace symgpu

struct sym_ptensor_s {
    symgpu::PartDesc D;
    int64_t cap;  // column stride of idx (the input entry count)
    int32_t* idx;
    float* val;
    sym_ptensor_info_t info;
    int device;
};

using namespace symgpu;

extern "C" sym_status sym_ptensor_create_bytes(int order, int nparts, const int32_t* part, const int64_t* dim,
                                               int64_t nnz, size_t* arena_bytes, size_t* ws_bytes) {
    PartDesc D;
    sym_status st = make_desc(order, nparts, part, dim, &D);
    if (st != SYM_OK) return st;
    if (nnz < 0 || nnz > 0xffffffffLL) return SYM_E_INVALID;
    const int kw = D.total_bits > 64 ? 2 : 1;
    SizeOnly a, w;
    int32_t* i;
    float* v;
    layout_parena(a, nnz, order, &i, &v);
    uint64_t *l0, *h0, *l1, *h1;
    uint32_t *p0, *p1, *kp, *ps;
    PCounters* c;
    void *r, *sc;
    layout_pws(w, nnz, kw, &l0, &h0, &p0, &l1, &h1, &p1, &kp, &ps, &c, &r, &sc);
    if (arena_bytes) *arena_bytes = a.s.used;
    if (ws_bytes) *ws_bytes = w.s.used;
    return SYM_OK;
}

extern "C" sym_status sym_ptensor_create(int order, int nparts, const int32_t* part, const int64_t* dim, int64_t nnz,
                                         const int32_t* idx, int64_t ld_idx, const float* val, sym_dup_policy dup,
                                         void* arena, size_t arena_bytes, void* ws, size_t ws_bytes,
                                         sym_stream_t stream, sym_ptensor* out) {
    if (!out) return SYM_E_INVALID;
    *out = nullptr;
    size_t need_a = 0, need_w = 0;
    sym_status st = sym_ptensor_create_bytes(order, nparts, part, dim, nnz, &need_a, &need_w);
    if (st != SYM_OK) return st;
    if (nnz > 0 && (!idx || !val || ld_idx < nnz)) return SYM_E_INVALID;
    if (dup != SYM_DUP_ERROR && dup != SYM_DUP_KEEP_EQUAL) return SYM_E_INVALID;
    if (!arena || !ws || !aligned(arena, 256) || !aligned(ws, 256)) return SYM_E_INVALID;
    if (arena_bytes < need_a || ws_bytes < need_w) return SYM_E_NOMEM;
    PartDesc D;
    make_desc(order, nparts, part, dim, &D);
    const int kw = D.total_bits > 64 ? 2 : 1;
    cudaStream_t s = as_stream(stream);
    Carver A(arena, arena_bytes), Wc(ws, ws_bytes);
    int32_t* oidx;
    float* oval;
    layout_parena(A, nnz, order, &oidx, &oval);
    uint64_t *l0, *h0, *l1, *h1;
    uint32_t *p0, *p1, *kp, *ps;
    PCounters* cnt;
    void *radix, *scan;
    layout_pws(Wc, nnz, kw, &l0, &h0, &p0, &l1, &h1, &p1, &kp, &ps, &cnt, &radix, &scan);
    const int64_t cap = nnz > 0 ? nnz : 1;
    SYM_CUDA(cudaMemsetAsync(cnt, 0, sizeof(PCounters), s));
    if (nnz > 0) {
        switch (order) {
            case 1: st = run_pcreate<1>(D, kw, idx, ld_idx, val, nnz, dup, l0, h0, p0, l1, h1, p1, kp, ps, cnt, radix, scan, oidx, cap, oval, s); break;
            case 2: st = run_pcreate<2>(D, kw, idx, ld_idx, val, nnz, dup, l0, h0, p0, l1, h1, p1, kp, ps, cnt, radix, scan, oidx, cap, oval, s); break;
            case 3: st = run_pcreate<3>(D, kw, idx, ld_idx, val, nnz, dup, l0, h0, p0, l1, h1, p1, kp, ps, cnt, radix, scan, oidx, cap, oval, s); break;
            case 4: st = run_pcreate<4>(D, kw, idx, ld_idx, val, nnz, dup, l0, h0, p0, l1, h1, p1, kp, ps, cnt, radix, scan, oidx, cap, oval, s); break;
            default: st = run_pcreate<5>(D, kw, idx, ld_idx, val, nnz, dup, l0, h0, p0, l1, h1, p1, kp, ps, cnt, radix, scan, oidx, cap, oval, s); break;
        }
        if (st != SYM_OK) return st;
    }
    PCounters h;
    SYM_CUDA(cudaMemcpyAsync(&h, cnt, sizeof(h), cudaMemcpyDeviceToHost, s));
    SYM_CUDA(cudaStreamSynchronize(s));
    if (h.range_bad) return SYM_E_RANGE;
    if (dup == SYM_DUP_ERROR && h.dup_seen) return SYM_E_DUPLICATE;
    if (dup == SYM_DUP_KEEP_EQUAL && h.dup_mismatch) return SYM_E_DUPLICATE;
    sym_ptensor_s* t = new (std::nothrow) sym_ptensor_s();
    if (!t) return SYM_E_NOMEM;
    t->D = D;
    t->cap = cap;
    t->idx = oidx;
    t->val = oval;
    t->device = current_device();
    sym_ptensor_info_t& I = t->info;
    memset(&I, 0, sizeof(I));
    I.order = order;
    I.nparts = nparts;
    I.key_bits = D.total_bits;
    I.nnz = (int64_t)h.kept;
    I.expanded_nnz = (int64_t)h.expanded;
    I.duplicates_dropped = (int64_t)h.dup_seen;
    I.normsq = h.normsq;
    *out = t;
    return SYM_OK;
}

extern "C" sym_status sym_ptensor_info(sym_ptensor X, sym_ptensor_info_t* out) {
    if (!X || !out) return SYM_E_INVALID;
    *out = X->info;
    return SYM_OK;
}

extern "C" sym_status sym_ptensor_export(sym_ptensor X, int32_t* cidx, int64_t ld_out, float* cval,
                                         sym_stream_t stream) {
    if (!X) return SYM_E_INVALID;
    const int64_t nnz = X->info.nnz;
    if (nnz == 0) return SYM_OK;
    if (!cidx || !cval || ld_out < nnz) return SYM_E_INVALID;
    const unsigned g = (unsigned)((nnz + 255) / 256);
    k_pexport<<<g, 256, 0, as_stream(stream)>>>(X->idx, X->cap, X->val, X->D.order, nnz, cidx, ld_out, cval);
    SYM_CHECK_LAUNCH();
    return SYM_OK;
}

extern "C" sym_status sym_pmttkrp(sym_ptensor X, const void* const* factors, const int64_t* ldf, sym_dtype dtype,
                                  int rank, int out_part, float* M, int64_t ldm, sym_stream_t stream) {
    if (!X || !factors || !ldf || !M) return SYM_E_INVALID;
    const PartDesc& D = X->D;
    if (out_part < 0 || out_part >= D.nparts) return SYM_E_INVALID;
    if (rank < 4 || rank > 128 || rank % 4) return SYM_E_INVALID;
    if (dtype != SYM_F32 && dtype != SYM_BF16) return SYM_E_INVALID;
    if (ldm < rank || !aligned(M, 16) || ldm % 4) return SYM_E_INVALID;
    ModeArgs A;
    memset(&A, 0, sizeof(A));
    const size_t esz = dtype == SYM_BF16 ? 2 : 4;
    for (int p = 0; p < D.nparts; ++p)
        if (!factors[p] || ldf[p] < rank || ldf[p] % 4 || !aligned(factors[p], 4 * esz)) return SYM_E_INVALID;
    for (int q = 0; q < D.order; ++q) {
        const int p = D.part_of[q];
        A.F[q] = factors[p];
        A.ld[q] = ldf[p];
        A.pos[q] = q - D.first[p];
        A.inP[q] = p == out_part ? 1 : 0;
    }
    A.s = D.size[out_part];
    cudaStream_t s = as_stream(stream);
    const int64_t rows = D.dim[out_part];
    {
        const int64_t tot = rows * rank;
        k_zero_rows<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(M, rows, rank, ldm);
        SYM_CHECK_LAUNCH();
    }
    const int64_t nnz = X->info.nnz;
    if (nnz == 0) return SYM_OK;
    int GP = 1;
    while (GP < rank / 4) GP <<= 1;
    const int64_t warps = (nnz + (32 / GP) - 1) / (32 / GP);
    const unsigned grid = (unsigned)std::min<int64_t>((warps + 7) / 8, (int64_t)sm_count() * 16);
    SYM_PROF("pmttkrp", s);
    const bool root = out_part == 0;  // output part starts at mode 0: entries sorted by its first index
    const int64_t chunk = 256;
    const unsigned rgrid = (unsigned)(((nnz + chunk - 1) / chunk + 7) / 8);
#define SYM_PM_CASE(NN)                                                                                         \
    if (root && dtype == SYM_BF16)                                                                              \
        k_pmttkrp_root<NN, true><<<rgrid, 256, 0, s>>>(A, X->idx, X->cap, X->val, nnz, rank, GP, M, ldm, chunk); \
    else if (root)                                                                                              \
        k_pmttkrp_root<NN, false><<<rgrid, 256, 0, s>>>(A, X->idx, X->cap, X->val, nnz, rank, GP, M, ldm,       \
                                                        chunk);                                                 \
    else if (dtype == SYM_BF16)                                                                                 \
        k_pmttkrp<NN, true><<<grid, 256, 0, s>>>(A, X->idx, X->cap, X->val, nnz, rank, GP, M, ldm);       \
    else                                                                                                        \
        k_pmttkrp<NN, false><<<grid, 256, 0, s>>>(A, X->idx, X->cap, X->val, nnz, rank, GP, M, ldm);
    switch (D.order) {
        case 1: SYM_PM_CASE(1) break;
        case 2: SYM_PM_CASE(2) break;
        case 3: SYM_PM_CASE(3) break;
        case 4: SYM_PM_CASE(4) break;
        default: SYM_PM_CASE(5) break;
    }
#undef SYM_PM_CASE
    SYM_CHECK_LAUNCH();
    return SYM_OK;
}

extern "C" int64_t sym_pttm_output_elems(sym_ptensor X, int rank, int layout) {
    if (!X || X->D.order != 3 || rank < 4 || rank > 128 || rank % 4) return -1;
    const PartDesc& D = X->D;
    const int64_t d2 = D.dim[D.part_of[1]], d3 = D.dim[D.part_of[2]];
    if (layout == SYM_TTM_FULL) return d2 * d3 * rank;
    if (layout == SYM_TTM_PACKED && D.part_of[1] == D.part_of[2]) return d2 * (d2 + 1) / 2 * rank;
    return -1;
}

extern "C" sym_status sym_pttm(sym_ptensor X, const void* B, sym_dtype bdt, int rank, int64_t ldb, float* C,
                               int layout, sym_stream_t stream) {
    if (!X || !B || !C) return SYM_E_INVALID;
    if (X->D.order != 3) return SYM_E_UNSUPPORTED;
    const int64_t elems = sym_pttm_output_elems(X, rank, layout);
    if (elems < 0) return SYM_E_INVALID;
    if (bdt != SYM_F32 && bdt != SYM_BF16) return SYM_E_INVALID;
    if (ldb < rank || ldb % 4 || !aligned(B, bdt == SYM_BF16 ? 8 : 16) || !aligned(C, 16)) return SYM_E_INVALID;
    const PartDesc& D = X->D;
    cudaStream_t s = as_stream(stream);
    SYM_CUDA(cudaMemsetAsync(C, 0, sizeof(float) * (size_t)elems, s));
    const int64_t nnz = X->info.nnz;
    if (nnz == 0) return SYM_OK;
    int GP = 1;
    while (GP < rank / 4) GP <<= 1;
    const int64_t warps = (nnz + (32 / GP) - 1) / (32 / GP);
    const unsigned grid = (unsigned)std::min<int64_t>((warps + 7) / 8, (int64_t)sm_count() * 16);
    const int64_t d3 = D.dim[D.part_of[2]];
    const bool packed = layout == SYM_TTM_PACKED;
    SYM_PROF("pttm", s);
    if (bdt == SYM_BF16) {
        if (packed)
            k_pttm3<true, true><<<grid, 256, 0, s>>>(D, X->idx, X->cap, X->val, nnz, B, ldb, rank, GP, C, d3);
        else
            k_pttm3<true, false><<<grid, 256, 0, s>>>(D, X->idx, X->cap, X->val, nnz, B, ldb, rank, GP, C, d3);
    } else {
        if (packed)
            k_pttm3<false, true><<<grid, 256, 0, s>>>(D, X->idx, X->cap, X->val, nnz, B, ldb, rank, GP, C, d3);
        else
            k_pttm3<false, false><<<grid, 256, 0, s>>>(D, X->idx, X->cap, X->val, nnz, B, ldb, rank, GP, C, d3);
    }
    SYM_CHECK_LAUNCH();
    return SYM_OK;
}

extern "C" sym_status sym_ptensor_destroy(sym_ptensor X) {
    delete X;
    return SYM_OK;
}

// ---------------------------------------------------------------- expansion (baseline)

extern "C" sym_status sym_ptensor_expand_bytes(sym_ptensor X, size_t* arena_bytes, size_t* ws_bytes) {
    if (!X) return SYM_E_INVALID;
    const PartDesc& D = X->D;
    const int64_t E = X->info.expanded_nnz;
    int32_t part[5];
    int64_t dim[5];
    for (int q = 0; q < D.order; ++q) {
        part[q] = 1;
        dim[q] = D.dim[D.part_of[q]];
    }
    size_t ca = 0, cw = 0;
    sym_status st = sym_ptensor_create_bytes(D.order, D.order, part, dim, E, &ca, &cw);
    if (st != SYM_OK) return st;
    Sizer w;
    w.take<int64_t>((size_t)std::max<int64_t>(X->info.nnz, 1) + 1);           // counts -> offsets
    w.take<char>(scan_ws_bytes(std::max<int64_t>(X->info.nnz, 1) + 1));
    w.take<int32_t>((size_t)std::max<int64_t>(E, 1) * (size_t)D.order);        // expanded coordinate list
    w.take<float>((size_t)std::max<int64_t>(E, 1));
    w.take<char>(cw);
    if (arena_bytes) *arena_bytes = ca;
    if (ws_bytes) *ws_bytes = w.used;
    return SYM_OK;
}

extern "C" sym_status sym_ptensor_expand(sym_ptensor X, void* arena, size_t arena_bytes, void* ws, size_t ws_bytes,
                                         sym_stream_t stream, sym_ptensor* out) {
    if (!X || !out) return SYM_E_INVALID;
    *out = nullptr;
    size_t na = 0, nw = 0;
    sym_status st = sym_ptensor_expand_bytes(X, &na, &nw);
    if (st != SYM_OK) return st;
    if (!arena || !ws || !aligned(arena, 256) || !aligned(ws, 256)) return SYM_E_INVALID;
    if (arena_bytes < na || ws_bytes < nw) return SYM_E_NOMEM;
    const PartDesc& D = X->D;
    const int64_t nnz = X->info.nnz, E = X->info.expanded_nnz;
    cudaStream_t s = as_stream(stream);
    Carver W(ws, ws_bytes);
    int64_t* offs = W.take<int64_t>((size_t)std::max<int64_t>(nnz, 1) + 1);
    char* sws = W.take<char>(scan_ws_bytes(std::max<int64_t>(nnz, 1) + 1));
    int32_t* eidx = W.take<int32_t>((size_t)std::max<int64_t>(E, 1) * (size_t)D.order);
    float* evals = W.take<float>((size_t)std::max<int64_t>(E, 1));
    const size_t rest = ws_bytes - W.used;
    char* cws = W.take<char>(1);
    if (!cws) return SYM_E_NOMEM;
    if (nnz > 0) {
        const unsigned g = (unsigned)((nnz + 255) / 256);
#define SYM_PX_CASE(NN)                                                                                  \
    k_pcount<NN><<<g, 256, 0, s>>>(D, X->idx, X->cap, nnz, offs);                                       \
    SYM_CHECK_LAUNCH();                                                                                  \
    st = exclusive_scan_i64(offs, offs, nnz, sws, s);                                                    \
    if (st != SYM_OK) return st;                                                                         \
    k_pexpand<NN><<<g, 256, 0, s>>>(D, X->idx, X->cap, X->val, nnz, offs, eidx, std::max<int64_t>(E, 1), \
                                    evals);                                                              \
    SYM_CHECK_LAUNCH();
        switch (D.order) {
            case 1: { SYM_PX_CASE(1) } break;
            case 2: { SYM_PX_CASE(2) } break;
            case 3: { SYM_PX_CASE(3) } break;
            case 4: { SYM_PX_CASE(4) } break;
            default: { SYM_PX_CASE(5) } break;
        }
#undef SYM_PX_CASE
    }
    int32_t part[5];
    int64_t dim[5];
    for (int q = 0; q < D.order; ++q) {
        part[q] = 1;
        dim[q] = D.dim[D.part_of[q]];
    }
    // cws .. end of ws is the create workspace (256-byte aligned: the carve above)
    return sym_ptensor_create(D.order, D.order, part, dim, E, eidx, std::max<int64_t>(E, 1), evals, SYM_DUP_ERROR,
                              arena, arena_bytes, cws, rest, stream, out);
}
