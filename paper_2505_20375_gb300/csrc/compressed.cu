// Categorically compressed sigma on the STP-DAS layout (Results: categorical compression,
// the CI vector as a direct sum of per-category compressed vectors (V^B, A^B) holding only
// the nonzero coefficients and their addresses; Methods, Algorithm 1 and the compression-
// preservation argument: only nonzero coefficients contribute, and sigma comes out
// compressed as well).
//
// The paper's CPU algorithm intersects, for every intermediate determinant J, the sorted
// excitation list of J with the sorted addresses of the nonzero coefficients (exponential
// search), and accumulates sigma in per-category hash tables.  On the GPU the columns J
// are found from the other side (no scan over every J of the connected categories), D is
// gathered with that exponential search, and sigma is gathered on its support:
//   1. every nonzero C_K emits its single replacements J = E_sr K (alpha and beta moves
//      from the string tables), which are the only intermediate determinants whose
//      D[rs, J] = sum_K <J|E_rs|K> C_K can be nonzero; a hash table gives each distinct J a
//      column.  D[rs, J] is then gathered per column as Algorithm 1 does: the source K of
//      each move of J (one alpha, one beta) is looked up in the ascending nonzero addresses
//      of K's category by exponential search (galloping, then a binary search for the
//      lower bound), and the (at most two) values found are summed;
//   2. E = G D over those columns only, as the dense FP64 contraction computes it but
//      skipping the zero entries of D (the same multiply-adds in the same order);
//   3. every column J emits its single replacements L inside the target space: the
//      structural support of sigma, made distinct by a second hash table and sorted
//      (radix sort on the address), which is the compressed output order;
//   4. sigma_L = sum_pq <L|E_pq|J> E[pq, J] + e_core C_L for every L of the support,
//      gathering over L's replacements in pair order (alpha then beta), looking each J up
//      in the first table (absent J have E = 0): the arithmetic and its order are those of
//      the dense FP64 DAS path, so the result equals the dense sigma on the support and
//      the dense sigma is zero elsewhere.
// The pair tables are read string-major (one string's row contiguous; copies built on the
// first call and kept by the handle).  Hash tables use open addressing with linear
// probing over a power-of-two capacity of at least twice the largest number of keys, so no
// probe sequence runs past a free slot; every probe loop is bounded by the capacity all
// the same and reports an overflow instead.
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "das_dev.cuh"

namespace {

using das_dev::das_addr;
using das_dev::das_strings;
using das_dev::DasDev;
using das_dev::make_dev;

constexpr unsigned long long HT_EMPTY = ~0ull;
constexpr int RS_THREADS = 256, RS_ITEMS = 32, RS_TILE = RS_THREADS * RS_ITEMS;  // radix sort tile (8192 keys)

inline size_t al(size_t b) { return (b + 255) & ~(size_t)255; }

// Home slot of key k in a table of mask + 1 (a power of two) slots: Fibonacci hashing, the
// top log2(capacity) bits of k times 2^64 / golden ratio (one multiply and a shift).
__device__ __forceinline__ uint64_t hslot(uint64_t k, uint64_t mask) {
    return (k * 0x9E3779B97F4A7C15ull) >> (64 - __popcll(mask));
}

// Insert key k (>= 0) once.  Returns false if every slot was probed (cannot happen at
// the capacities used; reported as an overflow).
__device__ bool ht_insert(unsigned long long *keys, uint64_t mask, uint64_t k) {
    uint64_t p = hslot(k, mask);
    for (uint64_t probe = 0; probe <= mask; ++probe) {
        const unsigned long long old = atomicCAS(keys + p, HT_EMPTY, (unsigned long long)k);
        if (old == HT_EMPTY || old == k) return true;
        p = (p + 1) & mask;
    }
    return false;
}

// Column of key k, or -1 if k is not in the table.
__device__ int64_t ht_find(const unsigned long long *__restrict__ keys, const int32_t *__restrict__ cols, uint64_t mask,
                           uint64_t k) {
    uint64_t p = hslot(k, mask);
    for (uint64_t probe = 0; probe <= mask; ++probe) {
        const unsigned long long v = keys[p];
        if (v == k) return cols[p];
        if (v == HT_EMPTY) return -1;
        p = (p + 1) & mask;
    }
    return -1;
}

struct CsArgs {
    DasDev d;
    int n_cat_int, nent_a, nent_b, npair;
    const uint64_t *rep_a, *rep_b;   // packed replacement lists [n_str][n_ent]
    const int32_t *pair_a, *pair_b;  // string-major pair tables [n_str][ldp]: (T << 1) | sign, or -1
    int ldp;                         // n_pair_pad
    const int64_t *c_addr;
    const double *c_val;
    int64_t nnz_c;
    int64_t *nz_lo;                  // [n_cat + 1]: first nonzero of each target category
    unsigned long long *hj;          // intermediate determinants J
    int32_t *hj_col;
    uint64_t hj_mask;
    int64_t *j_addr;                 // [n1]: the J of each column
    uint32_t *bm_a, *bm_b;           // bit A (B) set: some column has alpha (beta) string A (B)
    double *D, *E;                   // [n_pair][ldd]
    int64_t ldd;
    unsigned long long *hl;          // target determinants L of the support
    uint64_t hl_mask;
    int64_t *l_addr;                 // [n2]
    unsigned long long *counts;      // [0]: columns n1, [1]: support n2, [2]: overflow flag
    double e_core;
};

// Step 1: every move of every nonzero C_K inserts its target J.
__global__ void __launch_bounds__(256) k_cs_expand(const __grid_constant__ CsArgs a) {
    const int nm = a.nent_a + a.nent_b;
    const int64_t total = a.nnz_c * nm;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = t / nm;
        const int m = (int)(t - i * nm);
        int32_t A, B;
        int pb;
        das_strings(a.d, a.d.n_cat, a.c_addr[i], A, B, pb);
        uint64_t e;
        int64_t J;
        if (m < a.nent_a) {
            e = a.rep_a[(int64_t)A * a.nent_a + m];
            J = das_addr(a.d, (int32_t)rep_target(e), B);
        } else {
            e = a.rep_b[(int64_t)B * a.nent_b + (m - a.nent_a)];
            J = das_addr(a.d, A, (int32_t)rep_target(e));
        }
        if (J >= 0 && !ht_insert(a.hj, a.hj_mask, (uint64_t)J)) atomicExch(a.counts + 2, 1ull);
    }
}

// Index of key in the ascending a[lo, hi), or -1: steps of 1, 2, 4, ... from lo bracket
// the key (Algorithm 1's exponentialSearch), then a binary search finds its lower bound.
__device__ int64_t exp_search(const int64_t *__restrict__ a, int64_t lo, int64_t hi, int64_t key) {
    if (lo >= hi) return -1;
    int64_t b = 1;
    while (lo + b < hi && a[lo + b] < key) b <<= 1;
    int64_t l = lo + (b >> 1), r = min(lo + b, hi - 1);
    while (l < r) {
        const int64_t m = (l + r) >> 1;
        if (a[m] < key) l = m + 1;
        else r = m;
    }
    return a[l] == key ? l : -1;
}

// nz_lo[c] = first index of a nonzero coefficient at or after the start of target category c
// (c = n_cat: the end of the target space), by binary search.
__global__ void k_cs_cat_ranges(const __grid_constant__ CsArgs a) {
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c <= a.d.n_cat; c += gridDim.x * blockDim.x) {
        const int64_t key = c < a.d.n_cat ? a.d.cat_off[c] : a.d.n_det;
        int64_t lo = 0, hi = a.nnz_c;
        while (lo < hi) {
            const int64_t m = (lo + hi) >> 1;
            if (a.c_addr[m] < key) lo = m + 1;
            else hi = m;
        }
        a.nz_lo[c] = lo;
    }
}

// The value of the target determinant K in the compressed C, or 0.
__device__ __forceinline__ bool cs_coef(const CsArgs &a, int64_t K, double &v) {
    if (K < 0 || K >= a.d.n_det) return false;
    const int c = das_dev::find_cat(a.d.cat_off, a.d.n_cat, K);
    const int64_t i = exp_search(a.c_addr, a.nz_lo[c], a.nz_lo[c + 1], K);
    if (i < 0) return false;
    v = a.c_val[i];
    return true;
}

// D[pair, column] for every column J and pair: the alpha source and the beta source of J
// under the pair, each looked up among the nonzero coefficients (Algorithm 1's
// intersection of J's excitation list with the compressed vector).
__global__ void __launch_bounds__(256) k_cs_gather(const __grid_constant__ CsArgs a, int64_t n1) {
    const int64_t total = n1 * a.npair;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t j = t / a.npair;
        const int pp = (int)(t - j * a.npair);
        int32_t A, B;
        int pb;
        das_strings(a.d, a.n_cat_int, a.j_addr[j], A, B, pb);
        double d = 0.0, v;
        const int32_t ea = __ldg(a.pair_a + (int64_t)A * a.ldp + pp);
        if (ea >= 0 && cs_coef(a, das_addr(a.d, ea >> 1, B), v)) d += (ea & 1) ? -v : v;
        const int32_t eb = __ldg(a.pair_b + (int64_t)B * a.ldp + pp);
        if (eb >= 0 && cs_coef(a, das_addr(a.d, A, eb >> 1), v)) d += (eb & 1) ? -v : v;
        a.D[(int64_t)pp * a.ldd + j] = d;
    }
}

// Step 2: E[:, J] = G D[:, J] for every column, one warp per column: the warp walks the
// column 32 rows at a time, and for each nonzero D[rs, J] (ballot, ascending rs) every lane
// adds G[pq, rs] D[rs, J] to its rows pq = lane + 32 i with a fused multiply-add.  These
// are the multiply-adds of the dense product in the same order without its terms
// G[pq, rs] x 0 (which change no bit), so E equals the dense FP64 product; the columns hold
// only the moves into a sparse vector, so this is a small fraction of its work.
constexpr int CS_RPL = 17;  // rows per lane: n_pair <= 544 (32 orbitals)
__global__ void __launch_bounds__(256) k_cs_spmm(const double *__restrict__ G, int npair, const double *__restrict__ D,
                                                 int64_t ldd, int64_t n1, double *__restrict__ E) {
    const int lane = threadIdx.x & 31;
    const int64_t nw = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t j = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); j < n1; j += nw) {
        double acc[CS_RPL];
#pragma unroll
        for (int i = 0; i < CS_RPL; ++i) acc[i] = 0.0;
        for (int r0 = 0; r0 < npair; r0 += 32) {
            const int rs = r0 + lane;
            const double d = rs < npair ? D[(int64_t)rs * ldd + j] : 0.0;
            unsigned nz = __ballot_sync(0xFFFFFFFFu, d != 0.0);
            while (nz) {
                const int b = __ffs(nz) - 1;
                nz &= nz - 1;
                const double v = __shfl_sync(0xFFFFFFFFu, d, b);
                const double *g = G + (r0 + b);
#pragma unroll
                for (int i = 0; i < CS_RPL; ++i) {
                    const int pq = lane + 32 * i;
                    if (pq < npair) acc[i] = fma(g[(int64_t)pq * npair], v, acc[i]);
                }
            }
        }
#pragma unroll
        for (int i = 0; i < CS_RPL; ++i) {
            const int pq = lane + 32 * i;
            if (pq < npair) E[(int64_t)pq * ldd + j] = acc[i];
        }
    }
}

// dst[c][r] = src[r][c] for an R x C int32 table (32 x 32 tiles through shared memory, so
// that both the reads and the writes are coalesced).
__global__ void k_cs_transpose(const int32_t *__restrict__ src, int64_t R, int64_t C, int32_t *__restrict__ dst) {
    __shared__ int32_t t[32][33];
    const int64_t c0 = (int64_t)blockIdx.x * 32, r0 = (int64_t)blockIdx.y * 32;
    for (int i = threadIdx.y; i < 32; i += blockDim.y) {
        const int64_t r = r0 + i, c = c0 + threadIdx.x;
        if (r < R && c < C) t[i][threadIdx.x] = src[r * C + c];
    }
    __syncthreads();
    for (int i = threadIdx.y; i < 32; i += blockDim.y) {
        const int64_t c = c0 + i, r = r0 + threadIdx.x;
        if (r < R && c < C) dst[c * R + r] = t[threadIdx.x][i];
    }
}

// The alpha and beta strings of every column, as bitmaps (a sigma entry looks a candidate
// column up only if both of its strings occur in some column).
__global__ void k_cs_mark(const __grid_constant__ CsArgs a, int64_t n1) {
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < n1; j += (int64_t)gridDim.x * blockDim.x) {
        int32_t A, B;
        int pb;
        das_strings(a.d, a.n_cat_int, a.j_addr[j], A, B, pb);
        atomicOr(a.bm_a + (A >> 5), 1u << (A & 31));
        atomicOr(a.bm_b + (B >> 5), 1u << (B & 31));
    }
}

__device__ __forceinline__ bool bit(const uint32_t *__restrict__ bm, int32_t i) { return (__ldg(bm + (i >> 5)) >> (i & 31)) & 1u; }

// Distinct keys of a table get consecutive columns.
__global__ void k_cs_compact(unsigned long long *keys, int32_t *cols, uint64_t cap, int64_t *addr,
                             unsigned long long *counter) {
    for (uint64_t p = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; p < cap; p += (uint64_t)gridDim.x * blockDim.x) {
        const unsigned long long k = keys[p];
        if (k == HT_EMPTY) continue;
        const unsigned long long c = atomicAdd(counter, 1ull);
        if (cols) cols[p] = (int32_t)c;
        addr[c] = (int64_t)k;
    }
}

// Step 3: the target determinants one move away from a column J.
__global__ void __launch_bounds__(256) k_cs_support(const __grid_constant__ CsArgs a, int64_t n1) {
    const int nm = a.nent_a + a.nent_b;
    const int64_t total = n1 * nm;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t j = t / nm;
        const int m = (int)(t - j * nm);
        int32_t A, B;
        int pb;
        das_strings(a.d, a.n_cat_int, a.j_addr[j], A, B, pb);
        int64_t L;
        if (m < a.nent_a) L = das_addr(a.d, (int32_t)rep_target(a.rep_a[(int64_t)A * a.nent_a + m]), B);
        else L = das_addr(a.d, A, (int32_t)rep_target(a.rep_b[(int64_t)B * a.nent_b + (m - a.nent_a)]));
        if (L < 0 || L >= a.d.n_det) continue;
        if (!ht_insert(a.hl, a.hl_mask, (uint64_t)L)) atomicExch(a.counts + 2, 1ull);
    }
}

// Step 4: sigma on the sorted support, in the dense DAS path's order of terms.
__global__ void __launch_bounds__(256) k_cs_sigma(const __grid_constant__ CsArgs a, const int64_t *__restrict__ l_sorted,
                                                  int64_t n2, double *__restrict__ out_val) {
    for (int64_t o = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; o < n2; o += (int64_t)gridDim.x * blockDim.x) {
        const int64_t L = l_sorted[o];
        int32_t A, B;
        int pb;
        das_strings(a.d, a.d.n_cat, L, A, B, pb);
        double acc = 0.0;
        const int4 *ra = reinterpret_cast<const int4 *>(a.pair_a + (int64_t)A * a.ldp);
        const int4 *rb = reinterpret_cast<const int4 *>(a.pair_b + (int64_t)B * a.ldp);
        // an alpha move keeps B and a beta move keeps A: no column has them, no lookup
        const bool try_a = bit(a.bm_b, B), try_b = bit(a.bm_a, A);
        const int4 none = make_int4(-1, -1, -1, -1);
        for (int p4 = 0; p4 < a.npair && (try_a || try_b); p4 += 4) {  // four pairs per 16-byte load of a row
            const int4 va = try_a ? __ldg(ra + p4 / 4) : none, vb = try_b ? __ldg(rb + p4 / 4) : none;
            const int32_t ea4[4] = {va.x, va.y, va.z, va.w}, eb4[4] = {vb.x, vb.y, vb.z, vb.w};
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const double *Ep = a.E + (int64_t)(p4 + k) * a.ldd;  // rows past n_pair hold -1
                const int32_t ea = ea4[k];
                if (ea >= 0 && bit(a.bm_a, ea >> 1)) {
                    const int64_t J = das_addr(a.d, ea >> 1, B);
                    const int64_t col = J >= 0 ? ht_find(a.hj, a.hj_col, a.hj_mask, (uint64_t)J) : -1;
                    if (col >= 0) {
                        const double e = Ep[col];
                        acc += (ea & 1) ? -e : e;
                    }
                }
                const int32_t eb = eb4[k];
                if (eb >= 0 && bit(a.bm_b, eb >> 1)) {
                    const int64_t J = das_addr(a.d, A, eb >> 1);
                    const int64_t col = J >= 0 ? ht_find(a.hj, a.hj_col, a.hj_mask, (uint64_t)J) : -1;
                    if (col >= 0) {
                        const double e = Ep[col];
                        acc += (eb & 1) ? -e : e;
                    }
                }
            }
        }
        // C_L from the sorted nonzero addresses (binary search)
        double cl = 0.0;
        int64_t lo = 0, hi = a.nnz_c - 1;
        while (lo <= hi) {
            const int64_t mid = (lo + hi) >> 1;
            const int64_t v = a.c_addr[mid];
            if (v == L) { cl = a.c_val[mid]; break; }
            if (v < L) lo = mid + 1; else hi = mid - 1;
        }
        out_val[o] = fma(a.e_core, cl, acc);  // as the dense FP64 scatter
    }
}

// ------------------------------------------------------------------ LSD radix sort
// 8-bit digits, ascending, stable; one tile = RS_TILE keys.  Histograms per tile and
// digit, an exclusive scan over (digit, tile), then a stable scatter: inside a tile the
// keys keep their order (rounds of 256 keys; within a round, warps in order and lanes in
// order, ranks from __match_any_sync).

__global__ void __launch_bounds__(RS_THREADS) k_rs_hist(const uint64_t *__restrict__ keys, int64_t n, int shift,
                                                        int64_t ntiles, unsigned long long *__restrict__ counts) {
    __shared__ unsigned int h[256];
    for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        h[threadIdx.x] = 0;
        __syncthreads();
        for (int r = 0; r < RS_ITEMS; ++r) {
            const int64_t idx = tile * RS_TILE + r * RS_THREADS + threadIdx.x;
            if (idx < n) atomicAdd(&h[(keys[idx] >> shift) & 255], 1u);
        }
        __syncthreads();
        counts[(int64_t)threadIdx.x * ntiles + tile] = h[threadIdx.x];
        __syncthreads();
    }
}

// Exclusive scan of m counts in one block of 1024 threads, 8192 counts at a time: each
// thread loads 8 consecutive counts (issued together) and scans them, a scan of the 1024
// thread totals (inside each warp, then over the 32 warp totals) gives each thread its
// offset, plus the running total of the chunks before.
__global__ void __launch_bounds__(1024) k_rs_scan(unsigned long long *__restrict__ c, int64_t m) {
    constexpr int IPT = 8;
    __shared__ unsigned long long wsum[32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    unsigned long long carry = 0;  // the same in every thread
    for (int64_t base = 0; base < m; base += 1024 * IPT) {
        const int64_t i0 = base + (int64_t)threadIdx.x * IPT;
        unsigned long long v[IPT], tot = 0;
#pragma unroll
        for (int k = 0; k < IPT; ++k) v[k] = i0 + k < m ? c[i0 + k] : 0ull;
#pragma unroll
        for (int k = 0; k < IPT; ++k) {
            const unsigned long long t = v[k];
            v[k] = tot;  // exclusive inside the thread
            tot += t;
        }
        unsigned long long x = tot;  // inclusive scan of the thread totals inside the warp
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned long long y = __shfl_up_sync(0xFFFFFFFFu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) wsum[warp] = x;
        __syncthreads();
        if (warp == 0) {
            unsigned long long t = wsum[lane];
            for (int o = 1; o < 32; o <<= 1) {
                const unsigned long long y = __shfl_up_sync(0xFFFFFFFFu, t, o);
                if (lane >= o) t += y;
            }
            wsum[lane] = t;  // inclusive over the warps
        }
        __syncthreads();
        const unsigned long long off = carry + (warp ? wsum[warp - 1] : 0ull) + x - tot;
#pragma unroll
        for (int k = 0; k < IPT; ++k)
            if (i0 + k < m) c[i0 + k] = off + v[k];
        carry += wsum[31];
        __syncthreads();  // wsum is rewritten by the next chunk
    }
}

__global__ void __launch_bounds__(RS_THREADS) k_rs_scatter(const uint64_t *__restrict__ in, uint64_t *__restrict__ out,
                                                           int64_t n, int shift, int64_t ntiles,
                                                           const unsigned long long *__restrict__ base) {
    __shared__ unsigned int run[256];
    __shared__ unsigned int wc[RS_THREADS / 32][256];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        run[threadIdx.x] = 0;
        for (int r = 0; r < RS_ITEMS; ++r) {
            for (int w = 0; w < RS_THREADS / 32; ++w) wc[w][threadIdx.x] = 0;
            __syncthreads();
            const int64_t idx = tile * RS_TILE + r * RS_THREADS + threadIdx.x;
            const bool valid = idx < n;
            const uint64_t key = valid ? in[idx] : 0;
            const unsigned dg = valid ? (unsigned)((key >> shift) & 255) : 256u + lane;  // invalid lanes match no one
            const unsigned peers = __match_any_sync(0xFFFFFFFFu, dg);
            const unsigned rank = __popc(peers & ((1u << lane) - 1u));
            if (valid && rank == 0) wc[warp][dg] = __popc(peers);
            __syncthreads();
            if (valid) {
                unsigned off = run[dg] + rank;
                for (int w = 0; w < warp; ++w) off += wc[w][dg];
                out[base[(int64_t)dg * ntiles + tile] + off] = key;
            }
            __syncthreads();
            unsigned add = 0;
            for (int w = 0; w < RS_THREADS / 32; ++w) add += wc[w][threadIdx.x];
            run[threadIdx.x] += add;
            __syncthreads();
        }
    }
}

unsigned grid_of(int64_t n) { return (unsigned)std::max<int64_t>(1, std::min<int64_t>(ceil_div(n, 256), 152 * 32)); }

uint64_t pow2_at_least(uint64_t x) {
    uint64_t c = 1024;
    while (c < x) c <<= 1;
    return c;
}

// Sizes of the compressed sigma's buffers for nnz_c nonzero coefficients: columns and
// support are bounded by the number of moves; hash tables hold twice their bound.
struct CsSizes {
    int64_t n1max, n2max;
    uint64_t capj, capl;
    int64_t ntiles;
    size_t bytes;
    size_t off_hj, off_hjc, off_jaddr, off_D, off_E, off_hl, off_laddr, off_tmp, off_cnt, off_hist, off_nzlo, off_bm;
    size_t bm_bytes;
};

CsSizes cs_sizes(const fci_context *h, int64_t nnz_c) {
    CsSizes z;
    const int64_t nm = h->nent_a + h->nent_b;
    z.n1max = std::max<int64_t>(1, nnz_c * nm);
    z.n2max = std::max<int64_t>(1, z.n1max * nm);
    z.capj = pow2_at_least((uint64_t)(2 * z.n1max));
    z.capl = pow2_at_least((uint64_t)(2 * z.n2max));
    z.ntiles = ceil_div(z.n2max, RS_TILE);
    size_t o = 0;
    z.off_hj = o; o += al(z.capj * 8);
    z.off_hjc = o; o += al(z.capj * 4);
    z.off_jaddr = o; o += al((size_t)z.n1max * 8);
    z.off_D = o; o += al((size_t)h->npair * z.n1max * 8);
    z.off_E = o; o += al((size_t)h->npair * z.n1max * 8);
    z.off_hl = o; o += al(z.capl * 8);
    z.off_laddr = o; o += al((size_t)z.n2max * 8);
    z.off_tmp = o; o += al((size_t)z.n2max * 8);
    z.off_hist = o; o += al((size_t)256 * z.ntiles * 8);
    z.off_nzlo = o; o += al((size_t)(h->das.n_cat + 1) * 8);
    z.bm_bytes = (size_t)((h->nsa + 31) / 32 + (h->nsb + 31) / 32) * 4;
    z.off_bm = o; o += al(z.bm_bytes);
    z.off_cnt = o; o += 256;
    z.bytes = o;
    return z;
}

}  // namespace

extern "C" {

int fci_sigma_compressed_workspace_bytes(fci_handle h, int64_t nnz_c, size_t *bytes) {
    if (!h || !bytes || nnz_c < 0) return fci_fail(h, FCI_ERR_ARG, "bad argument");
    if (!h->das_active) return fci_fail(h, FCI_ERR_STATE, "compressed sigma needs the DAS layout");
    *bytes = cs_sizes(h, nnz_c).bytes;
    return FCI_OK;
}

int fci_sigma_compressed(fci_handle h, const int64_t *c_addr, const double *c_val, int64_t nnz_c, int64_t *out_addr,
                         double *out_val, int64_t capacity, int64_t *nnz_sigma, void *ws, size_t ws_bytes,
                         fci_stream stream) {
    if (!h) return fci_fail(nullptr, FCI_ERR_ARG, "NULL handle");
    if (!h->das_active) return fci_fail(h, FCI_ERR_STATE, "compressed sigma needs the DAS layout");
    if (h->dtype != FCI_R64) return fci_fail(h, FCI_ERR_UNSUPPORTED, "compressed sigma is built for real integrals");
    if (!nnz_sigma || nnz_c < 0 || capacity < 0 || (nnz_c && (!c_addr || !c_val)) || (capacity && (!out_addr || !out_val)))
        return fci_fail(h, FCI_ERR_ARG, "bad compressed-vector arguments");
    const CsSizes z = cs_sizes(h, nnz_c);
    if (!ws || ws_bytes < z.bytes || ((uintptr_t)ws & 255))
        return fci_fail(h, FCI_ERR_ARG, "workspace %zu < %zu bytes or misaligned", ws_bytes, z.bytes);
    if (z.n1max >= ((int64_t)1 << 31)) return fci_fail(h, FCI_ERR_UNSUPPORTED, "too many nonzero coefficients");
    if (h->npair > 32 * CS_RPL) return fci_fail(h, FCI_ERR_UNSUPPORTED, "compressed sigma: %d orbital pairs", h->npair);
    FCI_CUDA(h, cudaSetDevice(h->device));
    cudaStream_t s = (cudaStream_t)stream;
    *nnz_sigma = 0;
    if (nnz_c == 0) return FCI_OK;
    // the addresses must be ascending target addresses (checked on the device copy)
    std::vector<int64_t> hc(nnz_c);
    FCI_CUDA(h, cudaMemcpyAsync(hc.data(), c_addr, nnz_c * 8, cudaMemcpyDeviceToHost, s));
    FCI_CUDA(h, cudaStreamSynchronize(s));
    for (int64_t i = 0; i < nnz_c; ++i)
        if (hc[i] < 0 || hc[i] >= h->das.n_det || (i && hc[i] <= hc[i - 1]))
            return fci_fail(h, FCI_ERR_ARG, "compressed C: addresses must be ascending target addresses");
    char *w = (char *)ws;
    CsArgs a;
    a.d = make_dev(h);
    a.n_cat_int = h->das.n_cat_int;
    a.nent_a = h->nent_a;
    a.nent_b = h->nent_b;
    a.npair = h->npair;
    a.rep_a = h->d_rep_a;
    a.rep_b = h->d_rep_b;
    if (!h->d_pair_a_t) {  // string-major copies of the pair tables: one string's row is contiguous
        const int64_t R = h->npair_pad;
        int rc = fci_dev_alloc(h, (void **)&h->d_pair_a_t, (size_t)R * h->nsa * 4);
        if (!rc) rc = fci_dev_alloc(h, (void **)&h->d_pair_b_t, (size_t)R * h->nsb * 4);
        if (rc) {
            fci_dev_free(h->d_pair_a_t);
            h->d_pair_a_t = nullptr;
            return rc;
        }
        const dim3 blk(32, 8);
        const unsigned gy = (unsigned)ceil_div(R, 32);
        k_cs_transpose<<<dim3((unsigned)ceil_div(h->nsa, 32), gy), blk, 0, s>>>(h->d_pair_a, R, h->nsa, h->d_pair_a_t);
        k_cs_transpose<<<dim3((unsigned)ceil_div(h->nsb, 32), gy), blk, 0, s>>>(h->d_pair_b, R, h->nsb, h->d_pair_b_t);
        FCI_CUDA(h, cudaGetLastError());
    }
    a.pair_a = h->d_pair_a_t;
    a.pair_b = h->d_pair_b_t;
    a.ldp = h->npair_pad;
    a.c_addr = c_addr;
    a.c_val = c_val;
    a.nnz_c = nnz_c;
    a.nz_lo = (int64_t *)(w + z.off_nzlo);
    a.bm_a = (uint32_t *)(w + z.off_bm);
    a.bm_b = a.bm_a + (h->nsa + 31) / 32;
    a.hj = (unsigned long long *)(w + z.off_hj);
    a.hj_col = (int32_t *)(w + z.off_hjc);
    a.hj_mask = z.capj - 1;
    a.j_addr = (int64_t *)(w + z.off_jaddr);
    a.D = (double *)(w + z.off_D);
    a.E = (double *)(w + z.off_E);
    a.ldd = z.n1max;
    a.hl = (unsigned long long *)(w + z.off_hl);
    a.hl_mask = z.capl - 1;
    a.l_addr = (int64_t *)(w + z.off_laddr);
    a.counts = (unsigned long long *)(w + z.off_cnt);
    a.e_core = h->e_core;
    unsigned long long cnt[3] = {0, 0, 0};
    // 1. the intermediate determinants one move from a nonzero coefficient, and D on them
    {
        phase_scope ps(h, s, FCI_PHASE_GATHER, 4);
        FCI_CUDA(h, cudaMemsetAsync(a.hj, 0xFF, z.capj * 8, s));
        FCI_CUDA(h, cudaMemsetAsync(a.counts, 0, 256, s));
        const int64_t moves = nnz_c * (a.nent_a + a.nent_b);
        k_cs_expand<<<grid_of(moves), 256, 0, s>>>(a);
        k_cs_cat_ranges<<<(unsigned)ceil_div(h->das.n_cat + 1, 256), 256, 0, s>>>(a);
        k_cs_compact<<<grid_of((int64_t)z.capj), 256, 0, s>>>(a.hj, a.hj_col, z.capj, a.j_addr, a.counts);
        FCI_CUDA(h, cudaMemcpyAsync(cnt, a.counts, sizeof cnt, cudaMemcpyDeviceToHost, s));
        FCI_CUDA(h, cudaStreamSynchronize(s));
        if (cnt[2]) return fci_fail(h, FCI_ERR_CUDA, "compressed sigma: hash table overflow");
        k_cs_gather<<<grid_of((int64_t)cnt[0] * h->npair), 256, 0, s>>>(a, (int64_t)cnt[0]);
        FCI_CUDA(h, cudaMemsetAsync(a.bm_a, 0, z.bm_bytes, s));
        k_cs_mark<<<grid_of((int64_t)cnt[0]), 256, 0, s>>>(a, (int64_t)cnt[0]);
        FCI_CUDA(h, cudaGetLastError());
    }
    const int64_t n1 = (int64_t)cnt[0];
    // 2. E = G D on the n1 columns
    {
        phase_scope ps(h, s, FCI_PHASE_CONTRACT, 1);
        k_cs_spmm<<<(unsigned)std::max<int64_t>(1, std::min<int64_t>(ceil_div(n1, 8), 152 * 16)), 256, 0, s>>>(
            h->d_G, h->npair, a.D, z.n1max, n1, a.E);
        FCI_CUDA(h, cudaGetLastError());
    }
    // 3. the support of sigma, distinct and sorted
    {
        phase_scope ps(h, s, FCI_PHASE_OTHER, 3);
        FCI_CUDA(h, cudaMemsetAsync(a.hl, 0xFF, z.capl * 8, s));
        k_cs_support<<<grid_of(n1 * (a.nent_a + a.nent_b)), 256, 0, s>>>(a, n1);
        k_cs_compact<<<grid_of((int64_t)z.capl), 256, 0, s>>>(a.hl, nullptr, z.capl, a.l_addr, a.counts + 1);
        FCI_CUDA(h, cudaMemcpyAsync(cnt, a.counts, sizeof cnt, cudaMemcpyDeviceToHost, s));
        FCI_CUDA(h, cudaStreamSynchronize(s));
        if (cnt[2]) return fci_fail(h, FCI_ERR_CUDA, "compressed sigma: hash table overflow");
    }
    const int64_t n2 = (int64_t)cnt[1];
    *nnz_sigma = n2;
    if (n2 > capacity)
        return fci_fail(h, FCI_ERR_ARG, "output capacity %lld < %lld support entries", (long long)capacity, (long long)n2);
    uint64_t *src = (uint64_t *)a.l_addr, *dst = (uint64_t *)(w + z.off_tmp);
    {
        phase_scope ps(h, s, FCI_PHASE_OTHER, 1);
        int bits = 1;
        while (bits < 63 && ((uint64_t)1 << bits) < (uint64_t)h->das.n_det) ++bits;
        const int64_t nt = ceil_div(n2, RS_TILE);
        unsigned long long *hist = (unsigned long long *)(w + z.off_hist);
        const unsigned g = (unsigned)std::max<int64_t>(1, std::min<int64_t>(nt, 152 * 8));
        for (int shift = 0; shift < bits; shift += 8) {
            k_rs_hist<<<g, RS_THREADS, 0, s>>>(src, n2, shift, nt, hist);
            k_rs_scan<<<1, 1024, 0, s>>>(hist, 256 * nt);
            k_rs_scatter<<<g, RS_THREADS, 0, s>>>(src, dst, n2, shift, nt, hist);
            std::swap(src, dst);
        }
        FCI_CUDA(h, cudaGetLastError());
        FCI_CUDA(h, cudaMemcpyAsync(out_addr, src, n2 * 8, cudaMemcpyDeviceToDevice, s));
    }
    // 4. sigma on the support
    {
        phase_scope ps(h, s, FCI_PHASE_SCATTER, 1);
        k_cs_sigma<<<grid_of(n2), 256, 0, s>>>(a, out_addr, n2, out_val);
        FCI_CUDA(h, cudaGetLastError());
    }
    FCI_CUDA(h, cudaStreamSynchronize(s));
    return FCI_OK;
}

}  // extern "C"
