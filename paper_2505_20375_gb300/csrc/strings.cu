// Occupation strings and single-replacement lists on the device.
//
// A string of m orbitals with ne electrons is a bit mask; strings are numbered by the
// combinadic rank sum_j C(p_j, j) (occupied p_1 < ... < p_ne, j from 1), which is the
// position of the mask in ascending integer order.  The single-replacement list of a
// string S (the one-electron excitation list whose size the paper's Introduction gives
// as n_e (n_h + 1) per string) holds T = S - a + b for occupied a and b empty or b = a,
// with the sign <S|a+_a a_b|T> = (-1)^popc(S strictly between a and b).
#include "fci_internal.h"

namespace {

constexpr unsigned FULL = 0xFFFFFFFFu;

// Unrank: greedy descent through the combinatorial number system.
__global__ void k_strings_unrank(int m, int ne, int64_t ns, const uint64_t *__restrict__ binom,
                                 uint64_t *__restrict__ out) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= ns) return;
    uint64_t r = (uint64_t)i, mask = 0;
    int p = m - 1;
    for (int j = ne; j >= 1; --j) {
        while (binom[p * FCI_BINOM_LD + j] > r) --p;
        mask |= 1ull << p;
        r -= binom[p * FCI_BINOM_LD + j];
        --p;
    }
    out[i] = mask;
}

// Rank of a mask of at most 32 orbitals, with one lane per orbital: the lane of
// orbital p learns from the ballot how many electrons lie below p (its 1-based
// position j among the occupied orbitals) and contributes C(p, j); the warp sums.
__device__ __forceinline__ uint32_t warp_rank(uint32_t mask, const uint64_t *__restrict__ binom) {
    const int lane = threadIdx.x & 31;
    const uint32_t bit = (mask >> lane) & 1u;
    const uint32_t occ = __ballot_sync(FULL, bit);
    const uint32_t j = __popc(occ & ((1u << lane) - 1u)) + 1u;
    const uint32_t c = bit ? (uint32_t)binom[lane * FCI_BINOM_LD + j] : 0u;
    return __reduce_add_sync(FULL, c);
}

// One warp per string; lanes are orbitals for the ranking.  Writes the packed list and,
// optionally, the pair-major dense table pairtab[pair][string] = (T << 1) | neg.
__global__ void k_repl_table(int m, int ne, int64_t ns, const uint64_t *__restrict__ str,
                             const uint64_t *__restrict__ binom, int n_ent, int packed_pairs,
                             uint64_t *__restrict__ rep, int32_t *__restrict__ pairtab) {
    const int64_t w = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (w >= ns) return;  // uniform per warp
    const uint32_t S = (uint32_t)str[w];
    int e = 0;
    for (int a = 0; a < m; ++a) {
        if (!((S >> a) & 1u)) continue;
        for (int b = 0; b < m; ++b) {
            if (b != a && ((S >> b) & 1u)) continue;
            const uint32_t T = (S & ~(1u << a)) | (1u << b);
            const uint32_t t = warp_rank(T, binom);
            const int lo = a < b ? a : b, hi = a < b ? b : a;
            const uint32_t between = (hi > lo + 1) ? (((1u << hi) - 1u) & ~((2u << lo) - 1u)) : 0u;
            const int neg = __popc(S & between) & 1;
            const int pair = packed_pairs ? pair_index(a, b) : a * m + b;
            if (lane == 0) {
                rep[w * n_ent + e] = rep_pack(t, a, b, neg, pair);
                if (pairtab) pairtab[(int64_t)pair * ns + w] = (int32_t)((t << 1) | (uint32_t)neg);
            }
            ++e;
        }
    }
}

__global__ void k_export_repl(int64_t n, const uint64_t *__restrict__ rep, int32_t *__restrict__ dst) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    uint64_t e = rep[i];
    dst[4 * i + 0] = (int32_t)rep_target(e);
    dst[4 * i + 1] = rep_a(e);
    dst[4 * i + 2] = rep_b(e);
    dst[4 * i + 3] = rep_neg(e) ? -1 : 1;
}

}  // namespace

cudaError_t launch_strings_unrank(int m, int ne, int64_t ns, const uint64_t *binom, uint64_t *out,
                                  cudaStream_t s) {
    if (ns <= 0) return cudaSuccess;
    k_strings_unrank<<<(unsigned)ceil_div(ns, 256), 256, 0, s>>>(m, ne, ns, binom, out);
    return cudaGetLastError();
}

cudaError_t launch_repl_table(int m, int ne, int64_t ns, const uint64_t *str, const uint64_t *binom,
                              int n_ent, int packed_pairs, uint64_t *rep, int32_t *pairtab,
                              int npair, cudaStream_t s) {
    (void)ne;
    if (ns <= 0) return cudaSuccess;
    if (pairtab) {
        cudaError_t e = cudaMemsetAsync(pairtab, 0xFF, sizeof(int32_t) * (size_t)npair * ns, s);
        if (e != cudaSuccess) return e;
    }
    const int threads = 256;  // 8 strings per block
    k_repl_table<<<(unsigned)ceil_div(ns * 32, threads), threads, 0, s>>>(m, ne, ns, str, binom, n_ent,
                                                                       packed_pairs, rep, pairtab);
    return cudaGetLastError();
}

cudaError_t launch_export_repl(int64_t ns, int n_ent, const uint64_t *rep, int32_t *dst, cudaStream_t s) {
    int64_t n = ns * n_ent;
    if (n <= 0) return cudaSuccess;
    k_export_repl<<<(unsigned)ceil_div(n, 256), 256, 0, s>>>(n, rep, dst);
    return cudaGetLastError();
}
