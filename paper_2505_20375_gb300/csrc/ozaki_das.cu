// Split-precision sigma on the STP-DAS layout (Results: the CI vector as category
// blocks; Methods, Eqs. sigmaL1e/sigmaL2e: the sigma build as gather, dense
// contraction E = g' D and scatter), with the contraction on the tcgen05 tensor cores,
// Ozaki style.
//
// Same scheme as the alpha/beta kernel: both operands go to fixed point with one
// exponent each, are cut into s signed base-256 digits (exact in f16), and the level
// sums S_L = sum_{i+j=L} G_i D_j of the top s levels (L >= s - 1) accumulate exactly in
// FP32 TMEM columns.  The MMA operands are turned around to fit the DAS sizes (16 and
// 17 orbitals have 136 and 153 pair rows, more than one M = 128 tile):
//   M = 128 determinants of the intermediate space per tile (A operand: digit planes
//       of D^T, produced K-chunk by K-chunk into a shared-memory ring),
//   N = n_pair rounded up to 16 (B operand: the G digit slices, resident in shared
//       memory), K = the same padded n_pair.
// s = 2 or 3 slices: s level accumulators of N columns each fit the 512 TMEM columns.
// s = 4 .. 8 (FP64 class at 6 and 7) use the two-pass form at the end of this file: a
// digit image of D, the shared bulk-copy GEMM with pair rows on M, and an exact int64 E.
// At these s every |C_int| < 2^21, so C goes to int32 fixed point; the exact level
// combination E_int (|E_int| < 2^40) is stored rounded to FP32 (24 significant bits,
// far below the 2^-8s truncation of the split), and the scatter turns each stored value
// back into the integer it holds and sums in int64:
//   sigma_I = 2^{8(s-1) - sh_G - sh_C} sum <I|E_pq|K> E[pq, K] + e_core C_I.
// E spans the intermediate space (target plus one-more-transfer categories) in chunks
// of whole categories that fit the workspace.  Addressing: a per-string replacement
// table packs the target string's pattern and local index with the sign, so the
// address of a connected determinant is a table lookup, one block offset per
// (alpha pattern, beta pattern) held in shared memory, and a multiply-add.
//
// Kernel layout (one persistent CTA per SM, 672 threads; PW = 8 or 12 producer warps as
// tuned):
//   warps 0 .. PW-1       producers: decode the tile's determinants (category, strings,
//                         local indices) once per tile, then per K-chunk gather D_int for
//                         128 determinants x 8 KCH pairs from C_int and write its s digit
//                         planes;
//   warps PW .. 19        epilogue: per TMEM lane quadrant (20 - PW) / 4 warps take its
//                         16-column chunks in turn, read the s levels, combine in int64,
//                         store E (FP32, pair-major inside each tile of 128 determinants);
//   warp 20               allocates TMEM; lane 0 issues the MMAs and the commits.
// Tiles are dealt round-robin to the CTAs of a job, so at any time the CTAs work on
// neighbouring determinants and share the rows of C they gather (L2 locality).
// Waits on mbarriers are bounded in time as in the alpha/beta kernel.
#include <math.h>
#include <stdio.h>
#include <stdlib.h>

#include <algorithm>
#include <vector>

#include "das_dev.cuh"
#include "oz_gemm.cuh"
#include "tc_ptx.cuh"

namespace {

using namespace tc;
using das_dev::find_cat;

constexpr int DZ_TILE = 128;  // determinants per tile (the MMA's M)
// Epilogue warps: the CTA keeps 21 warps (96 registers per thread), so 8 epilogue warps
// (two per TMEM lane quadrant) beside 12 producers and 12 (three per quadrant) beside 8.
__host__ __device__ constexpr int dz_epi_warps(int pw) { return 20 - pw; }
__host__ __device__ constexpr int dz_threads(int pw) { return 32 * (pw + dz_epi_warps(pw) + 1); }
constexpr int DZ_MAX_RING = 4;
constexpr int DZ_LOC_BITS = 22;  // packed replacement entry: ((pattern << 22 | local) << 1) | sign
constexpr int32_t DZ_LOC_MASK = (1 << DZ_LOC_BITS) - 1;
constexpr int DZ_MAX_JOBS = 16;
constexpr size_t DZ_SMEM_MAX = 232448 - 1024;  // dynamic shared memory (static: the job parameters)

struct DzParams {
    int64_t a0, len;  // this launch covers intermediate addresses [a0, a0 + len)
    int64_t n_det;    // target determinants (C is zero beyond)
    int64_t nla, nlb; // strings of the listed patterns (the rows of the replacement tables)
    int n_cat_int;    // categories searched when decoding an address
    int n_pat_a, n_pat_b;
    int npair, Np, KC, ring;
    int g_slice_bytes, slot_bytes, tab_off;  // shared-memory layout
    const int32_t *repA, *repB;
    const int32_t *base_tgt;  // [n_pat_a * n_pat_b]: offset of a TARGET block, else -1 (C is zero)
    const int32_t *nstr_b32;  // [n_pat_b]
    const int64_t *cat_off;
    const int32_t *cat_pa, *cat_pb;
    const int64_t *locbase_a, *locbase_b;
    const int32_t *Cint;
    const uint4 *Gimg;
    float *E;
    int *status;
    long long timeout_cycles;
    int stall_test;  // test hook: producers never signal a filled slot, so the MMA wait expires
};

struct DzGroup {
    int n_jobs;
    int cta_start[DZ_MAX_JOBS + 1];
    DzParams job[DZ_MAX_JOBS];
};

struct DzShared {
    uint64_t plane_full[DZ_MAX_RING], plane_empty[DZ_MAX_RING];
    uint64_t acc_full[2], acc_empty[2];
    uint64_t drain;
    uint32_t tmem_base;
    int abort;
};

__device__ __forceinline__ bool dz_wait(uint32_t bar, uint32_t parity, volatile int *abort, int *status,
                                        long long timeout) {
    if (mbar_test_wait(bar, parity)) return true;  // usually complete already: no clock read
    const long long t0 = clock64();
    int spins = 0;
    while (!mbar_try_wait_sleep(bar, parity)) {
        if (((++spins) & 3) == 0) {
            if (*abort) return false;
            if (clock64() - t0 > timeout) {
                *abort = 1;
                atomicExch(status, FCI_ERR_TIMEOUT);
                return false;
            }
        }
    }
    return true;
}

__device__ __forceinline__ bool dz_wait_warp(uint32_t bar, uint32_t parity, volatile int *abort, int *status,
                                             long long timeout) {
    int ok = 0;
    if ((threadIdx.x & 31) == 0) ok = dz_wait(bar, parity, abort, status, timeout) ? 1 : 0;
    return __shfl_sync(0xFFFFFFFFu, ok, 0) != 0;
}

// S: slices per operand; KCH: K-cores (8 pairs each) per ring slot, 2, 4 or 6;
// PW: producer warps (8 or 12; KCH a multiple of PW / 4).  Warps PW .. 19 run the
// epilogue (20 - PW of them, evenly over the TMEM lane quadrants), warp 20 the MMAs.
template <int S, int KCH, int PW>
__global__ void __launch_bounds__(dz_threads(PW), 1) k_oz_das(const __grid_constant__ DzGroup grp) {
    __shared__ DzParams p;
    __shared__ int cta_lo, cta_n;
    if (threadIdx.x == 0) {
        int jb = 0;
        while (jb + 1 < grp.n_jobs && (int)blockIdx.x >= grp.cta_start[jb + 1]) ++jb;
        p = grp.job[jb];
        cta_lo = grp.cta_start[jb];
        cta_n = grp.cta_start[jb + 1] - grp.cta_start[jb];
    }
    __syncthreads();
    constexpr int HG = PW / 4;            // producer threads per determinant
    constexpr int UNITS = KCH / HG;       // K-cores per producer thread per chunk
    constexpr int EW = dz_epi_warps(PW);
    static_assert(EW % 4 == 0 && PW % 4 == 0, "epilogue warps must cover the TMEM lane quadrants evenly");
    constexpr int DZ_MMA_WARP = PW + EW;
    static_assert(KCH % HG == 0, "K-chunk not divisible among the producer threads");
    extern __shared__ __align__(1024) uint8_t dz_smem_raw[];
    uint8_t *smem = (uint8_t *)(((uintptr_t)dz_smem_raw + 1023) & ~(uintptr_t)1023);
    const int Np = p.Np, KC = p.KC, RING = p.ring;
    const int nbuf = (2 * S * Np <= 512) ? 2 : 1;
    const int plane_bytes = DZ_TILE * KCH * 16;
    uint8_t *sG = smem;
    uint8_t *sRing = sG + (size_t)S * p.g_slice_bytes;
    const int npab = p.n_pat_a * p.n_pat_b;
    int32_t *sBase = (int32_t *)(smem + p.tab_off);  // [n_pat_a * n_pat_b] target block offsets
    int32_t *sNstrB = sBase + npab;                  // [n_pat_b]
    int32_t *sRowAll = sNstrB + p.n_pat_b;           // [PW][n_pat_b]: per-warp row offsets
    DzShared *sh = (DzShared *)(((uintptr_t)(sRowAll + PW * p.n_pat_b) + 15) & ~(uintptr_t)15);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

    {
        const int n16 = S * p.g_slice_bytes / 16;
        uint4 *dst = (uint4 *)sG;
        for (int i = threadIdx.x; i < n16; i += blockDim.x) dst[i] = __ldg(p.Gimg + i);
        for (int i = threadIdx.x; i < npab; i += blockDim.x) sBase[i] = __ldg(p.base_tgt + i);
        for (int i = threadIdx.x; i < p.n_pat_b; i += blockDim.x) sNstrB[i] = __ldg(p.nstr_b32 + i);
    }
    if (threadIdx.x == 0) {
        for (int r = 0; r < RING; ++r) {
            mbar_init(smem_u32(&sh->plane_full[r]), PW);
            mbar_init(smem_u32(&sh->plane_empty[r]), 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(smem_u32(&sh->acc_full[b]), 1);
            mbar_init(smem_u32(&sh->acc_empty[b]), EW);
        }
        mbar_init(smem_u32(&sh->drain), 1);
        sh->abort = 0;
        fence_barrier_init();
    }
    if (warp == DZ_MMA_WARP) {
        tmem_alloc(smem_u32(&sh->tmem_base), 512);
        tmem_relinquish();
    }
    fence_proxy_async_smem();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = sh->tmem_base;
    volatile int *abort = &sh->abort;
    const int64_t ntiles = (p.len + DZ_TILE - 1) / DZ_TILE;
    const int64_t cta = (int64_t)blockIdx.x - cta_lo;
    const int nch = KC / KCH;

    if (warp < PW) {
        // ---------------------------------------------------------------- producers
        // Thread t: determinant r = t % 128 of the tile, K-cores hg, hg + HG, ... of each
        // chunk (hg = t / 128); a warp covers 32 consecutive determinants.  Replacement
        // tables are indexed by the pattern-local string (beta entries of a warp are
        // consecutive); block offsets are -1 where C is zero (non-target categories).
        // Common case, a warp whose determinants share the alpha string (one row of a
        // block): lanes 0-7 look up the alpha moves of the unit's 8 pairs once and
        // broadcast them (alpha targets are then 32 consecutive C values), and beta
        // targets go through a per-warp table of row offsets for that alpha string.
        // Otherwise every lane resolves its own moves.  Pair-table rows beyond n_pair
        // hold -1; all loads of a unit are issued before any is used.
        const int t = threadIdx.x;
        const int r = t & (DZ_TILE - 1), hg = t >> 7;
        constexpr uint32_t bias = S == 3 ? 0x808080u : 0x8080u;
        const int npb = p.n_pat_b;
        int32_t *sRow = sRowAll + warp * npb;
        const int32_t nla = (int32_t)p.nla, nlb = (int32_t)p.nlb;
        const int32_t zero2 = (int32_t)(2 * p.n_det);  // the zero pair of the signed C values
        uint32_t q = 0, slot = 0, ph = 0;  // chunks produced, ring slot, the slot's use parity
        for (int64_t tile = cta; tile < ntiles; tile += cta_n) {
            const int64_t off = tile * DZ_TILE + r;
            const bool live = off < p.len;
            int32_t pa = 0, pb = 0, la = 0, lb = 0, ida = 0, idb = 0, nb = 1;
            if (live) {
                const int64_t addr = p.a0 + off;
                const int c = find_cat(p.cat_off, p.n_cat_int, addr);
                pa = __ldg(p.cat_pa + c);
                pb = __ldg(p.cat_pb + c);
                nb = sNstrB[pb];
                const int32_t rr = (int32_t)(addr - __ldg(p.cat_off + c));
                la = rr / nb;
                lb = rr - la * nb;
                ida = (int32_t)__ldg(p.locbase_a + pa) + la;
                idb = (int32_t)__ldg(p.locbase_b + pb) + lb;
            }
            // one alpha string across the warp?  (lanes past the end agree trivially)
            const int pa0 = __shfl_sync(0xFFFFFFFFu, pa, 0), la0 = __shfl_sync(0xFFFFFFFFu, la, 0);
            const int pb0 = __shfl_sync(0xFFFFFFFFu, pb, 0), nb0 = __shfl_sync(0xFFFFFFFFu, nb, 0);
            const int32_t ida0 = __shfl_sync(0xFFFFFFFFu, ida, 0);
            const bool live0 = __shfl_sync(0xFFFFFFFFu, live ? 1 : 0, 0) != 0;  // false: no lane is live
            const bool uni = __all_sync(0xFFFFFFFFu, !live || (pa == pa0 && la == la0 && pb == pb0));
            if (uni) {
                __syncwarp();  // every lane is done with the previous tile's table
                for (int k = lane; k < npb; k += 32) {
                    const int32_t b = sBase[pa0 * npb + k];
                    sRow[k] = b >= 0 ? b + la0 * sNstrB[k] : -1;
                }
                __syncwarp();
            }
            const int32_t *bA = sBase + pb;  // alpha moves: [pa' * npb + pb]
            const int32_t *bB = sBase + pa * npb;  // beta moves: [pa * npb + pb']
            for (int ch = 0; ch < nch; ++ch, ++q) {
                uint32_t y[UNITS][8];
#pragma unroll
                for (int u = 0; u < UNITS; ++u) {
                    const int gc = ch * KCH + hg + HG * u;
                    // signed C values: C2[2 K] = +C_K, C2[2 K + 1] = -C_K, C2[2 n_det] = 0, so a
                    // move (target K, sign bit) reads C2[2 K + sign] and an absent one reads 0
                    int32_t Ka[8], Kb[8];
                    if (uni) {
                        // lane e < 8 resolves the alpha move of pair 8 gc + e for the warp's
                        // alpha string (lane 0's), as (target row offset << 1) | sign
                        int32_t ab = -1;
                        if (lane < 8 && live0) {
                            const int32_t ea = __ldg(p.repA + (8 * gc + lane) * nla + ida0);
                            if (ea >= 0) {
                                const int32_t b = sBase[(ea >> 23) * npb + pb0];
                                ab = b >= 0 ? ((b + ((ea >> 1) & DZ_LOC_MASK) * nb0) << 1) | (ea & 1) : -1;
                            }
                        }
                        int32_t eb[8];
#pragma unroll
                        for (int e = 0; e < 8; ++e) eb[e] = live ? __ldg(p.repB + (8 * gc + e) * nlb + idb) : -1;
#pragma unroll
                        for (int e = 0; e < 8; ++e) {
                            const int32_t a = __shfl_sync(0xFFFFFFFFu, ab, e);
                            Ka[e] = (a >= 0 && live) ? a + 2 * lb : zero2;
                            const int32_t rb = sRow[max(eb[e] >> 23, 0)];
                            Kb[e] = (eb[e] >= 0 && rb >= 0) ? 2 * rb + (eb[e] & 0x7FFFFF) : zero2;
                        }
                    } else {
                        int32_t ea[8], eb[8];
#pragma unroll
                        for (int e = 0; e < 8; ++e) {
                            ea[e] = live ? __ldg(p.repA + (8 * gc + e) * nla + ida) : -1;
                            eb[e] = live ? __ldg(p.repB + (8 * gc + e) * nlb + idb) : -1;
                        }
#pragma unroll
                        for (int e = 0; e < 8; ++e) {
                            const int32_t pat_b = max(eb[e] >> 23, 0);
                            const int32_t ba = bA[max(ea[e] >> 23, 0) * npb];
                            const int32_t bb = bB[pat_b];
                            Ka[e] = (ea[e] >= 0 && ba >= 0) ? 2 * (ba + ((ea[e] >> 1) & DZ_LOC_MASK) * nb + lb) + (ea[e] & 1)
                                                            : zero2;
                            Kb[e] = (eb[e] >= 0 && bb >= 0) ? 2 * (bb + la * sNstrB[pat_b]) + (eb[e] & 0x7FFFFF) : zero2;
                        }
                    }
#pragma unroll
                    for (int e = 0; e < 8; ++e)
                        y[u][e] = (uint32_t)(__ldg(p.Cint + Ka[e]) + __ldg(p.Cint + Kb[e])) + bias;
                }
                if (q >= (uint32_t)RING && !dz_wait_warp(smem_u32(&sh->plane_empty[slot]), ph ^ 1, abort, p.status,
                                                         p.timeout_cycles))
                    goto producer_done;
                {
                    uint8_t *sl = sRing + (size_t)slot * p.slot_bytes;
#pragma unroll
                    for (int j = 0; j < S; ++j) {
                        const uint32_t sel = (uint32_t)j | ((4u + (uint32_t)j) << 8);
#pragma unroll
                        for (int u = 0; u < UNITS; ++u) {
                            const int c = hg + HG * u;
                            uint32_t w[4];
#pragma unroll
                            for (int e = 0; e < 8; e += 2) w[e / 2] = digits_f16x2(y[u][e], y[u][e + 1], sel);
                            const uint32_t o = (uint32_t)(((r >> 3) * KCH + c) * 128 + (r & 7) * 16);
                            *(uint4 *)(sl + j * plane_bytes + o) = make_uint4(w[0], w[1], w[2], w[3]);
                        }
                    }
                }
                fence_proxy_async_smem();
                __syncwarp();
                if (lane == 0 && !p.stall_test) mbar_arrive(smem_u32(&sh->plane_full[slot]));
                if (++slot == (uint32_t)RING) {
                    slot = 0;
                    ph ^= 1;
                }
            }
        }
    producer_done:;
    } else if (warp < DZ_MMA_WARP) {
        // ---------------------------------------------------------------- epilogue
        const int ew = warp - PW;
        const int qd = warp & 3;  // the TMEM lane quadrant this warp may access
        const int part = ew >> 2;  // the warps of a quadrant take its 16-column chunks in turn
        const int nck = Np / 16;
        const int row = 32 * qd + lane;  // determinant within the tile
        uint32_t tau = 0;
        for (int64_t tile = cta; tile < ntiles; tile += cta_n, ++tau) {
            const int buf = nbuf == 2 ? (int)(tau & 1) : 0;
            const uint32_t par = nbuf == 2 ? (tau >> 1) & 1 : tau & 1;
            if (!dz_wait_warp(smem_u32(&sh->acc_full[buf]), par, abort, p.status, p.timeout_cycles)) break;
            tc_fence_after();
            const uint32_t tl = tmem + ((uint32_t)(32 * qd) << 16) + (uint32_t)(buf * S * Np);
            float *Et = p.E + tile * ((int64_t)p.npair * DZ_TILE) + row;
#pragma unroll 1
            for (int ck = part; ck < nck; ck += EW / 4) {
                int64_t acc[16];
#pragma unroll
                for (int c = 0; c < 16; ++c) acc[c] = 0;
                uint32_t vs[S][16];  // all levels of the chunk in flight, one wait
#pragma unroll
                for (int l = 0; l < S; ++l) tmem_ld16(tl + (uint32_t)(l * Np + 16 * ck), vs[l]);
                tmem_ld_wait();
#pragma unroll
                for (int l = 0; l < S; ++l) {
                    tmem_regs_ready(vs[l]);
#pragma unroll
                    for (int c = 0; c < 16; ++c)
                        acc[c] += (int64_t)__float2int_rn(__uint_as_float(vs[l][c])) * ((int64_t)1 << (8 * l));
                }
                // E = acc rounded to FP32 (|acc| < 2^40): acc = hi 2^16 + lo with |hi| < 2^24
                // and 0 <= lo < 2^16 both exact in FP32, so one fused multiply-add rounds
                // hi 2^16 + lo exactly as a direct int64 -> FP32 conversion would, with
                // 32-bit conversions only
#pragma unroll
                for (int c = 0; c < 16; ++c) {
                    const int pp = 16 * ck + c;
                    const float hi = __int2float_rn((int32_t)(acc[c] >> 16));
                    const float lo = __int2float_rn((int32_t)(acc[c] & 0xFFFF));
                    if (pp < p.npair) __stcs(Et + (int64_t)pp * DZ_TILE, __fmaf_rn(hi, 65536.0f, lo));
                }
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(smem_u32(&sh->acc_empty[buf]));
        }
    } else if (lane == 0) {
        // ---------------------------------------------------------------- MMA issuer
        const uint32_t idesc = idesc_f16(DZ_TILE, Np);
        uint64_t bdesc[S];
#pragma unroll
        for (int i = 0; i < S; ++i)
            bdesc[i] = smem_desc(smem_u32(sG) + (uint32_t)(i * p.g_slice_bytes), 128, (uint32_t)(KC * 128));
        const uint64_t adesc0 = smem_desc(smem_u32(sRing), 128, (uint32_t)(KCH * 128));
        const uint32_t slot_step = (uint32_t)(p.slot_bytes >> 4), plane_step = (uint32_t)(plane_bytes >> 4);
        uint32_t slot = 0, ph = 0, tau = 0;  // ring slot, its use parity, tile counter
        bool issued = false;
        for (int64_t tile = cta; tile < ntiles; tile += cta_n, ++tau) {
            const int buf = nbuf == 2 ? (int)(tau & 1) : 0;
            if (tau >= (uint32_t)nbuf) {
                const uint32_t par = nbuf == 2 ? ((tau >> 1) - 1) & 1 : (tau - 1) & 1;
                if (!dz_wait(smem_u32(&sh->acc_empty[buf]), par, abort, p.status, p.timeout_cycles)) break;
            }
            tc_fence_after();
            const uint32_t dbase = tmem + (uint32_t)(buf * S * Np);
            bool ok = true;
            for (int ch = 0; ch < nch; ++ch) {
                if (!dz_wait(smem_u32(&sh->plane_full[slot]), ph, abort, p.status, p.timeout_cycles)) {
                    ok = false;
                    break;
                }
                tc_fence_after();
                const uint64_t a0 = adesc0 + (uint64_t)(slot * slot_step);
#pragma unroll
                for (int kk = 0; kk < KCH / 2; ++kk) {
                    const uint32_t koff = (uint32_t)((ch * (KCH / 2) + kk) * 16);
#pragma unroll
                    for (int j = S - 1; j >= 0; --j) {
                        const uint64_t a = a0 + (uint64_t)(j * plane_step + kk * 16);
                        const uint32_t acc_in = (ch != 0 || kk != 0 || j != S - 1) ? 1u : 0u;
#pragma unroll
                        for (int i = S - 1 - j; i < S; ++i)
                            mma_f16(dbase + (uint32_t)((i + j - (S - 1)) * Np), a, bdesc[i] + koff, idesc, acc_in);
                    }
                }
                issued = true;
                mma_commit(smem_u32(&sh->plane_empty[slot]));
                if (++slot == (uint32_t)RING) {
                    slot = 0;
                    ph ^= 1;
                }
            }
            if (!ok) break;
            mma_commit(smem_u32(&sh->acc_full[buf]));
        }
        if (issued) {
            // every MMA issued must complete before TMEM is freed: a first bounded wait,
            // and a second one if the first expires (FCI_ERR_TIMEOUT recorded)
            mma_commit(smem_u32(&sh->drain));
            for (int pass = 0; pass < 2; ++pass) {
                const long long t0 = clock64();
                bool done = true;
                while (!mbar_try_wait(smem_u32(&sh->drain), 0)) {
                    if (clock64() - t0 > p.timeout_cycles) {
                        atomicExch(p.status, FCI_ERR_TIMEOUT);
                        done = false;
                        break;
                    }
                }
                if (done) break;
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == DZ_MMA_WARP) tmem_dealloc(tmem, 512);
}

// ------------------------------------------------------------- helper kernels

// Packed replacement table of one spin, rows = pair index, columns = the strings of the
// listed patterns in pattern-local order (pattern by pattern, local index ascending):
// entry (pair row, string) of the alpha/beta pair table, (target << 1) | sign, becomes
// ((pattern(target) << 22 | local(target)) << 1) | sign, or -1 when there is no
// replacement or the target's pattern is outside the layout (more than max_transfer + 1
// electrons moved).
__global__ void k_dz_rep(const int32_t *__restrict__ pairtab, int64_t ns, int rows,
                         const int32_t *__restrict__ str_of_loc, int64_t nl, const int32_t *__restrict__ pat_of,
                         const int32_t *__restrict__ loc_of, int32_t *__restrict__ out) {
    const int64_t n = (int64_t)rows * nl;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t row = i / nl, col = i - row * nl;
        const int32_t e = pairtab[row * ns + str_of_loc[col]];
        int32_t o = -1;
        if (e >= 0) {
            const int32_t T = e >> 1, pt = pat_of[T];
            if (pt >= 0) o = (((pt << DZ_LOC_BITS) | loc_of[T]) << 1) | (e & 1);
        }
        out[i] = o;
    }
}

__global__ void k_dz_absmax(const double *__restrict__ x, int64_t n, unsigned long long *__restrict__ out) {
    unsigned long long m = 0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        m = max(m, (unsigned long long)__double_as_longlong(x[i]) & 0x7FFFFFFFFFFFFFFFull);
    for (int o = 16; o; o >>= 1) m = max(m, __shfl_xor_sync(0xFFFFFFFFu, m, o));
    if ((threadIdx.x & 31) == 0 && m) atomicMax(out, m);
}

// C_int = round(C 2^{sh_C}), sh_C = 8 s - 3 - e_C with max|C| < 2^{e_C}: |C_int| < 2^{8s-3}
// (< 2^21 for s <= 3, so int32 holds it), stored as signed pairs (C_int, -C_int) per
// determinant followed by one zero pair at index n: the producers read the value of a
// move with its sign, or zero for an absent move, with one load and no arithmetic.
__global__ void k_dz_to_fixed(const double *__restrict__ C, int64_t n, int s,
                              const unsigned long long *__restrict__ maxbits, int32_t *__restrict__ Cint,
                              int *__restrict__ shC) {
    const unsigned long long mb = *maxbits;
    const int e = mb ? (int)((mb >> 52) & 0x7FF) - 1022 : 0;
    const int sh = 8 * s - 3 - e;
    if (blockIdx.x == 0 && threadIdx.x == 0) *shC = sh;
    if (blockIdx.x == 0 && threadIdx.x == 0) *(int2 *)(Cint + 2 * n) = make_int2(0, 0);
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int32_t v = (int32_t)__double2ll_rn(scalbn(C[i], sh));
        *(int2 *)(Cint + 2 * i) = make_int2(v, -v);
    }
}

struct DzScatter {
    int64_t n_det, a0, len;
    int nla, nlb;
    int n_cat, n_pat_a, n_pat_b, npair;
    const int32_t *repA, *repB;
    const int32_t *base_int;  // [n_pat_a * n_pat_b]: offset of a block of the intermediate space, else -1
    const int32_t *nstr_b32;
    const int64_t *cat_off, *locbase_a, *locbase_b;
    const int32_t *cat_pa, *cat_pb;
    const void *E;  // FP32 [tile of 128][n_pair][128] (fused form) or int64 [tile of 64][n_pair][64] (two-pass)
    const double *C;
    double e_core;
    int ushift;  // 8 L0 - sh_G (L0 = s - 1 in the fused form); the scale is 2^(ushift - sh_C)
    const int *shC, *status;
    int *sticky;  // the handle's status word (fci_sync_status)
    int mode;    // 0: single chunk (write sigma); 1: first of several; 2: middle; 3: last
    int64_t *acc;
    double *sigma;
};

// sigma_I for every target determinant: sum of <I|E_pq|K> E[pq, K] over the K of this
// chunk, in int64 (exact), then one conversion.  A warp takes 32 consecutive target
// determinants; when they share the alpha string, lanes 0-7 resolve the alpha moves of 8
// pairs at a time and broadcast them (alpha targets are 32 consecutive K), and beta
// targets use a per-warp table of row offsets.  Loads are issued 16 at a time.
// ET, LOG2T: the element type of E and the log2 of its tile width (FP32 holding an
// integer and 128 for the fused kernel, int64 and 64 for the two-pass GEMM).
template <typename ET, int LOG2T>
__global__ void __launch_bounds__(256) k_dz_scatter(const __grid_constant__ DzScatter a) {
    extern __shared__ int32_t sc_tab[];
    const int npb = a.n_pat_b, npab = a.n_pat_a * npb;
    int32_t *cb = sc_tab, *nst = sc_tab + npab, *rowAll = nst + npb;
    for (int i = threadIdx.x; i < npab; i += blockDim.x) cb[i] = __ldg(a.base_int + i);
    for (int i = threadIdx.x; i < npb; i += blockDim.x) nst[i] = __ldg(a.nstr_b32 + i);
    __syncthreads();
    const int lane = threadIdx.x & 31;
    int32_t *row = rowAll + (threadIdx.x >> 5) * npb;
    const int u = a.ushift - *a.shC;
    const bool bad = *a.status != 0;
    if (bad && blockIdx.x == 0 && threadIdx.x == 0) atomicExch(a.sticky, *a.status);  // kept for fci_sync_status
    constexpr int32_t TMASK = (1 << LOG2T) - 1;
    const ET *E = (const ET *)a.E;
    const int64_t tstride = (int64_t)a.npair << LOG2T;
    const int32_t len = (int32_t)a.len, a0 = (int32_t)a.a0;
    const int64_t nwarps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t wbase = (blockIdx.x * (int64_t)(blockDim.x >> 5) + (threadIdx.x >> 5)) * 32; wbase < a.n_det;
         wbase += nwarps * 32) {
        const int64_t I = wbase + lane;
        const bool live = I < a.n_det;
        int32_t pa = 0, pb = 0, la = 0, lb = 0, ida = 0, idb = 0, nb = 1;
        if (live) {
            const int c = find_cat(a.cat_off, a.n_cat, I);
            pa = __ldg(a.cat_pa + c);
            pb = __ldg(a.cat_pb + c);
            nb = nst[pb];
            const int32_t rr = (int32_t)(I - __ldg(a.cat_off + c));
            la = rr / nb;
            lb = rr - la * nb;
            ida = (int32_t)__ldg(a.locbase_a + pa) + la;
            idb = (int32_t)__ldg(a.locbase_b + pb) + lb;
        }
        const int pa0 = __shfl_sync(0xFFFFFFFFu, pa, 0), la0 = __shfl_sync(0xFFFFFFFFu, la, 0);
        const int pb0 = __shfl_sync(0xFFFFFFFFu, pb, 0), nb0 = __shfl_sync(0xFFFFFFFFu, nb, 0);
        const int32_t ida0 = __shfl_sync(0xFFFFFFFFu, ida, 0);
        const bool uni = __all_sync(0xFFFFFFFFu, !live || (pa == pa0 && la == la0 && pb == pb0));
        if (uni) {
            __syncwarp();
            for (int k = lane; k < npb; k += 32) {
                const int32_t b = cb[pa0 * npb + k];
                row[k] = b >= 0 ? b + la0 * nst[k] : -1;
            }
            __syncwarp();
        }
        int64_t acc = 0;
        for (int p0 = 0; p0 < a.npair; p0 += 8) {  // pair-table rows beyond n_pair hold -1
            int32_t Ka[8], Kb[8];
            uint32_t sgn = 0;
            if (uni) {
                int32_t ab = INT32_MIN;  // (K - a0) * 2 + sign; the offset may be negative
                if (lane < 8) {
                    const int32_t ea = __ldg(a.repA + (p0 + lane) * a.nla + ida0);
                    if (ea >= 0) {
                        const int32_t b = cb[(ea >> 23) * npb + pb0];
                        ab = b >= 0 ? ((b + ((ea >> 1) & DZ_LOC_MASK) * nb0 - a0) * 2) | (ea & 1) : INT32_MIN;
                    }
                }
                int32_t eb[8];
#pragma unroll
                for (int e = 0; e < 8; ++e) eb[e] = live ? __ldg(a.repB + (p0 + e) * a.nlb + idb) : -1;
#pragma unroll
                for (int e = 0; e < 8; ++e) {
                    const int32_t x = __shfl_sync(0xFFFFFFFFu, ab, e);
                    Ka[e] = x != INT32_MIN ? (x >> 1) + lb : -1;
                    sgn |= (uint32_t)(x & 1) << e;
                    const int32_t rb = eb[e] >= 0 ? row[eb[e] >> 23] : -1;
                    Kb[e] = rb >= 0 ? rb + ((eb[e] >> 1) & DZ_LOC_MASK) - a0 : -1;
                    sgn |= (uint32_t)(eb[e] & 1) << (8 + e);
                }
            } else {
#pragma unroll
                for (int e = 0; e < 8; ++e) {
                    const int32_t ea = live ? __ldg(a.repA + (p0 + e) * a.nla + ida) : -1;
                    const int32_t eb = live ? __ldg(a.repB + (p0 + e) * a.nlb + idb) : -1;
                    const int32_t ba = ea >= 0 ? cb[(ea >> 23) * npb + pb] : -1;
                    const int32_t bb = eb >= 0 ? cb[pa * npb + (eb >> 23)] : -1;
                    Ka[e] = ba >= 0 ? ba + ((ea >> 1) & DZ_LOC_MASK) * nb + lb - a0 : -1;
                    Kb[e] = bb >= 0 ? bb + la * nst[eb >> 23] + ((eb >> 1) & DZ_LOC_MASK) - a0 : -1;
                    sgn |= ((uint32_t)(ea & 1) << e) | ((uint32_t)(eb & 1) << (8 + e));
                }
            }
            ET va[8], vb[8];
#pragma unroll
            for (int e = 0; e < 8; ++e) {
                const bool oa = live && Ka[e] >= 0 && Ka[e] < len, ob = Kb[e] >= 0 && Kb[e] < len;
                const int32_t ka = oa ? Ka[e] : 0, kb = ob ? Kb[e] : 0;
                va[e] = oa ? __ldg(E + (int64_t)(ka >> LOG2T) * tstride + ((p0 + e) << LOG2T) + (ka & TMASK)) : (ET)0;
                vb[e] = ob ? __ldg(E + (int64_t)(kb >> LOG2T) * tstride + ((p0 + e) << LOG2T) + (kb & TMASK)) : (ET)0;
            }
#pragma unroll
            for (int e = 0; e < 8; ++e) {
                int64_t xa, xb;
                if constexpr (sizeof(ET) == 4) {
                    xa = __float2ll_rn(va[e]);
                    xb = __float2ll_rn(vb[e]);
                } else {
                    xa = va[e];
                    xb = vb[e];
                }
                acc += (((sgn >> e) & 1) ? -xa : xa) + (((sgn >> (8 + e)) & 1) ? -xb : xb);
            }
        }
        if (!live) continue;
        if (a.mode == 1) { a.acc[I] = acc; continue; }
        if (a.mode == 2) { a.acc[I] += acc; continue; }
        if (a.mode == 3) acc += a.acc[I];
        a.sigma[I] = bad ? __longlong_as_double(0x7FF8000000000000ll)
                         : scalbn(__ll2double_rn(acc), u) + a.e_core * a.C[I];
    }
}

inline size_t al256(size_t b) { return (b + 255) & ~(size_t)255; }

uint16_t half_bits_of_small_int(int d) {  // IEEE binary16 of an integer |d| <= 1024 (exact)
    if (d == 0) return 0;
    const uint16_t sign = d < 0 ? 0x8000 : 0;
    unsigned m = (unsigned)(d < 0 ? -d : d);
    int e = 31 - __builtin_clz(m);
    const unsigned mant = (m << (10 - e)) & 0x3FF;
    return (uint16_t)(sign | ((unsigned)(e + 15) << 10) | mant);
}

// Shared tables of the contraction kernel: target block offsets [n_pat_a * n_pat_b],
// string counts [n_pat_b], one row-offset table [n_pat_b] per producer warp (int32),
// padded to 16 bytes.
size_t dz_table_bytes(const fci_das_layout &L, int pw) {
    return (((size_t)L.n_pat_a * L.n_pat_b + (size_t)(1 + pw) * L.n_pat_b) * 4 + 15) & ~(size_t)15;
}

// Shared tables of the scatter kernel (256 threads: 8 row-offset tables).
size_t dz_scatter_table_bytes(const fci_das_layout &L) { return dz_table_bytes(L, 8); }

int64_t dz_nloc(const std::vector<int64_t> &nstr) {
    int64_t t = 0;
    for (int64_t v : nstr) t += v;
    return t;
}

struct DzGeom {
    int Np, KC, KCH, PW, ring, g_slice_bytes, slot_bytes, tab_off;
    size_t smem;
};

// Shared-memory plan for a K-chunk of kch cores and pw producer warps: G slices, the
// ring (two slots at least, up to four), the tables, the barriers.
bool dz_geom_for(const fci_context *h, int s, int kch, int pw, DzGeom &g) {
    const fci_das_layout &L = h->das;
    g.Np = h->npair_pad;
    g.KC = g.Np / 8;
    g.g_slice_bytes = g.Np * g.KC * 16;
    if (kch <= 0 || g.KC % kch || kch % (pw / 4)) return false;
    const size_t tabs = dz_table_bytes(L, pw);
    const int slot = s * DZ_TILE * kch * 16;
    const size_t fixed = 1024 + (size_t)s * g.g_slice_bytes + tabs + sizeof(DzShared) + 64;
    if (fixed + 2 * (size_t)slot > DZ_SMEM_MAX) return false;
    g.KCH = kch;
    g.PW = pw;
    g.slot_bytes = slot;
    g.ring = (int)std::min<size_t>(DZ_MAX_RING, (DZ_SMEM_MAX - fixed) / slot);
    g.tab_off = s * g.g_slice_bytes + g.ring * slot;
    g.smem = fixed + (size_t)g.ring * slot;
    return true;
}

// Kernel configurations (K-chunk cores, producer warps) that exist.
constexpr int DZ_CONFIGS[][2] = {{6, 12}, {6, 8}, {4, 8}, {2, 8}};

// The configuration of this handle: the one the tuner chose (fci_tune_sigma), else
// FCI_DZ_CONFIG="kch,pw" from the environment, else the first configuration in the
// list above that fits.
bool dz_geom(const fci_context *h, int s, DzGeom &g) {
    const fci_das_layout &L = h->das;
    int want_k = 0, want_p = 0;
    if (L.dz_tuned_slices == s) {
        want_k = L.dz_tuned_kch;
        want_p = L.dz_tuned_pw;
    } else if (const char *env = getenv("FCI_DZ_CONFIG")) {
        if (sscanf(env, "%d,%d", &want_k, &want_p) != 2) want_k = want_p = 0;
    }
    for (const auto &c : DZ_CONFIGS)
        if (c[0] == want_k && c[1] == want_p && dz_geom_for(h, s, want_k, want_p, g)) return true;
    for (const auto &c : DZ_CONFIGS)
        if (dz_geom_for(h, s, c[0], c[1], g)) return true;
    return false;
}

}  // namespace

int dz_check(fci_context *h, int s) {
    const fci_das_layout &L = h->das;
    if (h->dtype != FCI_R64) return fci_fail(h, FCI_ERR_UNSUPPORTED, "split precision is built for real integrals");
    if (s < 2 || s > 3)
        return fci_fail(h, FCI_ERR_UNSUPPORTED,
                        "the DAS split path takes 2 or 3 slices (s level accumulators of n_pair columns in TMEM); "
                        "use FCI_PREC_FP64 for the FP64 phase");
    if (s * h->npair_pad > 512)
        return fci_fail(h, FCI_ERR_UNSUPPORTED, "%d slices x %d pair columns exceed the 512 TMEM columns", s,
                        h->npair_pad);
    if (L.n_pat_a > 256 || L.n_pat_b > 256) return fci_fail(h, FCI_ERR_UNSUPPORTED, "more than 256 patterns per spin");
    if (L.n_cat_int > 32767) return fci_fail(h, FCI_ERR_UNSUPPORTED, "more than 32767 categories");
    if (L.n_det_int >= ((int64_t)1 << 30))
        return fci_fail(h, FCI_ERR_UNSUPPORTED, "the split path takes < 2^30 intermediate determinants");
    for (int64_t v : L.pat_nstr_a)
        if (v > DZ_LOC_MASK) return fci_fail(h, FCI_ERR_UNSUPPORTED, "a pattern has more than 2^22 strings");
    for (int64_t v : L.pat_nstr_b)
        if (v > DZ_LOC_MASK) return fci_fail(h, FCI_ERR_UNSUPPORTED, "a pattern has more than 2^22 strings");
    DzGeom g;
    if (!dz_geom(h, s, g)) return fci_fail(h, FCI_ERR_UNSUPPORTED, "%d slices do not fit in shared memory", s);
    return FCI_OK;
}

namespace {

// The packed replacement tables and the block-offset table (both split forms).
int dz_prepare_tables(fci_context *h, cudaStream_t st) {
    fci_das_layout &L = h->das;
    int rc = FCI_OK;
    if (!L.d_dz_rep_a) {
        const int Np = h->npair_pad;
        const int64_t nla = dz_nloc(L.pat_nstr_a), nlb = dz_nloc(L.pat_nstr_b);
        rc = fci_dev_alloc(h, (void **)&L.d_dz_rep_a, (size_t)Np * nla * 4);
        if (!rc) rc = fci_dev_alloc(h, (void **)&L.d_dz_rep_b, (size_t)Np * nlb * 4);
        if (!rc) rc = fci_dev_alloc(h, (void **)&L.d_dz_base, (size_t)(2 * L.n_pat_a * L.n_pat_b + L.n_pat_b) * 4);
        if (rc) return rc;
        k_dz_rep<<<152 * 8, 256, 0, st>>>(h->d_pair_a, h->nsa, Np, L.d_str_of_loc_a, nla, L.d_pat_of_a, L.d_loc_a,
                                          L.d_dz_rep_a);
        k_dz_rep<<<152 * 8, 256, 0, st>>>(h->d_pair_b, h->nsb, Np, L.d_str_of_loc_b, nlb, L.d_pat_of_b, L.d_loc_b,
                                          L.d_dz_rep_b);
        FCI_CUDA(h, cudaGetLastError());
        // [target block offsets | intermediate block offsets | string counts], int32
        const size_t npab = (size_t)L.n_pat_a * L.n_pat_b;
        std::vector<int32_t> tb(2 * npab + L.n_pat_b, -1);
        for (int c = 0; c < L.n_cat_int; ++c) {
            const size_t k = (size_t)L.cat_pa[c] * L.n_pat_b + L.cat_pb[c];
            if (c < L.n_cat) tb[k] = (int32_t)L.cat_off[c];
            tb[npab + k] = (int32_t)L.cat_off[c];
        }
        for (int b = 0; b < L.n_pat_b; ++b) tb[2 * npab + b] = (int32_t)L.pat_nstr_b[b];
        FCI_CUDA(h, cudaMemcpy(L.d_dz_base, tb.data(), tb.size() * 4, cudaMemcpyHostToDevice));
    }
    return rc;
}

// G digit slices (B operand: N = pair rows pq, K = pair columns rs, canonical K-major
// core matrices), the packed replacement tables and the block-offset table.
int dz_prepare(fci_context *h, int s, cudaStream_t st) {
    fci_das_layout &L = h->das;
    int rc = dz_check(h, s);
    if (!rc) rc = dz_prepare_tables(h, st);
    if (rc) return rc;
    if (L.dz_slices != s || !L.d_dz_G) {
        const int np = h->npair, Np = h->npair_pad, KC = Np / 8;
        std::vector<double> G((size_t)np * np);
        if (cudaMemcpy(G.data(), h->d_G, G.size() * 8, cudaMemcpyDeviceToHost) != cudaSuccess)
            return fci_cuda_check(h, cudaGetLastError(), "G download");
        double gmax = 0.0;
        for (double v : G) gmax = std::max(gmax, fabs(v));
        int eG = 0;
        if (gmax > 0) frexp(gmax, &eG);  // gmax < 2^eG
        const int shG = 8 * s - 2 - eG;
        const uint64_t bias = 0x8080808080808080ull >> (8 * (8 - s));
        const size_t slice = (size_t)Np * KC * 16;
        std::vector<uint16_t> img(slice / 2 * s, 0);
        for (int pq = 0; pq < Np; ++pq)
            for (int rs = 0; rs < Np; ++rs) {
                int64_t gi = 0;
                if (pq < np && rs < np) gi = llrint(ldexp(G[(size_t)pq * np + rs], shG));
                const uint64_t y = (uint64_t)gi + bias;
                const size_t off = ((size_t)(pq >> 3) * KC + (rs >> 3)) * 128 + (pq & 7) * 16 + (rs & 7) * 2;
                for (int j = 0; j < s; ++j) img[(j * slice + off) / 2] = half_bits_of_small_int((int)((y >> (8 * j)) & 0xFF) - 128);
            }
        fci_dev_free(L.d_dz_G);
        L.d_dz_G = nullptr;
        L.dz_slices = 0;
        rc = fci_dev_alloc(h, &L.d_dz_G, img.size() * 2);
        if (rc) return rc;
        FCI_CUDA(h, cudaMemcpy(L.d_dz_G, img.data(), img.size() * 2, cudaMemcpyHostToDevice));
        L.dz_slices = s;
        L.dz_shG = shG;
    }
    return FCI_OK;
}

// Intermediate-space chunk: whole categories whose E fits the cap (a single category
// larger than the cap is a chunk of its own).  FCI_DAS_CHUNK_DETS overrides the cap
// (in determinants) so tests can force several chunks on small problems.
int64_t dz_chunk_cap(const fci_context *h) {
    const char *env = getenv("FCI_DAS_CHUNK_DETS");
    if (env && atoll(env) > 0) return atoll(env);
    const int64_t cap_bytes = (int64_t)96 << 30;
    return cap_bytes / (4 * (int64_t)h->npair);
}

void dz_chunks(const fci_context *h, std::vector<std::pair<int, int>> &out, int64_t &max_len) {
    const fci_das_layout &L = h->das;
    const int64_t cap = dz_chunk_cap(h);
    out.clear();
    max_len = 0;
    int c0 = 0;
    while (c0 < L.n_cat_int) {
        int c1 = c0 + 1;
        while (c1 < L.n_cat_int && L.cat_off[c1 + 1] - L.cat_off[c0] <= cap) ++c1;
        out.push_back({c0, c1});
        max_len = std::max(max_len, L.cat_off[c1] - L.cat_off[c0]);
        c0 = c1;
    }
}

struct DzJob {
    fci_context *h;
    const double *C;
    double *sigma;
    int32_t *Cint;
    float *E;
    int64_t *acc;
    int *shC, *status;
    std::vector<std::pair<int, int>> chunks;
};

int dz_prepare_job(fci_context *h, const double *C, double *sigma, int s, void *ws, cudaStream_t st, DzJob &j) {
    int rc = dz_prepare(h, s, st);
    if (rc) return rc;
    const fci_das_layout &L = h->das;
    int64_t max_len = 0;
    dz_chunks(h, j.chunks, max_len);
    char *p = (char *)ws;
    j.h = h;
    j.C = C;
    j.sigma = sigma;
    j.Cint = (int32_t *)p;  // signed pairs (+C, -C) per determinant, then a zero pair
    p += al256((size_t)(L.n_det + 1) * 8);
    j.E = (float *)p;
    p += al256((size_t)ceil_div(max_len, DZ_TILE) * h->npair * DZ_TILE * 4);
    j.acc = nullptr;
    if (j.chunks.size() > 1) {
        j.acc = (int64_t *)p;
        p += al256((size_t)L.n_det * 8);
    }
    unsigned long long *maxbits = (unsigned long long *)p;
    j.shC = (int *)(p + 8);
    j.status = (int *)(p + 16);
    phase_scope ps(h, st, FCI_PHASE_OTHER, 2);
    FCI_CUDA(h, cudaMemsetAsync(p, 0, 256, st));
    const unsigned nb = (unsigned)std::min<int64_t>(ceil_div(L.n_det, 256), 152 * 8);
    k_dz_absmax<<<nb, 256, 0, st>>>(C, L.n_det, maxbits);
    k_dz_to_fixed<<<nb, 256, 0, st>>>(C, L.n_det, s, maxbits, j.Cint, j.shC);
    FCI_CUDA(h, cudaGetLastError());
    return FCI_OK;
}

void dz_params(const DzJob &j, int s, const DzGeom &g, int chunk, DzParams &prm) {
    const fci_context *h = j.h;
    const fci_das_layout &L = h->das;
    const int c0 = j.chunks[chunk].first, c1 = j.chunks[chunk].second;
    prm.a0 = L.cat_off[c0];
    prm.len = L.cat_off[c1] - L.cat_off[c0];
    prm.n_det = L.n_det;
    prm.nla = dz_nloc(L.pat_nstr_a);
    prm.nlb = dz_nloc(L.pat_nstr_b);
    prm.n_cat_int = L.n_cat_int;
    prm.n_pat_a = L.n_pat_a;
    prm.n_pat_b = L.n_pat_b;
    prm.npair = h->npair;
    prm.Np = g.Np;
    prm.KC = g.KC;
    prm.ring = g.ring;
    prm.g_slice_bytes = g.g_slice_bytes;
    prm.slot_bytes = g.slot_bytes;
    prm.tab_off = g.tab_off;
    prm.repA = L.d_dz_rep_a;
    prm.repB = L.d_dz_rep_b;
    prm.base_tgt = L.d_dz_base;
    prm.nstr_b32 = L.d_dz_base + 2 * (size_t)L.n_pat_a * L.n_pat_b;
    prm.cat_off = L.d_cat_off;
    prm.cat_pa = L.d_cat_pa;
    prm.cat_pb = L.d_cat_pb;
    prm.locbase_a = L.d_pat_locbase_a;
    prm.locbase_b = L.d_pat_locbase_b;
    prm.Cint = j.Cint;
    prm.Gimg = (const uint4 *)L.d_dz_G;
    prm.E = j.E;
    prm.status = j.status;
    const char *to = getenv("FCI_WAIT_TIMEOUT_MS");
    const double ms = to ? atof(to) : 2000.0;
    prm.timeout_cycles = (long long)(ms * 2.1e6);
    const char *stall = getenv("FCI_TEST_STALL_PRODUCER");
    prm.stall_test = stall ? atoi(stall) : 0;
    (void)s;
}

template <int S>
void (*dz_kernel(int kch, int pw))(const DzGroup) {
    if (kch == 6 && pw == 12) return k_oz_das<S, 6, 12>;
    if (kch == 6 && pw == 8) return k_oz_das<S, 6, 8>;
    if (kch == 4 && pw == 8) return k_oz_das<S, 4, 8>;
    if (kch == 2 && pw == 8) return k_oz_das<S, 2, 8>;
    return nullptr;
}

int dz_launch(fci_context *h, const DzGroup &grp, int s, const DzGeom &g, size_t smem, cudaStream_t st) {
    void (*kern)(const DzGroup) = s == 2 ? dz_kernel<2>(g.KCH, g.PW) : s == 3 ? dz_kernel<3>(g.KCH, g.PW) : nullptr;
    if (!kern) return fci_fail(h, FCI_ERR_UNSUPPORTED, "slice count %d, K-chunk %d, %d producer warps", s, g.KCH, g.PW);
    FCI_CUDA(h, cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    phase_scope ps(h, st, FCI_PHASE_CONTRACT, 1);
    kern<<<grp.cta_start[grp.n_jobs], dz_threads(g.PW), smem, st>>>(grp);
    FCI_CUDA(h, cudaGetLastError());
    return FCI_OK;
}

int dz_scatter(const DzJob &j, int s, int chunk, cudaStream_t st) {
    fci_context *h = j.h;
    const fci_das_layout &L = h->das;
    DzScatter a;
    const int c0 = j.chunks[chunk].first, c1 = j.chunks[chunk].second;
    const int nchunks = (int)j.chunks.size();
    a.n_det = L.n_det;
    a.nla = (int)dz_nloc(L.pat_nstr_a);
    a.nlb = (int)dz_nloc(L.pat_nstr_b);
    a.a0 = L.cat_off[c0];
    a.len = L.cat_off[c1] - L.cat_off[c0];
    a.n_cat = L.n_cat;
    a.n_pat_a = L.n_pat_a;
    a.n_pat_b = L.n_pat_b;
    a.npair = h->npair;
    a.repA = L.d_dz_rep_a;
    a.repB = L.d_dz_rep_b;
    a.base_int = L.d_dz_base + (size_t)L.n_pat_a * L.n_pat_b;
    a.nstr_b32 = L.d_dz_base + 2 * (size_t)L.n_pat_a * L.n_pat_b;
    a.cat_off = L.d_cat_off;
    a.locbase_a = L.d_pat_locbase_a;
    a.locbase_b = L.d_pat_locbase_b;
    a.cat_pa = L.d_cat_pa;
    a.cat_pb = L.d_cat_pb;
    a.E = j.E;
    a.C = j.C;
    a.e_core = h->e_core;
    a.ushift = 8 * (s - 1) - L.dz_shG;
    a.shC = j.shC;
    a.status = j.status;
    a.sticky = h->d_status;
    a.mode = nchunks == 1 ? 0 : chunk == 0 ? 1 : chunk == nchunks - 1 ? 3 : 2;
    a.acc = j.acc;
    a.sigma = j.sigma;
    const size_t smem = dz_scatter_table_bytes(L);
    if (smem > 48 * 1024)
        FCI_CUDA(h, cudaFuncSetAttribute(k_dz_scatter<float, 7>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    phase_scope ps(h, st, FCI_PHASE_SCATTER, 1);
    const unsigned nb = (unsigned)std::max<int64_t>(1, std::min<int64_t>(ceil_div(L.n_det, 256), 152 * 8));
    k_dz_scatter<float, 7><<<nb, 256, smem, st>>>(a);
    FCI_CUDA(h, cudaGetLastError());
    return FCI_OK;
}

int dz_num_sms(fci_context *h, int *nsm) {
    FCI_CUDA(h, cudaDeviceGetAttribute(nsm, cudaDevAttrMultiProcessorCount, h->device));
    return FCI_OK;
}

}  // namespace

// ------------------------------------------------------- two-pass form (s = 4 .. 8)
//
// For an FP64-class split (6 or 7 slices) the s level accumulators of the fused form do not
// fit in TMEM, and neither do its G slices in shared memory, so the contraction turns back
// to the orientation of the alpha/beta two-pass path: pair rows on M (ceil(n_pair / 128)
// M-tiles of G digits), 64 determinants on N, and the operands streamed from HBM:
//   k_dg_split   writes the digit image of D (int64 fixed point of C, gathered through the
//                packed replacement tables and the target block offsets) for a piece of
//                the intermediate space, in the B-tile layout of the bulk-copy GEMM;
//   k_oz_gemm    (8-bit digits, K-chunks of 32) sums the top s levels exactly in TMEM and
//                stores E_int (int64) [tile of 64][n_pair][64];
//   k_dz_scatter (int64 form) sums E_int exactly per target determinant.
// Every level sum stays an integer below 2^24 when s n_pair <= 1023 (n_pair nonzero terms
// of products below 2^14, s products per level), which the check enforces.  E covers up to
// a cap of the intermediate space at a time (the scatter runs once per E chunk); the digit
// image covers a smaller piece of that chunk at a time.
namespace {

constexpr int DG_KCC = 4;                      // core matrices (8 pairs) per K-chunk of the GEMM
constexpr int DG_KW = 8 * DG_KCC;              // 32 pairs per K-chunk
constexpr int DG_B_PLANE = OZG_N * DG_KW * 2;  // 4 KB: 64 determinants x 32 pairs, f16
constexpr int DG_A_PLANE = OZG_M * DG_KW * 2;  // 8 KB: 128 pair rows x 32 pairs, f16

struct DgGeom {
    int n_mt, n_kc;        // M-tiles of 128 pair rows; K-chunks of 32 pairs
    int64_t e_cap, d_cap;  // determinants per E chunk and per digit-image piece (multiples of 64)
    int n_echunks;
};

// FCI_DAS_CHUNK_DETS and FCI_DAS_IMAGE_DETS lower the two caps (in determinants) so that
// tests can force several chunks and pieces on small problems.
DgGeom dg_geom(const fci_context *h, int s) {
    const fci_das_layout &L = h->das;
    DgGeom g;
    g.n_mt = (h->npair + OZG_M - 1) / OZG_M;
    g.n_kc = (h->npair_pad + DG_KW - 1) / DG_KW;
    const int64_t all = ceil_div(std::max<int64_t>(L.n_det_int, 1), OZG_N) * OZG_N;
    int64_t e = (((int64_t)96 << 30) / (8 * (int64_t)h->npair)) / OZG_N * OZG_N;
    if (const char *env = getenv("FCI_DAS_CHUNK_DETS"))
        if (atoll(env) > 0) e = ceil_div(atoll(env), OZG_N) * OZG_N;
    g.e_cap = std::max<int64_t>(OZG_N, std::min(e, all));
    int64_t d = (((int64_t)24 << 30) / ((int64_t)g.n_kc * s * DG_B_PLANE / OZG_N)) / OZG_N * OZG_N;
    if (const char *env = getenv("FCI_DAS_IMAGE_DETS"))
        if (atoll(env) > 0) d = ceil_div(atoll(env), OZG_N) * OZG_N;
    g.d_cap = std::max<int64_t>(OZG_N, std::min(d, g.e_cap));
    g.n_echunks = (int)ceil_div(all, g.e_cap);
    return g;
}

struct DgSplit {
    int64_t a0, len;   // intermediate addresses [a0, a0 + len) of this piece
    int64_t n_nt;      // tiles of 64
    int n_kc, npair_pad, n_cat_int, n_pat_b;
    int64_t nla, nlb;
    const int32_t *repA, *repB;
    const int32_t *base_tgt;  // [n_pat_a * n_pat_b]: offset of a TARGET block, else -1 (C is zero)
    const int32_t *nstr_b32;
    const int64_t *cat_off, *locbase_a, *locbase_b;
    const int32_t *cat_pa, *cat_pb;
    const int64_t *Cint;
    uint8_t *Dimg;
};

// Digit image of D for one piece: tile nt (64 determinants) holds, per K-chunk of 32
// pairs, S f16 planes of 64 x 32 in canonical K-major core matrices.  Thread t covers
// determinant t % 64 of the tile (decoded once: category, patterns, local indices) and
// pairs 8 (t / 64) .. 8 (t / 64) + 7 of every chunk; D_int of a pair is the alpha move's
// and the beta move's signed C_int (zero where the move leaves the target space or does
// not exist; replacement-table rows past n_pair_pad count as absent).  Capped at 64
// registers for four resident blocks per SM (measured 4% faster than three at C3').
template <int S>
__global__ void __launch_bounds__(64 * DG_KCC, 4) k_dg_split(const __grid_constant__ DgSplit a) {
    constexpr uint64_t bias = 0x8080808080808080ull >> (8 * (8 - S));
    const int row = threadIdx.x & 63, cc = threadIdx.x >> 6;
    const int npb = a.n_pat_b;
    for (int64_t nt = blockIdx.x; nt < a.n_nt; nt += gridDim.x) {
        const int64_t off = nt * OZG_N + row;
        const bool live = off < a.len;
        int32_t pa = 0, pb = 0, la = 0, lb = 0, nb = 1;
        int64_t ida = 0, idb = 0;
        if (live) {
            const int64_t addr = a.a0 + off;
            const int c = find_cat(a.cat_off, a.n_cat_int, addr);
            pa = __ldg(a.cat_pa + c);
            pb = __ldg(a.cat_pb + c);
            nb = __ldg(a.nstr_b32 + pb);
            const int32_t rr = (int32_t)(addr - __ldg(a.cat_off + c));
            la = rr / nb;
            lb = rr - la * nb;
            ida = __ldg(a.locbase_a + pa) + la;
            idb = __ldg(a.locbase_b + pb) + lb;
        }
        uint8_t *tile = a.Dimg + (size_t)nt * a.n_kc * S * DG_B_PLANE + ((row >> 3) * DG_KCC + cc) * 128 + (row & 7) * 16;
#pragma unroll 1
        for (int kc = 0; kc < a.n_kc; ++kc) {
            const int rs0 = kc * DG_KW + cc * 8;
            int32_t ea[8], eb[8];
#pragma unroll
            for (int e = 0; e < 8; ++e) {
                const bool ok = live && rs0 + e < a.npair_pad;
                ea[e] = ok ? __ldg(a.repA + (int64_t)(rs0 + e) * a.nla + ida) : -1;
                eb[e] = ok ? __ldg(a.repB + (int64_t)(rs0 + e) * a.nlb + idb) : -1;
            }
            int32_t Ka[8], Kb[8];
#pragma unroll
            for (int e = 0; e < 8; ++e) {
                const int32_t ba = ea[e] >= 0 ? __ldg(a.base_tgt + (ea[e] >> 23) * npb + pb) : -1;
                const int32_t bb = eb[e] >= 0 ? __ldg(a.base_tgt + pa * npb + (eb[e] >> 23)) : -1;
                Ka[e] = ba >= 0 ? ba + ((ea[e] >> 1) & DZ_LOC_MASK) * nb + lb : -1;
                Kb[e] = bb >= 0 ? bb + la * __ldg(a.nstr_b32 + (eb[e] >> 23)) + ((eb[e] >> 1) & DZ_LOC_MASK) : -1;
            }
            uint32_t ylo[8], yhi[8];
#pragma unroll
            for (int e = 0; e < 8; ++e) {
                const int64_t xa = Ka[e] >= 0 ? __ldg(a.Cint + Ka[e]) : 0;
                const int64_t xb = Kb[e] >= 0 ? __ldg(a.Cint + Kb[e]) : 0;
                const int64_t v = ((ea[e] & 1) ? -xa : xa) + ((eb[e] & 1) ? -xb : xb);
                const uint64_t y = (uint64_t)v + bias;
                ylo[e] = (uint32_t)y;
                yhi[e] = (uint32_t)(y >> 32);
            }
            uint8_t *base = tile + (size_t)kc * S * DG_B_PLANE;
#pragma unroll
            for (int j = 0; j < S; ++j) {
                const uint32_t bj = (uint32_t)(j & 3), sel = bj | ((4u + bj) << 8);
                uint32_t w[4];
#pragma unroll
                for (int e = 0; e < 8; e += 2)
                    w[e / 2] = j < 4 ? digits_f16x2(ylo[e], ylo[e + 1], sel) : digits_f16x2(yhi[e], yhi[e + 1], sel);
                __stcs((uint4 *)(base + j * DG_B_PLANE), make_uint4(w[0], w[1], w[2], w[3]));
            }
        }
    }
}

// G digit slices in the A-tile layout of the bulk-copy GEMM: [M-tile][K-chunk][plane][128 x 32].
int dg_prepare_G(fci_context *h, int s) {
    fci_das_layout &L = h->das;
    if (L.dg_slices == s && L.d_dg_G) return FCI_OK;
    const DgGeom g = dg_geom(h, s);
    const int np = h->npair;
    std::vector<double> G((size_t)np * np);
    if (cudaMemcpy(G.data(), h->d_G, G.size() * 8, cudaMemcpyDeviceToHost) != cudaSuccess)
        return fci_cuda_check(h, cudaGetLastError(), "G download");
    double gmax = 0.0;
    for (double v : G) gmax = std::max(gmax, fabs(v));
    int eG = 0;
    if (gmax > 0) frexp(gmax, &eG);  // gmax < 2^eG
    const int shG = 8 * s - 2 - eG;
    const uint64_t bias = 0x8080808080808080ull >> (8 * (8 - s));
    const size_t stage = (size_t)s * DG_A_PLANE;
    std::vector<uint16_t> img((size_t)g.n_mt * g.n_kc * stage / 2, 0);
    for (int m = 0; m < g.n_mt * OZG_M; ++m)
        for (int k = 0; k < g.n_kc * DG_KW; ++k) {
            int64_t gi = 0;
            if (m < np && k < np) gi = llrint(ldexp(G[(size_t)m * np + k], shG));
            const uint64_t y = (uint64_t)gi + bias;
            const int mt = m / OZG_M, mm = m % OZG_M, kc = k / DG_KW, kk = k % DG_KW;
            const size_t off = ((size_t)mt * g.n_kc + kc) * stage + ((mm >> 3) * DG_KCC + (kk >> 3)) * 128 + (mm & 7) * 16 +
                               (kk & 7) * 2;
            for (int j = 0; j < s; ++j)
                img[(off + (size_t)j * DG_A_PLANE) / 2] = half_bits_of_small_int((int)((y >> (8 * j)) & 0xFF) - 128);
        }
    fci_dev_free(L.d_dg_G);
    L.d_dg_G = nullptr;
    L.dg_slices = 0;
    int rc = fci_dev_alloc(h, &L.d_dg_G, img.size() * 2);
    if (rc) return rc;
    FCI_CUDA(h, cudaMemcpy(L.d_dg_G, img.data(), img.size() * 2, cudaMemcpyHostToDevice));
    L.dg_slices = s;
    L.dg_shG = shG;
    return FCI_OK;
}

}  // namespace

int dg_check(fci_context *h, int s) {
    const fci_das_layout &L = h->das;
    if (h->dtype != FCI_R64) return fci_fail(h, FCI_ERR_UNSUPPORTED, "split precision is built for real integrals");
    if (s < 4 || s > 8) return fci_fail(h, FCI_ERR_UNSUPPORTED, "the DAS two-pass split takes 4 to 8 slices");
    if (s * h->npair > 1023)
        return fci_fail(h, FCI_ERR_UNSUPPORTED, "%d slices x %d pairs: level sums could exceed 2^24", s, h->npair);
    if (L.n_pat_a > 256 || L.n_pat_b > 256) return fci_fail(h, FCI_ERR_UNSUPPORTED, "more than 256 patterns per spin");
    if (L.n_det_int >= ((int64_t)1 << 30))
        return fci_fail(h, FCI_ERR_UNSUPPORTED, "the split path takes < 2^30 intermediate determinants");
    for (int64_t v : L.pat_nstr_a)
        if (v > DZ_LOC_MASK) return fci_fail(h, FCI_ERR_UNSUPPORTED, "a pattern has more than 2^22 strings");
    for (int64_t v : L.pat_nstr_b)
        if (v > DZ_LOC_MASK) return fci_fail(h, FCI_ERR_UNSUPPORTED, "a pattern has more than 2^22 strings");
    if (!oz_gemm_ring(s, DG_KCC, 0)) return fci_fail(h, FCI_ERR_UNSUPPORTED, "%d slices do not fit the GEMM pipeline", s);
    return FCI_OK;
}

int das_split_check(fci_context *h, int s) { return s <= 3 ? dz_check(h, s) : dg_check(h, s); }

size_t dg_workspace_bytes(const fci_context *h, int s) {
    const DgGeom g = dg_geom(h, std::max(s, 4));
    size_t b = al256((size_t)h->das.n_det * 8) + al256((size_t)(g.d_cap / OZG_N) * g.n_kc * std::max(s, 4) * DG_B_PLANE) +
               al256((size_t)g.e_cap * h->npair * 8);
    if (g.n_echunks > 1) b += al256((size_t)h->das.n_det * 8);
    return b + 256;
}

int dg_sigma(fci_context *h, const double *C, double *sigma, int s, void *ws, cudaStream_t st) {
    int rc = dg_check(h, s);
    if (!rc) rc = dz_prepare_tables(h, st);
    if (!rc) rc = dg_prepare_G(h, s);
    if (rc) return rc;
    const fci_das_layout &L = h->das;
    const DgGeom g = dg_geom(h, s);
    char *p = (char *)ws;
    int64_t *Cint = (int64_t *)p;
    p += al256((size_t)L.n_det * 8);
    uint8_t *Dimg = (uint8_t *)p;
    p += al256((size_t)(g.d_cap / OZG_N) * g.n_kc * s * DG_B_PLANE);
    int64_t *E = (int64_t *)p;
    p += al256((size_t)g.e_cap * h->npair * 8);
    int64_t *acc = nullptr;
    if (g.n_echunks > 1) {
        acc = (int64_t *)p;
        p += al256((size_t)L.n_det * 8);
    }
    unsigned long long *maxbits = (unsigned long long *)p;
    int *shC = (int *)(p + 8), *status = (int *)(p + 16);
    {
        phase_scope ps(h, st, FCI_PHASE_OTHER, 2);
        FCI_CUDA(h, cudaMemsetAsync(p, 0, 256, st));
        FCI_CUDA(h, launch_to_fixed64(C, L.n_det, s, maxbits, Cint, shC, st));
    }
    const size_t npab = (size_t)L.n_pat_a * L.n_pat_b;
    DgSplit sp;
    sp.n_kc = g.n_kc;
    sp.npair_pad = h->npair_pad;
    sp.n_cat_int = L.n_cat_int;
    sp.n_pat_b = L.n_pat_b;
    sp.nla = dz_nloc(L.pat_nstr_a);
    sp.nlb = dz_nloc(L.pat_nstr_b);
    sp.repA = L.d_dz_rep_a;
    sp.repB = L.d_dz_rep_b;
    sp.base_tgt = L.d_dz_base;
    sp.nstr_b32 = L.d_dz_base + 2 * npab;
    sp.cat_off = L.d_cat_off;
    sp.locbase_a = L.d_pat_locbase_a;
    sp.locbase_b = L.d_pat_locbase_b;
    sp.cat_pa = L.d_cat_pa;
    sp.cat_pb = L.d_cat_pb;
    sp.Cint = Cint;
    sp.Dimg = Dimg;
    for (int ec = 0; ec < g.n_echunks; ++ec) {
        const int64_t e0 = (int64_t)ec * g.e_cap, elen = std::min(g.e_cap, L.n_det_int - e0);
        for (int64_t d0 = 0; d0 < elen; d0 += g.d_cap) {
            sp.a0 = e0 + d0;
            sp.len = std::min(g.d_cap, elen - d0);
            sp.n_nt = ceil_div(sp.len, OZG_N);
            {
                phase_scope ps(h, st, FCI_PHASE_GATHER, 1);
                const unsigned gb = (unsigned)std::max<int64_t>(1, std::min<int64_t>(sp.n_nt, 152 * 16));
                switch (s) {
                    case 4: k_dg_split<4><<<gb, 64 * DG_KCC, 0, st>>>(sp); break;
                    case 5: k_dg_split<5><<<gb, 64 * DG_KCC, 0, st>>>(sp); break;
                    case 6: k_dg_split<6><<<gb, 64 * DG_KCC, 0, st>>>(sp); break;
                    case 7: k_dg_split<7><<<gb, 64 * DG_KCC, 0, st>>>(sp); break;
                    default: k_dg_split<8><<<gb, 64 * DG_KCC, 0, st>>>(sp); break;
                }
                FCI_CUDA(h, cudaGetLastError());
            }
            oz_gemm_args a;
            a.n_mt = g.n_mt;
            a.n_kc = g.n_kc;
            a.M_pad = h->npair;  // E row stride: the n_pair rows of each tile, no padding
            a.M_real = h->npair;
            a.n_nt = sp.n_nt;
            a.Gimg = L.d_dg_G;
            a.Dimg = Dimg;
            a.E = E + (size_t)(d0 / OZG_N) * h->npair * OZG_N;
            a.status = status;
            if ((rc = oz_gemm_launch(h, s, 8, DG_KCC, false, a, st))) return rc;
        }
        DzScatter sc;
        sc.n_det = L.n_det;
        sc.nla = (int)sp.nla;
        sc.nlb = (int)sp.nlb;
        sc.a0 = e0;
        sc.len = elen;
        sc.n_cat = L.n_cat;
        sc.n_pat_a = L.n_pat_a;
        sc.n_pat_b = L.n_pat_b;
        sc.npair = h->npair;
        sc.repA = L.d_dz_rep_a;
        sc.repB = L.d_dz_rep_b;
        sc.base_int = L.d_dz_base + npab;
        sc.nstr_b32 = L.d_dz_base + 2 * npab;
        sc.cat_off = L.d_cat_off;
        sc.locbase_a = L.d_pat_locbase_a;
        sc.locbase_b = L.d_pat_locbase_b;
        sc.cat_pa = L.d_cat_pa;
        sc.cat_pb = L.d_cat_pb;
        sc.E = E;
        sc.C = C;
        sc.e_core = h->e_core;
        sc.ushift = 8 * oz_gemm_L0(s, 8) - L.dg_shG;
        sc.shC = shC;
        sc.status = status;
        sc.sticky = h->d_status;
        sc.mode = g.n_echunks == 1 ? 0 : ec == 0 ? 1 : ec == g.n_echunks - 1 ? 3 : 2;
        sc.acc = acc;
        sc.sigma = sigma;
        const size_t smem = dz_scatter_table_bytes(L);
        if (smem > 48 * 1024)
            FCI_CUDA(h, cudaFuncSetAttribute(k_dz_scatter<int64_t, 6>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem));
        phase_scope ps(h, st, FCI_PHASE_SCATTER, 1);
        const unsigned nb = (unsigned)std::max<int64_t>(1, std::min<int64_t>(ceil_div(L.n_det, 256), 152 * 8));
        k_dz_scatter<int64_t, 6><<<nb, 256, smem, st>>>(sc);
        FCI_CUDA(h, cudaGetLastError());
    }
    return FCI_OK;
}

void dz_free(fci_das_layout &L) {
    fci_dev_free(L.d_dz_rep_a);
    fci_dev_free(L.d_dz_rep_b);
    fci_dev_free(L.d_dz_base);
    fci_dev_free(L.d_dz_G);
    fci_dev_free(L.d_dg_G);
    L.d_dz_rep_a = L.d_dz_rep_b = nullptr;
    L.d_dz_base = nullptr;
    L.d_dz_G = nullptr;
    L.d_dg_G = nullptr;
    L.dz_slices = 0;
    L.dg_slices = 0;
}

size_t dz_workspace_bytes(const fci_context *h, int s) {
    if (s >= 4) return dg_workspace_bytes(h, s);
    std::vector<std::pair<int, int>> ch;
    int64_t max_len = 0;
    dz_chunks(h, ch, max_len);
    size_t b = al256((size_t)(h->das.n_det + 1) * 8) + al256((size_t)ceil_div(max_len, DZ_TILE) * h->npair * DZ_TILE * 4);
    if (ch.size() > 1) b += al256((size_t)h->das.n_det * 8);
    return b + 256;
}

int dz_sigma(fci_context *h, const double *C, double *sigma, int s, void *ws, size_t ws_bytes, cudaStream_t st) {
    if (s >= 4) return dg_sigma(h, C, sigma, s, ws, st);
    (void)ws_bytes;
    DzJob j;
    int rc = dz_prepare_job(h, C, sigma, s, ws, st, j);
    if (rc) return rc;
    DzGeom g;
    dz_geom(h, s, g);
    int nsm = 0;
    if ((rc = dz_num_sms(h, &nsm))) return rc;
    for (int c = 0; c < (int)j.chunks.size(); ++c) {
        DzGroup grp;
        dz_params(j, s, g, c, grp.job[0]);
        grp.n_jobs = 1;
        grp.cta_start[0] = 0;
        grp.cta_start[1] = (int)std::max<int64_t>(1, std::min<int64_t>(nsm, ceil_div(grp.job[0].len, DZ_TILE)));
        if ((rc = dz_launch(h, grp, s, g, g.smem, st))) return rc;
        if ((rc = dz_scatter(j, s, c, st))) return rc;
    }
    return FCI_OK;
}

// Several DAS problems with the same slice count and shared-memory plan in one
// persistent contraction launch (CTAs in proportion to tiles, at least one per job);
// problems whose intermediate space takes several chunks run on their own.
int dz_sigma_group(fci_context *const *hs, const double *const *Cs, double *const *sigmas, void *const *wss, int n,
                   int s, cudaStream_t st) {
    std::vector<int> single;
    for (int i = 0; i < n; ++i) {
        std::vector<std::pair<int, int>> ch;
        int64_t ml = 0;
        int rc = dz_check(hs[i], s);
        if (rc) return rc;
        dz_chunks(hs[i], ch, ml);
        if (ch.size() > 1) {
            if ((rc = dz_sigma(hs[i], Cs[i], sigmas[i], s, wss[i], 0, st))) return rc;
        } else {
            single.push_back(i);
        }
    }
    int nsm = 0;
    if (single.empty()) return FCI_OK;
    int rc = dz_num_sms(hs[single[0]], &nsm);
    if (rc) return rc;
    std::vector<char> done(single.size(), 0);
    for (size_t a = 0; a < single.size(); ++a) {
        if (done[a]) continue;
        DzGeom ga;
        dz_geom(hs[single[a]], s, ga);
        // jobs sharing the K-chunk width (the kernel's template argument)
        std::vector<int> grp_idx;
        for (size_t b = a; b < single.size() && (int)grp_idx.size() < std::min(DZ_MAX_JOBS, nsm); ++b) {
            if (done[b]) continue;
            DzGeom gb;
            dz_geom(hs[single[b]], s, gb);
            if (gb.KCH != ga.KCH || gb.PW != ga.PW) continue;
            grp_idx.push_back((int)b);
            done[b] = 1;
        }
        const int m = (int)grp_idx.size();
        std::vector<DzJob> jobs(m);
        DzGroup grp;
        size_t smem = 0;
        int64_t tiles[DZ_MAX_JOBS], total = 0;
        for (int k = 0; k < m; ++k) {
            const int i = single[grp_idx[k]];
            if ((rc = dz_prepare_job(hs[i], Cs[i], sigmas[i], s, wss[i], st, jobs[k]))) return rc;
            DzGeom g;
            dz_geom(hs[i], s, g);
            dz_params(jobs[k], s, g, 0, grp.job[k]);
            smem = std::max(smem, g.smem);
            tiles[k] = std::max<int64_t>(1, ceil_div(grp.job[k].len, DZ_TILE));
            total += tiles[k];
        }
        int ctas[DZ_MAX_JOBS], used = 0;
        for (int k = 0; k < m; ++k) {
            ctas[k] = (int)std::max<int64_t>(1, std::min<int64_t>(tiles[k], (int64_t)(nsm - m) * tiles[k] / total + 1));
            used += ctas[k];
        }
        while (used > nsm) {
            int kmax = 0;
            for (int k = 1; k < m; ++k) if (ctas[k] > ctas[kmax]) kmax = k;
            if (ctas[kmax] <= 1) break;
            --ctas[kmax];
            --used;
        }
        grp.n_jobs = m;
        grp.cta_start[0] = 0;
        for (int k = 0; k < m; ++k) grp.cta_start[k + 1] = grp.cta_start[k] + ctas[k];
        if ((rc = dz_launch(hs[single[grp_idx[0]]], grp, s, ga, smem, st))) return rc;
        for (int k = 0; k < m; ++k)
            if ((rc = dz_scatter(jobs[k], s, 0, st))) return rc;
    }
    return FCI_OK;
}

int dz_tune_candidates(const fci_context *h, int s, int *kch, int *pw, int max) {
    int n = 0;
    DzGeom g;
    for (const auto &c : DZ_CONFIGS)
        if (n < max && dz_geom_for(h, s, c[0], c[1], g)) {
            kch[n] = c[0];
            pw[n] = c[1];
            ++n;
        }
    return n;
}

void dz_set_config(fci_context *h, int s, int kch, int pw) {
    fci_das_layout &L = h->das;
    L.dz_tuned_slices = kch ? s : 0;
    L.dz_tuned_kch = kch;
    L.dz_tuned_pw = pw;
}
