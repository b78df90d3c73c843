// Split-precision contraction E = G D on the 5th-generation tensor cores (tcgen05),
// Ozaki style, for alpha/beta strings with real pair-packed integrals.
//
// Both operands go to fixed point with one exponent each (C and hence D by
// 2^{sh_C}, G by 2^{sh_G}) and are cut into s signed base-256 digits in [-128, 127]:
//   X_int = sum_{j<s} x_j 256^j.
// Digits are exact in f16 (the tensor rate of f16 and bf16 is the same; f16 makes the
// digit-to-float conversion two integer instructions and one packed subtraction per two
// digits), products of two digits are below 2^14, and every partial sum of the MMA stays
// an integer below 2^24, so the FP32 accumulation in TMEM is exact.
// The product is regrouped by significance level L = i + j of the digit pair; only the
// top s levels (L >= s - 1) are formed (the usual triangular truncation), each into its
// own TMEM accumulator:
//   S_L = sum_{i+j=L} G_i D_j,     G_int D_int ~ sum_L S_L 256^L.
// The epilogue turns the exact level sums into one int64 per element (levels below L0
// rounded away, L0 = max(s-1, 2s-6) keeps |E_int| < 2^54) and writes E_int; the scatter
// sums E_int values exactly in int64 and converts once:
//   sigma_I = 2^{8 L0 - sh_G - sh_C} sum <I|E_pq|K> E_int[pq, K] + e_core C_I.
// (Methods, Eqs. sigmaL/sigmaL2e: E = g' D is the dense contraction of the sigma build.)
//
// Kernel layout (one persistent CTA per SM, 512 threads, one job per CTA; a grouped
// launch shares the CTAs among several sigma builds in proportion to their tiles):
//   warps 0-6  producers: gather D_int for a tile of 64 determinants from the fixed-point
//              C and the pair tables, keep it in registers, and write its s digit planes
//              (f16, canonical K-major core-matrix layout) into a 2- or 3-slot shared ring;
//   warps 7-14 epilogue: read the s level accumulators of a tile from TMEM (two warps per
//              32-lane quadrant, 32 columns each, in chunks of 16), combine them in int64,
//              store E_int in a tile-major layout;
//   warp 15    allocates TMEM; lane 0 issues tcgen05.mma (M = 128 pair rows of G digits
//              resident in shared memory, N = 64 determinants, K = 16 per instruction) and
//              tcgen05.commit to the mbarriers that hand buffers between the roles.
// Level accumulators take s x 64 TMEM columns, double-buffered when 2 s x 64 <= 512.
// Every wait on an mbarrier is bounded in time; on expiry the kernel records
// FCI_ERR_TIMEOUT in a device status word, stops issuing work, drains the MMAs it issued,
// frees TMEM and returns.
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include <cuda_fp16.h>

#include "fci_internal.h"
#include "oz_gemm.cuh"
#include "tc_ptx.cuh"

namespace {

using namespace tc;

constexpr int OZ_PRODUCER_WARPS = 7;  // 16 warps in all: up to 128 registers per thread
constexpr int OZ_EPILOGUE_WARPS = 8;  // two per TMEM lane quadrant, 16 columns each
constexpr int OZ_MMA_WARP = OZ_PRODUCER_WARPS + OZ_EPILOGUE_WARPS;
constexpr int OZ_THREADS = 32 * (OZ_MMA_WARP + 1);  // 512
constexpr int OZ_MAX_RING = 3;  // digit-plane slots (2 or 3, whatever shared memory allows)
// Determinants per tile (the MMA's N): 64 by default, or 32 (chosen per slice count by
// the tuner).  A tcgen05.mma costs at least ~45 cycles to issue whatever its size, so
// an M=128 N=32 K=16 MMA reaches only about a third of the tensor rate, but at N=32 the
// level accumulators are double-buffered up to s = 8; N=64 is the largest tile for which
// the s level accumulators fit in TMEM (s <= 7) and the producers' registers suffice.
constexpr int OZ_TILE = 64;      // the largest tile (workspace sizing)
constexpr int OZ_MAXS = 7;

struct OzParams {
    int64_t N, nsa, nsb;
    int npair, KC, s, L0, g_slice_bytes;
    const int32_t *pairA, *pairB;
    const int64_t *Cint;
    const uint4 *Gimg;
    int64_t *E;
    int64_t ldE;
    int *status;
    long long timeout_cycles;
    int stall_test;
    int ring;  // digit-plane slots in use
    int nt;    // determinants per tile (the kernel's NT)
};

// Several sigma builds in one launch: CTAs [cta_start[j], cta_start[j+1]) serve job j.
// Passed by value (kernel parameter space), so the launch needs no device-side table.
constexpr int OZ_MAX_JOBS = 32;
struct OzGroup {
    int n_jobs;
    int cta_start[OZ_MAX_JOBS + 1];
    OzParams job[OZ_MAX_JOBS];
};

// Warp-uniform variant: lane 0 waits, every lane gets the same answer, so no lane can
// leave a loop that the others continue (the tcgen05.ld/alloc forms are .sync.aligned).
__device__ __forceinline__ bool oz_wait_warp(uint32_t bar, uint32_t parity, volatile int *abort, int *status,
                                             long long timeout);

struct OzShared {  // lives after the operand buffers
    uint64_t plane_full[OZ_MAX_RING], plane_empty[OZ_MAX_RING];
    uint64_t acc_full[2], acc_empty[2];
    uint64_t drain;
    uint32_t tmem_base;
    int abort;
};

// Bounded wait: returns false on timeout or when another role has aborted.
__device__ __forceinline__ bool oz_wait(uint32_t bar, uint32_t parity, volatile int *abort, int *status,
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

__device__ __forceinline__ bool oz_wait_warp(uint32_t bar, uint32_t parity, volatile int *abort, int *status,
                                             long long timeout) {
    int ok = 0;
    if ((threadIdx.x & 31) == 0) ok = oz_wait(bar, parity, abort, status, timeout) ? 1 : 0;
    return __shfl_sync(0xFFFFFFFFu, ok, 0) != 0;
}

// S: slices per operand; NT: determinants per tile (the MMA's N).  Accumulators are
// double-buffered when 2 x S x NT TMEM columns fit in 512, single-buffered otherwise.
template <int S, int NT>
__global__ void __launch_bounds__(OZ_THREADS, 1) k_oz_contract(const __grid_constant__ OzGroup grp) {
    // this CTA's job, and its place among the CTAs of that job
    // (the job's parameters are copied to shared memory once; roles read them there)
    __shared__ OzParams p;
    __shared__ int64_t cta_lo, cta_n;
    if (threadIdx.x == 0) {
        int jb = 0;
        while (jb + 1 < grp.n_jobs && (int)blockIdx.x >= grp.cta_start[jb + 1]) ++jb;
        p = grp.job[jb];
        cta_lo = grp.cta_start[jb];
        cta_n = grp.cta_start[jb + 1] - grp.cta_start[jb];
    }
    __syncthreads();
    constexpr int NBUF = (2 * S * NT <= 512) ? 2 : 1;
    constexpr int PT = 32 * OZ_PRODUCER_WARPS;
    constexpr int UNITS = (NT * 16 + PT - 1) / PT;  // producer units per thread (KC <= 16)
    constexpr int L0 = (S - 1 > 2 * S - 6) ? S - 1 : 2 * S - 6;
    extern __shared__ __align__(1024) uint8_t oz_smem_raw[];
    uint8_t *smem = (uint8_t *)(((uintptr_t)oz_smem_raw + 1023) & ~(uintptr_t)1023);
    const int KC = p.KC, RING = p.ring;
    const int plane_bytes = NT * KC * 16;
    uint8_t *sG = smem;
    uint8_t *sRing = sG + (size_t)S * p.g_slice_bytes;
    OzShared *sh = (OzShared *)(sRing + RING * plane_bytes);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

    // G digit slices: one copy per CTA, reused for every tile
    {
        const int n16 = S * p.g_slice_bytes / 16;
        uint4 *dst = (uint4 *)sG;
        for (int i = threadIdx.x; i < n16; i += blockDim.x) dst[i] = __ldg(p.Gimg + i);
    }
    if (threadIdx.x == 0) {
        for (int r = 0; r < RING; ++r) {
            mbar_init(smem_u32(&sh->plane_full[r]), OZ_PRODUCER_WARPS);
            mbar_init(smem_u32(&sh->plane_empty[r]), 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(smem_u32(&sh->acc_full[b]), 1);
            mbar_init(smem_u32(&sh->acc_empty[b]), OZ_EPILOGUE_WARPS);
        }
        mbar_init(smem_u32(&sh->drain), 1);
        sh->abort = 0;
        fence_barrier_init();
    }
    if (warp == OZ_MMA_WARP) {
        tmem_alloc(smem_u32(&sh->tmem_base), 512);
        tmem_relinquish();
    }
    fence_proxy_async_smem();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = sh->tmem_base;
    volatile int *abort = &sh->abort;
    // Each CTA takes one contiguous range of tiles, so consecutive tiles of a CTA share
    // alpha strings and read the same rows of C (cache and TLB locality).
    const int64_t ntiles = (p.N + NT - 1) / NT;
    const int64_t cta = (int64_t)blockIdx.x - cta_lo;
    const int64_t t_begin = ntiles * cta / cta_n, t_end = ntiles * (cta + 1) / cta_n;

    if (warp < OZ_PRODUCER_WARPS) {
        // ---------------------------------------------------------------- producers
        // Thread t owns units (det r, K-core c) t, t + 224, ... of the tile: 8 pair
        // indices rs = 8c..8c+7 of one determinant.  The pair tables have rows up to the
        // padded K, filled with -1, so no range test is needed.
        const int t = threadIdx.x;  // 0..223
        const int units = NT * KC;
        constexpr uint64_t bias = 0x8080808080808080ull >> (8 * (8 - S));
        uint32_t q = 0, slot = 0, ph = 0;  // planes produced, ring slot, the slot's use parity
        for (int64_t tile = t_begin; tile < t_end; ++tile) {
            uint32_t ylo[UNITS][8], yhi[UNITS][8];
#pragma unroll
            for (int u = 0; u < UNITS; ++u) {
                const int unit = t + PT * u;
                const int r = unit % NT, c = unit / NT;
                // determinant counts of the split path fit 32 bits (n <= 15 orbitals)
                const uint32_t det = (uint32_t)tile * NT + (uint32_t)r;
                const bool live = unit < units && det < (uint32_t)p.N;
                const uint32_t nsa = (uint32_t)p.nsa, nsb = (uint32_t)p.nsb;
                const uint32_t ka = live ? det / nsb : 0u, kb = live ? det - ka * nsb : 0u;
                const uint32_t rowoff = ka * nsb;
                const int32_t *pa = p.pairA + ((uint32_t)(8 * c) * nsa + ka);
                const int32_t *pb = p.pairB + ((uint32_t)(8 * c) * nsb + kb);
                int32_t ea[8], eb[8];
#pragma unroll
                for (int e = 0; e < 8; ++e) {
                    ea[e] = live ? __ldg(pa + e * nsa) : -1;
                    eb[e] = live ? __ldg(pb + e * nsb) : -1;
                }
                // entry e = 2 x (source string) + odd, or -1: ((x & valid) ^ odd) - odd is
                // +x, -x or 0 (absent entries load a clamped, valid element)
#pragma unroll
                for (int e = 0; e < 8; ++e) {
                    const int64_t xa = __ldg(p.Cint + ((uint32_t)max(ea[e] >> 1, 0) * nsb + kb));
                    const int64_t xb = __ldg(p.Cint + (rowoff + (uint32_t)max(eb[e] >> 1, 0)));
                    const int64_t va = ~(int64_t)(ea[e] >> 31), oa = -(int64_t)(ea[e] & 1);
                    const int64_t vb = ~(int64_t)(eb[e] >> 31), ob = -(int64_t)(eb[e] & 1);
                    const int64_t v = (((xa & va) ^ oa) - oa) + (((xb & vb) ^ ob) - ob);
                    const uint64_t y = (uint64_t)v + bias;
                    ylo[u][e] = (uint32_t)y;
                    yhi[u][e] = (uint32_t)(y >> 32);
                }
            }
#pragma unroll
            for (int j = S - 1; j >= 0; --j, ++q) {
                if (q >= (uint32_t)RING && !oz_wait_warp(smem_u32(&sh->plane_empty[slot]), ph ^ 1, abort, p.status,
                                                         p.timeout_cycles))
                    goto producer_done;
                uint8_t *plane = sRing + slot * plane_bytes;
                const uint32_t bj = (uint32_t)(j & 3);
                const uint32_t sel = bj | ((4u + bj) << 8);
#pragma unroll
                for (int u = 0; u < UNITS; ++u) {
                    const int unit = t + PT * u;
                    if (unit >= units) continue;
                    const int r = unit % NT, c = unit / NT;
                    uint32_t w[4];
#pragma unroll
                    for (int e = 0; e < 8; e += 2)
                        w[e / 2] = j < 4 ? digits_f16x2(ylo[u][e], ylo[u][e + 1], sel)
                                         : digits_f16x2(yhi[u][e], yhi[u][e + 1], sel);
                    const uint32_t off = (uint32_t)(((r >> 3) * KC + c) * 128 + (r & 7) * 16);
                    *(uint4 *)(plane + off) = make_uint4(w[0], w[1], w[2], w[3]);
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
    } else if (warp < OZ_MMA_WARP) {
        // ---------------------------------------------------------------- epilogue
        // Warp (quadrant qd, half h) reads lanes 32 qd .. 32 qd + 31 and columns
        // [h NT/2, (h+1) NT/2) in chunks of 16, every level of a chunk into int64.
        // A warp may only access the TMEM lane quadrant warp_id % 4; the two warps of a
        // quadrant split the tile's columns.
        const int ew = warp - OZ_PRODUCER_WARPS;
        const int qd = warp & 3;
        const int cbeg = (NT / 2) * (ew >> 2);
        const int row = 32 * qd + lane;
        constexpr int lowshift = 8 * (L0 - (S - 1));
        uint32_t tau = 0;
        for (int64_t tile = t_begin; tile < t_end; ++tile, ++tau) {
            const int buf = NBUF == 2 ? (int)(tau & 1) : 0;
            const uint32_t par = NBUF == 2 ? (tau >> 1) & 1 : tau & 1;
            if (!oz_wait_warp(smem_u32(&sh->acc_full[buf]), par, abort, p.status, p.timeout_cycles)) break;
            tc_fence_after();
            const uint32_t tlane = tmem + ((uint32_t)(32 * qd) << 16) + (uint32_t)(buf * S * NT);
            int64_t *dst_tile = p.E + tile * ((int64_t)p.npair * NT) + (int64_t)row * NT;
#pragma unroll 1
            for (int c0 = cbeg; c0 < cbeg + NT / 2; c0 += 16) {
                int64_t acc[16];
#pragma unroll
                for (int c = 0; c < 16; ++c) acc[c] = 0;
                uint32_t vs[S][16];  // all levels of the chunk in flight, one wait
#pragma unroll
                for (int l = 0; l < S; ++l) tmem_ld16(tlane + (uint32_t)(l * NT + c0), vs[l]);
                tmem_ld_wait();
#pragma unroll
                for (int l = 0; l < S; ++l) tmem_regs_ready(vs[l]);
#pragma unroll
                for (int L = S - 1; L <= 2 * S - 2; ++L) {
                    const uint32_t *v = vs[L - (S - 1)];
                    if (L < L0) {
#pragma unroll
                        for (int c = 0; c < 16; ++c)
                            acc[c] += (int64_t)__float2int_rn(__uint_as_float(v[c])) * ((int64_t)1 << (8 * (L - (S - 1))));
                    } else {
                        if (L == L0 && lowshift > 0) {
#pragma unroll
                            for (int c = 0; c < 16; ++c)
                                acc[c] = (acc[c] + ((int64_t)1 << (lowshift > 0 ? lowshift - 1 : 0))) >> lowshift;
                        }
#pragma unroll
                        for (int c = 0; c < 16; ++c)
                            acc[c] += (int64_t)__float2int_rn(__uint_as_float(v[c])) * ((int64_t)1 << (8 * (L - L0)));
                    }
                }
                if (row < p.npair) {
                    // tile-major E: the block of one tile (n_pair rows x NT) is contiguous
                    const int64_t d0 = tile * NT + c0;
                    int64_t *dst = dst_tile + c0;
                    if (d0 + 16 <= p.N) {
#pragma unroll
                        for (int c = 0; c < 16; c += 2)  // streaming stores: E is read once, by the scatter
                            __stcs((longlong2 *)(dst + c), make_longlong2(acc[c], acc[c + 1]));
                    } else {
                        for (int c = 0; c < 16; ++c)
                            if (d0 + c < p.N) dst[c] = acc[c];
                    }
                }
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(smem_u32(&sh->acc_empty[buf]));
        }
    } else if (lane == 0) {
        // ---------------------------------------------------------------- MMA issuer
        // Descriptors differ only in the 14-bit start-address field: one base per G slice
        // and for the ring, plus 16 (= 256 bytes >> 4) per K-step.
        const uint32_t idesc = idesc_f16(128, NT);
        const uint32_t sbo = (uint32_t)(KC * 128);
        uint64_t adesc[S];
#pragma unroll
        for (int i = 0; i < S; ++i) adesc[i] = smem_desc(smem_u32(sG) + (uint32_t)(i * p.g_slice_bytes), 128, sbo);
        const uint64_t bdesc0 = smem_desc(smem_u32(sRing), 128, sbo);
        const uint32_t bstep = (uint32_t)(plane_bytes >> 4);  // ring slots are contiguous
        const int ksteps = KC / 2;
        uint32_t slot = 0, ph = 0, tau = 0;  // ring slot, its use parity, tile counter
        bool issued = false;
        for (int64_t tile = t_begin; tile < t_end; ++tile, ++tau) {
            const int buf = NBUF == 2 ? (int)(tau & 1) : 0;
            if (tau >= (uint32_t)NBUF) {
                const uint32_t par = NBUF == 2 ? ((tau >> 1) - 1) & 1 : (tau - 1) & 1;
                if (!oz_wait(smem_u32(&sh->acc_empty[buf]), par, abort, p.status, p.timeout_cycles)) break;
            }
            tc_fence_after();
            const uint32_t dbase = tmem + (uint32_t)(buf * S * NT);
            bool ok = true;
#pragma unroll
            for (int j = S - 1; j >= 0; --j) {
                if (!oz_wait(smem_u32(&sh->plane_full[slot]), ph, abort, p.status, p.timeout_cycles)) {
                    ok = false;
                    break;
                }
                tc_fence_after();
                const uint64_t b0 = bdesc0 + (uint64_t)(slot * bstep);
                for (int kk = 0; kk < ksteps; ++kk) {
                    const uint64_t b = b0 + (uint64_t)(kk * 16);
                    const uint32_t acc_in = (j != S - 1 || kk != 0) ? 1u : 0u;
#pragma unroll
                    for (int i = S - 1 - j; i < S; ++i)
                        mma_f16(dbase + (uint32_t)((i + j - (S - 1)) * NT), adesc[i] + (uint64_t)(kk * 16), b,
                                idesc, acc_in);
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
        if (issued) {  // drain: every MMA this thread issued has completed before TMEM is freed
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
    if (warp == OZ_MMA_WARP) tmem_dealloc(tmem, 512);
}

// ------------------------------------------------------------- helper kernels

__global__ void k_absmax_bits(const double *__restrict__ x, int64_t n, unsigned long long *__restrict__ out) {
    unsigned long long m = 0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        m = max(m, (unsigned long long)__double_as_longlong(x[i]) & 0x7FFFFFFFFFFFFFFFull);
    for (int o = 16; o; o >>= 1) m = max(m, __shfl_xor_sync(0xFFFFFFFFu, m, o));
    if ((threadIdx.x & 31) == 0 && m) atomicMax(out, m);
}

// C_int = round(C 2^{sh_C}), sh_C = 8 s - 3 - e_C with max|C| < 2^{e_C}: |C_int| < 2^{8s-3}
// and |D_int| < 2^{8s-2}, inside the range of s balanced digits.
__global__ void k_to_fixed(const double *__restrict__ C, int64_t n, int s,
                           const unsigned long long *__restrict__ maxbits, int64_t *__restrict__ Cint,
                           int *__restrict__ shC) {
    const unsigned long long mb = *maxbits;
    const int e = mb ? (int)((mb >> 52) & 0x7FF) - 1022 : 0;  // max|C| < 2^e (normal numbers)
    const int sh = 8 * s - 3 - e;
    if (blockIdx.x == 0 && threadIdx.x == 0) *shC = sh;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        Cint[i] = __double2ll_rn(scalbn(C[i], sh));
}

// sigma_I = scale * sum over the replacements of I of sign * E_int[pq, K] + e_core C_I, in
// int64.  Thread = beta string ib (consecutive threads, consecutive determinants), looping
// over alpha strings; pairs are taken 8 at a time, their 16 table entries loaded first,
// then their 16 E_int values (loads predicated off for absent replacements), so that each
// thread keeps up to 16 loads in flight.  Pair-table rows run to n_pair_pad (multiple of
// 16) and hold -1 past n_pair.  The sign is applied as x ^ -odd, and the number of odd
// terms is added at the end ((x ^ -1) + 1 = -x; integer sums, so the bits are those of
// the plain signed sum).
__global__ void __launch_bounds__(256) k_scatter_int(uint32_t nsa, uint32_t nsb, int npair_pad, int log2T,
                                                     const int32_t *__restrict__ pairA,
                                                     const int32_t *__restrict__ pairB,
                                                     const int64_t *__restrict__ E, int64_t ldE,
                                                     const double *__restrict__ C, double e_core, int ushift,
                                                     const int *__restrict__ shC, const int *__restrict__ status,
                                                     int *__restrict__ sticky, double *__restrict__ sigma) {
    const uint32_t ib = blockIdx.x * blockDim.x + threadIdx.x;
    if (ib >= nsb) return;
    const int u = ushift - *shC;
    const bool bad = *status != 0;
    if (bad && ib == 0 && blockIdx.y == 0) atomicExch(sticky, *status);  // kept for fci_sync_status
    // E is tile-major: element (pq, K) at (K / T) * R * T + pq * T + K % T, T = 2^log2T,
    // R = ldE rows per tile (n_pair for the fused kernel, 128 for the two-pass GEMM).
    // Determinant indices are 32-bit (ndet < 2^31); a pair-table entry e is 2 x (source
    // string) + (1 if odd) or -1 (absent).
    const uint64_t tstride = (uint64_t)ldE << log2T;
    const uint32_t tmask = (1u << log2T) - 1u;
    for (uint32_t ia = blockIdx.y; ia < nsa; ia += gridDim.y) {
        const uint32_t rowoff = ia * nsb;
        const int32_t *pa = pairA + ia, *pb = pairB + ib;
        int64_t acc = 0;
        int32_t nodd = 0;
        for (int p0 = 0; p0 < npair_pad; p0 += 8, pa += 8 * nsa, pb += 8 * nsb) {
            int32_t ea[8], eb[8];
#pragma unroll
            for (int e = 0; e < 8; ++e) {
                ea[e] = __ldg(pa + e * nsa);
                eb[e] = __ldg(pb + e * nsb);
            }
            int64_t xa[8], xb[8];
#pragma unroll
            for (int e = 0; e < 8; ++e) {
                const uint32_t Ka = (uint32_t)(ea[e] >> 1) * nsb + ib;
                const uint32_t Kb = rowoff + (uint32_t)(eb[e] >> 1);
                const uint32_t r = (uint32_t)(p0 + e) << log2T;
                xa[e] = ea[e] >= 0 ? __ldg(E + ((uint64_t)(Ka >> log2T) * tstride + (r + (Ka & tmask)))) : 0;
                xb[e] = eb[e] >= 0 ? __ldg(E + ((uint64_t)(Kb >> log2T) * tstride + (r + (Kb & tmask)))) : 0;
            }
#pragma unroll
            for (int e = 0; e < 8; ++e) {
                const int32_t oa = (ea[e] & 1) & ~(ea[e] >> 31), ob = (eb[e] & 1) & ~(eb[e] >> 31);
                acc += (xa[e] ^ -(int64_t)oa) + (xb[e] ^ -(int64_t)ob);
                nodd += oa + ob;
            }
        }
        acc += nodd;
        const uint32_t det = rowoff + ib;
        sigma[det] = bad ? __longlong_as_double(0x7FF8000000000000ll) : scalbn(__ll2double_rn(acc), u) + e_core * C[det];
    }
}

// The same gather-back for the two-pass layout (tiles of 64 determinants, 128 rows), with
// compile-time tile arithmetic (IDX32: element offsets below 2^32), loads predicated off
// for absent replacements, and the sign applied as x ^ -odd with the odd count added at
// the end ((x ^ -1) + 1 = -x; integer sums, so the result is the same bits).
template <bool IDX32>
__global__ void __launch_bounds__(128) k_scatter_int2p(uint32_t nsa, uint32_t nsb, int npair_pad,
                                                       const int32_t *__restrict__ pairA,
                                                       const int32_t *__restrict__ pairB,
                                                       const int64_t *__restrict__ E,
                                                       const double *__restrict__ C, double e_core, int ushift,
                                                       const int *__restrict__ shC, const int *__restrict__ status,
                                                       int *__restrict__ sticky, double *__restrict__ sigma) {
    const uint32_t ib = blockIdx.x * blockDim.x + threadIdx.x;
    if (ib >= nsb) return;
    const int u = ushift - *shC;
    const bool bad = *status != 0;
    if (bad && ib == 0 && blockIdx.y == 0) atomicExch(sticky, *status);
    auto at = [&](uint32_t K, int row) -> const int64_t * {
        if (IDX32) return E + (((K >> 6) << 13) + ((uint32_t)row << 6) + (K & 63u));
        return E + ((((uint64_t)(K >> 6)) << 13) + (uint32_t)(row << 6) + (K & 63u));
    };
    for (uint32_t ia = blockIdx.y; ia < nsa; ia += gridDim.y) {
        const uint32_t rowoff = ia * nsb;
        const int32_t *pa = pairA + ia, *pb = pairB + ib;
        int64_t acc = 0;
        int32_t nodd = 0;
        for (int p0 = 0; p0 < npair_pad; p0 += 8, pa += 8 * nsa, pb += 8 * nsb) {
            int32_t ea[8], eb[8];
#pragma unroll
            for (int e = 0; e < 8; ++e) {
                ea[e] = __ldg(pa + e * nsa);
                eb[e] = __ldg(pb + e * nsb);
            }
            int64_t xa[8], xb[8];
#pragma unroll
            for (int e = 0; e < 8; ++e) {
                xa[e] = ea[e] >= 0 ? __ldg(at((uint32_t)(ea[e] >> 1) * nsb + ib, p0 + e)) : 0;
                xb[e] = eb[e] >= 0 ? __ldg(at(rowoff + (uint32_t)(eb[e] >> 1), p0 + e)) : 0;
            }
#pragma unroll
            for (int e = 0; e < 8; ++e) {
                const int32_t oa = (ea[e] & 1) & ~(ea[e] >> 31), ob = (eb[e] & 1) & ~(eb[e] >> 31);
                acc += (xa[e] ^ -(int64_t)oa) + (xb[e] ^ -(int64_t)ob);
                nodd += oa + ob;
            }
        }
        acc += nodd;
        const uint32_t det = rowoff + ib;
        sigma[det] = bad ? __longlong_as_double(0x7FF8000000000000ll) : scalbn(__ll2double_rn(acc), u) + e_core * C[det];
    }
}

// Two-pass path, first pass: the digit image of D for the bulk-copy GEMM.  Block (N-tile
// nt, K-chunk kc) of the image holds S planes of 64 determinants x 8 KCC pairs in canonical
// K-major core matrices.  One alpha string (one row of C) at a time: a block stages the
// C_int row of its alpha string and the row's alpha-move table entries (the same for every
// determinant of the row) in shared memory, so the beta moves of every determinant read
// shared memory instead of scattered global words, and the alpha moves read coalesced runs
// of C_int rows after one shared-memory lookup (a row is at most C(15,7) x 8 bytes = 51 KB
// for the at most 15 orbitals of this path).  Thread t takes pairs 8 (t / (256 / KCC)) .. + 7 of each
// K-chunk and determinants t % (256 / KCC) + j (256 / KCC) of the row; block 0 also writes
// the zero digits of the padding determinants of the last tile (pair-table rows past
// n_pair_pad give zero digits too).  Index arithmetic is 32-bit (the caller guarantees
// ndet < 2^31), and the sign is branch-free: an entry e of a pair table is
// 2 x (source string) + (1 if the excitation is odd), or -1 for none;
// ((x & valid) ^ odd) - odd with valid = ~(e >> 31) and odd = -(e & 1) gives +x, -x or 0
// (the load index of an absent entry is clamped to a valid element).  Capped at 40
// registers for six resident blocks per SM (the loads of the pair table and of C rows are
// what the warps wait on; measured 11% faster at 14e/14o).
template <int S, int KCC>
__global__ void __launch_bounds__(256, 6) k_fci_split_rows(uint32_t ndet, uint32_t nsa, uint32_t nsb, int npair_pad,
                                                        int n_kc, int64_t n_nt, const int32_t *__restrict__ pairA,
                                                        const int32_t *__restrict__ pairB,
                                                        const int64_t *__restrict__ Cint, uint8_t *__restrict__ Dimg) {
    extern __shared__ int64_t sC[];
    int32_t *sEa = reinterpret_cast<int32_t *>(sC + nsb);  // [npair_pad]: the row's alpha-move entries
    constexpr uint64_t bias = 0x8080808080808080ull >> (8 * (8 - S));
    constexpr int B_PLANE = OZG_N * KCC * 16;
    constexpr int DPT = 256 / KCC;  // determinants of the row per pass of the block
    const int cc = threadIdx.x / DPT, dl = threadIdx.x % DPT;
    const uint32_t stepb = 8u * KCC * nsb;
    for (uint32_t ka = blockIdx.x; ka < nsa; ka += gridDim.x) {
        __syncthreads();  // the previous row is no longer read
        for (uint32_t i = threadIdx.x; i < nsb; i += blockDim.x) sC[i] = Cint[(size_t)ka * nsb + i];
        for (int i = threadIdx.x; i < npair_pad; i += blockDim.x) sEa[i] = __ldg(pairA + (uint32_t)i * nsa + ka);
        __syncthreads();
        for (uint32_t kb = dl; kb < nsb; kb += DPT) {
            const uint32_t det = ka * nsb + kb;
            const int row = (int)(det & 63);
            uint8_t *tile = Dimg + (size_t)(det >> 6) * n_kc * S * B_PLANE + ((row >> 3) * KCC + cc) * 128 + (row & 7) * 16;
            const int32_t *pb = pairB + ((uint32_t)(cc * 8) * nsb + kb);
#pragma unroll 1
            for (int kc = 0; kc < n_kc; ++kc, pb += stepb) {
                const int rs0 = kc * 8 * KCC + cc * 8;
                int32_t ea[8], eb[8];
#pragma unroll
                for (int e = 0; e < 8; ++e) {
                    const bool ok = rs0 + e < npair_pad;
                    ea[e] = ok ? sEa[rs0 + e] : -1;
                    eb[e] = ok ? __ldg(pb + e * nsb) : -1;
                }
                uint32_t ylo[8], yhi[8];
#pragma unroll
                for (int e = 0; e < 8; ++e) {
                    const int64_t xa = __ldg(Cint + ((uint32_t)max(ea[e] >> 1, 0) * nsb + kb));
                    const int64_t xb = sC[max(eb[e] >> 1, 0)];
                    const int64_t va = ~(int64_t)(ea[e] >> 31), oa = -(int64_t)(ea[e] & 1);
                    const int64_t vb = ~(int64_t)(eb[e] >> 31), ob = -(int64_t)(eb[e] & 1);
                    const int64_t v = (((xa & va) ^ oa) - oa) + (((xb & vb) ^ ob) - ob);
                    const uint64_t y = (uint64_t)v + bias;
                    ylo[e] = (uint32_t)y;
                    yhi[e] = (uint32_t)(y >> 32);
                }
                uint8_t *base = tile + (size_t)kc * S * B_PLANE;
#pragma unroll
                for (int j = 0; j < S; ++j) {
                    const uint32_t bj = (uint32_t)(j & 3), sel = bj | ((4u + bj) << 8);
                    uint32_t w[4];
#pragma unroll
                    for (int e = 0; e < 8; e += 2)
                        w[e / 2] = j < 4 ? digits_f16x2(ylo[e], ylo[e + 1], sel) : digits_f16x2(yhi[e], yhi[e + 1], sel);
                    __stcs((uint4 *)(base + j * B_PLANE), make_uint4(w[0], w[1], w[2], w[3]));
                }
            }
        }
    }
    if (blockIdx.x == 0) {
        // digit 0 is the binary16 +0.0, so a padding determinant's planes are zero bytes
        const uint32_t npad = (uint32_t)(n_nt * OZG_N - ndet);
        const uint32_t items = npad * KCC * n_kc * S;
        for (uint32_t i = threadIdx.x; i < items; i += blockDim.x) {
            uint32_t r = i;
            const int j = (int)(r % S);
            r /= S;
            const int kc = (int)(r % n_kc);
            r /= n_kc;
            const int c2 = (int)(r % KCC);
            r /= KCC;
            const uint32_t det = ndet + r;
            const int row = (int)(det & 63);
            uint8_t *q = Dimg + ((size_t)(det >> 6) * n_kc + kc) * S * B_PLANE + (size_t)j * B_PLANE +
                         ((row >> 3) * KCC + c2) * 128 + (row & 7) * 16;
            *(uint4 *)q = make_uint4(0, 0, 0, 0);
        }
    }
}

inline size_t al256(size_t b) { return (b + 255) & ~(size_t)255; }

int oz_kc(const fci_context *h) { return ((h->npair + 15) / 16) * 2; }
int oz_L0(int s) { return std::max(s - 1, 2 * s - 6); }
constexpr size_t OZ_SMEM_MAX = 232448;
size_t oz_smem_bytes(int s, int KC, int ring, int nt) {
    return 1024 + (size_t)s * 128 * KC * 16 + (size_t)ring * nt * KC * 16 + sizeof(OzShared);
}
int oz_ring(int s, int KC, int nt) {
    if (oz_smem_bytes(s, KC, 3, nt) <= OZ_SMEM_MAX) return 3;
    if (oz_smem_bytes(s, KC, 2, nt) <= OZ_SMEM_MAX) return 2;
    return 0;
}
// Tile width of this handle for s slices: the tuner's choice, else FCI_OZ_TILE from the
// environment (32 or 64), else 64.
// Contraction path for s slices: 1 = two-pass (digit image of D in HBM, then the
// bulk-copy GEMM), 0 = fused producer kernel.  The tuner's choice, else FCI_OZ_PATH
// ("gemm" / "fused") from the environment, else two-pass from 2^20 determinants on (where
// it was measured faster at every slice count) and fused below (small problems, which
// also share grouped launches).
int oz_path(const fci_context *h, int s) {
    if (s >= 2 && s <= 8 && h->oz_tuned_nt[s]) return h->oz_tuned_path[s];
    if (const char *env = getenv("FCI_OZ_PATH")) return strcmp(env, "gemm") == 0 ? 1 : 0;
    return (h->ndet >= ((int64_t)1 << 20) && s <= 7) ? 1 : 0;
}
int oz_nt(const fci_context *h, int s) {
    if (s >= 2 && s <= 8 && h->oz_tuned_nt[s]) return h->oz_tuned_nt[s];
    if (const char *env = getenv("FCI_OZ_TILE")) {
        const int v = atoi(env);
        if (v == 32 || v == 64) return v;
    }
    return 64;
}

}  // namespace

// Fixed point of C for the split paths with int64 digits: maxbits (zeroed by the caller)
// receives the largest |C| bit pattern, shC the shift, Cint = round(C 2^{sh_C}).
cudaError_t launch_to_fixed64(const double *C, int64_t n, int s, unsigned long long *maxbits, int64_t *Cint, int *shC,
                              cudaStream_t st) {
    const unsigned nb = (unsigned)std::max<int64_t>(1, std::min<int64_t>(ceil_div(n, 256), 152 * 8));
    k_absmax_bits<<<nb, 256, 0, st>>>(C, n, maxbits);
    k_to_fixed<<<nb, 256, 0, st>>>(C, n, s, maxbits, Cint, shC);
    return cudaGetLastError();
}

// IEEE binary16 encoding of an integer |d| <= 1024 (exact).
static uint16_t half_bits_of_small_int(int d) {
    if (d == 0) return 0;
    const uint16_t sign = d < 0 ? 0x8000 : 0;
    unsigned m = (unsigned)(d < 0 ? -d : d);
    int e = 31 - __builtin_clz(m);  // m in [2^e, 2^(e+1))
    const unsigned mant = (m << (10 - e)) & 0x3FF;
    return (uint16_t)(sign | ((unsigned)(e + 15) << 10) | mant);
}

int oz_prepare_G(fci_context *h, int s) {
    if (h->Gs_slices == s && h->d_Gs) return FCI_OK;
    const int np = h->npair, KC = oz_kc(h);
    const int Kp = KC * 8;
    if (np > 128) return fci_fail(h, FCI_ERR_UNSUPPORTED, "split precision needs <= 128 orbital pairs (n <= 15)");
    if (h->ndet >= ((int64_t)1 << 31)) return fci_fail(h, FCI_ERR_UNSUPPORTED, "split precision needs < 2^31 determinants");
    if (s < 2 || s > OZ_MAXS) return fci_fail(h, FCI_ERR_UNSUPPORTED, "split precision supports 2..%d slices", OZ_MAXS);
    if (s * np > 1023) return fci_fail(h, FCI_ERR_UNSUPPORTED, "level sums would exceed 2^24");
    if (!oz_ring(s, KC, 64)) return fci_fail(h, FCI_ERR_UNSUPPORTED, "%d slices do not fit in shared memory", s);
    std::vector<double> G((size_t)np * np);
    if (cudaMemcpy(G.data(), h->d_G, G.size() * 8, cudaMemcpyDeviceToHost) != cudaSuccess)
        return fci_cuda_check(h, cudaGetLastError(), "G download");
    double gmax = 0.0;
    for (double v : G) gmax = std::max(gmax, fabs(v));
    int eG = 0;
    if (gmax > 0) { frexp(gmax, &eG); }  // gmax < 2^eG
    const int shG = 8 * s - 2 - eG;
    uint64_t bias = 0;
    for (int j = 0; j < s; ++j) bias |= (uint64_t)0x80 << (8 * j);
    const size_t slice_bytes = (size_t)128 * KC * 16;
    std::vector<uint16_t> img(slice_bytes / 2 * s, 0);
    for (int pq = 0; pq < 128; ++pq) {
        for (int rs = 0; rs < Kp; ++rs) {
            int64_t gi = 0;
            if (pq < np && rs < np) gi = llrint(ldexp(G[(size_t)pq * np + rs], shG));
            const uint64_t y = (uint64_t)gi + bias;
            for (int j = 0; j < s; ++j) {
                const int d = (int)((y >> (8 * j)) & 0xFF) - 128;
                const size_t off = ((size_t)(pq >> 3) * KC + (rs >> 3)) * 128 + (pq & 7) * 16 + (rs & 7) * 2;
                img[(j * slice_bytes + off) / 2] = half_bits_of_small_int(d);
            }
        }
    }
    fci_dev_free(h->d_Gs);
    h->d_Gs = nullptr;
    int rc = fci_dev_alloc(h, &h->d_Gs, img.size() * 2);
    if (rc) return rc;
    FCI_CUDA(h, cudaMemcpy(h->d_Gs, img.data(), img.size() * 2, cudaMemcpyHostToDevice));
    h->Gs_slices = s;
    h->G_exp = shG;  // stores sh_G
    return FCI_OK;
}

// Two-pass path geometry: one M-tile of 128 pair rows.  K-chunks of 16 (kcc = 2) with the G
// image resident in shared memory when it fits next to a two-stage ring (K = n_pair_pad),
// else streamed K-chunks of 32 (kcc = 4, K = n_pair_pad rounded up to 32).
struct OzTwoPass {
    int kcc, n_kc;
    bool resa;
    int64_t n_nt;
    size_t d_bytes() const { return (size_t)n_nt * n_kc * OZG_N * kcc * 16; }  // per slice
};
static OzTwoPass oz_gemm_geom(const fci_context *h, int s) {
    OzTwoPass g;
    g.n_nt = (h->ndet + OZG_N - 1) / OZG_N;
    g.kcc = 2;
    g.n_kc = h->npair_pad / 16;
    g.resa = oz_gemm_ring(s, 2, g.n_kc) > 0;
    if (!g.resa) {
        g.kcc = 4;
        g.n_kc = (h->npair_pad + OZG_KC - 1) / OZG_KC;
    }
    return g;
}

// Both paths' buffers fit (the tuner may switch between them): C_int, then either E_int of
// the fused kernel or the D digit image + E_int of the two-pass path.
size_t oz_workspace_bytes(const fci_context *h, int s) {
    const int64_t ntiles = (h->ndet + OZ_TILE - 1) / OZ_TILE;  // E for the widest tile covers the others
    const size_t fused = al256((size_t)ntiles * h->npair * OZ_TILE * 8);
    const OzTwoPass g = oz_gemm_geom(h, std::max(s, 2));
    const size_t two = al256(g.d_bytes() * std::max(s, 2)) + al256((size_t)g.n_nt * OZG_M * OZG_N * 8);
    return al256((size_t)h->ndet * 8) + std::max(fused, two) + 256;
}

// G digit image in the A-tile layout of the bulk-copy GEMM ([K-chunk][plane][128 x 32]).
static int oz_prepare_Gt(fci_context *h, int s) {
    if (h->Gt_slices == s && h->d_Gt) return FCI_OK;  // the layout depends on s only
    int rc = oz_prepare_G(h, s);  // checks, and sh_G
    if (rc) return rc;
    const int np = h->npair;
    const OzTwoPass tg = oz_gemm_geom(h, s);
    const int n_kc = tg.n_kc, kw = 8 * tg.kcc;  // K per chunk
    std::vector<double> G((size_t)np * np);
    if (cudaMemcpy(G.data(), h->d_G, G.size() * 8, cudaMemcpyDeviceToHost) != cudaSuccess)
        return fci_cuda_check(h, cudaGetLastError(), "G download");
    const int shG = h->G_exp;
    uint64_t bias = 0;
    for (int j = 0; j < s; ++j) bias |= (uint64_t)0x80 << (8 * j);
    const size_t a_plane = (size_t)OZG_M * kw * 2, stageA = (size_t)s * a_plane;
    std::vector<uint16_t> img((size_t)n_kc * stageA / 2, 0);
    for (int m = 0; m < OZG_M; ++m)
        for (int k = 0; k < n_kc * kw; ++k) {
            int64_t gi = 0;
            if (m < np && k < np) gi = llrint(ldexp(G[(size_t)m * np + k], shG));
            const uint64_t y = (uint64_t)gi + bias;
            const int kc = k / kw, kk = k % kw;
            const size_t off = (size_t)kc * stageA + ((m >> 3) * tg.kcc + (kk >> 3)) * 128 + (m & 7) * 16 + (kk & 7) * 2;
            for (int j = 0; j < s; ++j)
                img[(off + (size_t)j * a_plane) / 2] = half_bits_of_small_int((int)((y >> (8 * j)) & 0xFF) - 128);
        }
    fci_dev_free(h->d_Gt);
    h->d_Gt = nullptr;
    h->Gt_slices = 0;
    rc = fci_dev_alloc(h, &h->d_Gt, img.size() * 2);
    if (rc) return rc;
    FCI_CUDA(h, cudaMemcpy(h->d_Gt, img.data(), img.size() * 2, cudaMemcpyHostToDevice));
    h->Gt_slices = s;
    return FCI_OK;
}

// Fixed-point conversion of C and the job's kernel parameters (first half of a split sigma).
static int oz_prepare_job(fci_context *h, const double *C, int s, void *ws, cudaStream_t st, OzParams &prm,
                          int64_t **E_out, int **shC_out, int **status_out) {
    if (h->mode != FCI_MODE_FCI) return fci_fail(h, FCI_ERR_UNSUPPORTED, "split precision needs alpha/beta strings");
    if (h->ndet >= ((int64_t)1 << 31)) return fci_fail(h, FCI_ERR_UNSUPPORTED, "split precision: 2^31 determinants or more");
    int rc = oz_prepare_G(h, s);
    if (rc) return rc;
    const int KC = oz_kc(h);
    const int64_t N = h->ndet;
    char *p = (char *)ws;
    int64_t *Cint = (int64_t *)p;
    p += al256((size_t)N * 8);
    int64_t *E = (int64_t *)p;
    p += al256((size_t)((N + OZ_TILE - 1) / OZ_TILE) * h->npair * OZ_TILE * 8);
    unsigned long long *maxbits = (unsigned long long *)p;
    int *shC = (int *)(p + 8);
    int *status = (int *)(p + 16);
    {
        phase_scope ps(h, st, FCI_PHASE_OTHER, 2);
        FCI_CUDA(h, cudaMemsetAsync(p, 0, 256, st));
        const unsigned nb = (unsigned)std::min<int64_t>(ceil_div(N, 256), 152 * 8);
        k_absmax_bits<<<nb, 256, 0, st>>>(C, N, maxbits);
        k_to_fixed<<<nb, 256, 0, st>>>(C, N, s, maxbits, Cint, shC);
        FCI_CUDA(h, cudaGetLastError());
    }
    prm.N = N;
    prm.nsa = h->nsa;
    prm.nsb = h->nsb;
    prm.npair = h->npair;
    prm.KC = KC;
    prm.s = s;
    prm.L0 = oz_L0(s);
    prm.g_slice_bytes = 128 * KC * 16;
    prm.pairA = h->d_pair_a;
    prm.pairB = h->d_pair_b;
    prm.Cint = Cint;
    prm.Gimg = (const uint4 *)h->d_Gs;
    prm.E = E;
    prm.ldE = 0;
    prm.status = status;
    const char *to = getenv("FCI_WAIT_TIMEOUT_MS");
    const double ms = to ? atof(to) : 2000.0;
    prm.timeout_cycles = (long long)(ms * 2.1e6);  // cycles at up to 2.1 GHz
    const char *stall = getenv("FCI_TEST_STALL_PRODUCER");
    prm.stall_test = stall ? atoi(stall) : 0;
    prm.nt = oz_nt(h, s);
    prm.ring = oz_ring(s, KC, prm.nt);
    *E_out = E;
    *shC_out = shC;
    *status_out = status;
    return FCI_OK;
}

template <int NT>
static void (*oz_kernel(int s))(const OzGroup) {
    switch (s) {
        case 2: return k_oz_contract<2, NT>;
        case 3: return k_oz_contract<3, NT>;
        case 4: return k_oz_contract<4, NT>;
        case 5: return k_oz_contract<5, NT>;
        case 6: return k_oz_contract<6, NT>;
        case 7: return k_oz_contract<7, NT>;
        default: return nullptr;
    }
}

static int oz_launch_group(fci_context *h, const OzGroup &grp, int s, int nt, size_t smem, cudaStream_t st) {
    void (*kern)(const OzGroup) = nt == 32 ? oz_kernel<32>(s) : nt == 64 ? oz_kernel<64>(s) : nullptr;
    if (!kern) return fci_fail(h, FCI_ERR_UNSUPPORTED, "slice count %d, tile %d", s, nt);
    FCI_CUDA(h, cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    phase_scope ps(h, st, FCI_PHASE_CONTRACT, 1);
    kern<<<grp.cta_start[grp.n_jobs], OZ_THREADS, smem, st>>>(grp);
    FCI_CUDA(h, cudaGetLastError());
    return FCI_OK;
}

static int oz_finish_job(fci_context *h, const double *C, double *sigma, const OzParams &prm, int64_t *E, int *shC,
                         int *status, cudaStream_t st) {
    phase_scope ps(h, st, FCI_PHASE_SCATTER, 1);
    const int threads = 128;
    dim3 g((unsigned)ceil_div(h->nsb, threads), (unsigned)std::min<int64_t>(h->nsa, 65535));
    k_scatter_int<<<g, threads, 0, st>>>(h->nsa, h->nsb, h->npair_pad, prm.nt == 32 ? 5 : 6, h->d_pair_a, h->d_pair_b,
                                       E, prm.npair,
                                       C, h->e_core,
                                       8 * prm.L0 - h->G_exp, shC, status, h->d_status, sigma);
    FCI_CUDA(h, cudaGetLastError());
    return FCI_OK;
}

static int oz_num_sms(fci_context *h, int *nsm) {
    FCI_CUDA(h, cudaDeviceGetAttribute(nsm, cudaDevAttrMultiProcessorCount, h->device));
    return FCI_OK;
}

// Two-pass split sigma: fixed point, D digit image (k_fci_split_rows), bulk-copy GEMM (8-bit
// digits, one M-tile of 128 pair rows), integer scatter.
static int oz_sigma_fci_gemm(fci_context *h, const double *C, double *sigma, int s, void *ws, cudaStream_t st) {
    if (h->ndet >= ((int64_t)1 << 31)) return fci_fail(h, FCI_ERR_UNSUPPORTED, "split precision: 2^31 determinants or more");
    int rc = oz_prepare_Gt(h, s);
    if (rc) return rc;
    const OzTwoPass tg = oz_gemm_geom(h, s);
    if (!oz_gemm_ring(s, tg.kcc, tg.resa ? tg.n_kc : 0))
        return fci_fail(h, FCI_ERR_UNSUPPORTED, "%d slices do not fit the GEMM pipeline", s);
    const int n_kc = tg.n_kc;
    const int64_t n_nt = tg.n_nt;
    const int64_t N = h->ndet;
    char *p = (char *)ws;
    int64_t *Cint = (int64_t *)p;
    p += al256((size_t)N * 8);
    uint8_t *Dimg = (uint8_t *)p;
    p += al256(tg.d_bytes() * s);
    int64_t *E = (int64_t *)p;
    p += al256((size_t)n_nt * OZG_M * OZG_N * 8);
    // the misc block sits at the end of the larger of the two layouts
    char *misc = (char *)ws + (oz_workspace_bytes(h, s) - 256);
    unsigned long long *maxbits = (unsigned long long *)misc;
    int *shC = (int *)(misc + 8), *status = (int *)(misc + 16);
    {
        phase_scope ps(h, st, FCI_PHASE_GATHER, 3);
        FCI_CUDA(h, cudaMemsetAsync(misc, 0, 256, st));
        const unsigned nb = (unsigned)std::min<int64_t>(ceil_div(N, 256), 152 * 8);
        k_absmax_bits<<<nb, 256, 0, st>>>(C, N, maxbits);
        k_to_fixed<<<nb, 256, 0, st>>>(C, N, s, maxbits, Cint, shC);
        const size_t row_smem = (size_t)h->nsb * 8 + (size_t)h->npair_pad * 4;  // one C row + its alpha entries
        if (row_smem > OZ_SMEM_MAX) return fci_fail(h, FCI_ERR_UNSUPPORTED, "split precision: %lld beta strings", (long long)h->nsb);
        const unsigned gr = (unsigned)h->nsa;  // one block per alpha string: no tail of unequal row counts
        switch (s * 10 + tg.kcc) {
#define OZ_SPLIT(S_, K_)                                                                                          \
    case S_ * 10 + K_:                                                                                            \
        FCI_CUDA(h, cudaFuncSetAttribute(k_fci_split_rows<S_, K_>, cudaFuncAttributeMaxDynamicSharedMemorySize,     \
                                         (int)row_smem));                                                         \
        k_fci_split_rows<S_, K_><<<gr, 256, row_smem, st>>>((uint32_t)N, (uint32_t)h->nsa, (uint32_t)h->nsb,       \
                                                            h->npair_pad, n_kc, n_nt, h->d_pair_a, h->d_pair_b,   \
                                                            Cint, Dimg);                                          \
        break;
            OZ_SPLIT(2, 2) OZ_SPLIT(3, 2) OZ_SPLIT(4, 2) OZ_SPLIT(5, 2) OZ_SPLIT(6, 2) OZ_SPLIT(7, 2)
            OZ_SPLIT(2, 4) OZ_SPLIT(3, 4) OZ_SPLIT(4, 4) OZ_SPLIT(5, 4) OZ_SPLIT(6, 4) OZ_SPLIT(7, 4)
#undef OZ_SPLIT
            default: return fci_fail(h, FCI_ERR_UNSUPPORTED, "slice count %d", s);
        }
        FCI_CUDA(h, cudaGetLastError());
    }
    oz_gemm_args a;
    a.n_mt = 1;
    a.n_kc = n_kc;
    a.M_pad = OZG_M;
    a.M_real = h->npair;
    a.n_nt = n_nt;
    a.Gimg = h->d_Gt;
    a.Dimg = Dimg;
    a.E = E;
    a.status = status;
    if ((rc = oz_gemm_launch(h, s, 8, tg.kcc, tg.resa, a, st))) return rc;
    phase_scope ps(h, st, FCI_PHASE_SCATTER, 1);
    const int threads = 128;
    dim3 g((unsigned)ceil_div(h->nsb, threads), (unsigned)std::min<int64_t>(h->nsa, 65535));
    const int ush = 8 * oz_gemm_L0(s, 8) - h->G_exp;
    if ((uint64_t)n_nt * OZG_M * OZG_N < ((uint64_t)1 << 32))
        k_scatter_int2p<true><<<g, threads, 0, st>>>(h->nsa, h->nsb, h->npair_pad, h->d_pair_a, h->d_pair_b, E, C,
                                                     h->e_core, ush, shC, status, h->d_status, sigma);
    else
        k_scatter_int2p<false><<<g, threads, 0, st>>>(h->nsa, h->nsb, h->npair_pad, h->d_pair_a, h->d_pair_b, E, C,
                                                      h->e_core, ush, shC, status, h->d_status, sigma);
    FCI_CUDA(h, cudaGetLastError());
    return FCI_OK;
}

int oz_sigma_fci(fci_context *h, const double *C, double *sigma, int s, void *ws, size_t ws_bytes, cudaStream_t st) {
    (void)ws_bytes;
    if (oz_path(h, s) == 1) return oz_sigma_fci_gemm(h, C, sigma, s, ws, st);
    OzGroup grp;
    int64_t *E;
    int *shC, *status;
    int rc = oz_prepare_job(h, C, s, ws, st, grp.job[0], &E, &shC, &status);
    if (rc) return rc;
    int nsm = 0;
    if ((rc = oz_num_sms(h, &nsm))) return rc;
    const int nt = grp.job[0].nt;
    const int64_t ntiles = (h->ndet + nt - 1) / nt;
    grp.n_jobs = 1;
    grp.cta_start[0] = 0;
    grp.cta_start[1] = (int)std::min<int64_t>(nsm, ntiles);
    if ((rc = oz_launch_group(h, grp, s, nt, oz_smem_bytes(s, grp.job[0].KC, grp.job[0].ring, nt), st))) return rc;
    return oz_finish_job(h, C, sigma, grp.job[0], E, shC, status, st);
}

// Split-precision sigma of several problems sharing one slice count and tile width: one
// fixed-point pre-pass per job, ONE persistent contraction launch for all jobs (CTAs
// shared in proportion to tiles, at least one per job), one scatter per job.
static int oz_sigma_group_nt(fci_context *const *hs, const double *const *Cs, double *const *sigmas,
                             void *const *wss, int n, int s, int nt, cudaStream_t st) {
    int nsm = 0;
    int rc = oz_num_sms(hs[0], &nsm);
    if (rc) return rc;
    for (int base = 0; base < n;) {
        const int m = std::min({n - base, OZ_MAX_JOBS, nsm});
        OzGroup grp;
        int64_t *E[OZ_MAX_JOBS];
        int *shC[OZ_MAX_JOBS], *status[OZ_MAX_JOBS];
        size_t smem = 0;
        int64_t tiles[OZ_MAX_JOBS], total = 0;
        for (int j = 0; j < m; ++j) {
            fci_context *h = hs[base + j];
            if ((rc = oz_prepare_job(h, Cs[base + j], s, wss[base + j], st, grp.job[j], &E[j], &shC[j], &status[j])))
                return rc;
            smem = std::max(smem, oz_smem_bytes(s, grp.job[j].KC, grp.job[j].ring, nt));
            tiles[j] = (h->ndet + nt - 1) / nt;
            total += tiles[j];
        }
        // CTAs in proportion to tiles, at least one per job, never more CTAs than tiles
        int ctas[OZ_MAX_JOBS], used = 0;
        for (int j = 0; j < m; ++j) {
            ctas[j] = (int)std::max<int64_t>(1, std::min<int64_t>(tiles[j], (int64_t)(nsm - m) * tiles[j] / total + 1));
            used += ctas[j];
        }
        while (used > nsm) {  // trim the largest shares
            int jmax = 0;
            for (int j = 1; j < m; ++j) if (ctas[j] > ctas[jmax]) jmax = j;
            if (ctas[jmax] <= 1) break;
            --ctas[jmax];
            --used;
        }
        grp.n_jobs = m;
        grp.cta_start[0] = 0;
        for (int j = 0; j < m; ++j) grp.cta_start[j + 1] = grp.cta_start[j] + ctas[j];
        if ((rc = oz_launch_group(hs[base], grp, s, nt, smem, st))) return rc;
        for (int j = 0; j < m; ++j)
            if ((rc = oz_finish_job(hs[base + j], Cs[base + j], sigmas[base + j], grp.job[j], E[j], shC[j], status[j], st)))
                return rc;
        base += m;
    }
    return FCI_OK;
}

// Jobs grouped by their tile width (the kernel's template argument), one launch per group;
// jobs configured for the two-pass path run one after another.
int oz_sigma_group(fci_context *const *hs, const double *const *Cs, double *const *sigmas, void *const *wss, int n,
                   int s, cudaStream_t st) {
    for (int i = 0; i < n; ++i)
        if (oz_path(hs[i], s) == 1) {
            const int rc = oz_sigma_fci_gemm(hs[i], Cs[i], sigmas[i], s, wss[i], st);
            if (rc) return rc;
        }
    for (int nt : {64, 32}) {
        std::vector<fci_context *> h2;
        std::vector<const double *> c2;
        std::vector<double *> s2;
        std::vector<void *> w2;
        for (int i = 0; i < n; ++i)
            if (oz_path(hs[i], s) == 0 && oz_nt(hs[i], s) == nt) {
                h2.push_back(hs[i]);
                c2.push_back(Cs[i]);
                s2.push_back(sigmas[i]);
                w2.push_back(wss[i]);
            }
        if (h2.empty()) continue;
        const int rc = oz_sigma_group_nt(h2.data(), c2.data(), s2.data(), w2.data(), (int)h2.size(), s, nt, st);
        if (rc) return rc;
    }
    return FCI_OK;
}

int oz_tune_candidates(const fci_context *h, int s, int *nt, int *path, int max) {
    const int KC = oz_kc(h);
    int n = 0;
    for (int t : {64, 32})
        if (n < max && s * t <= 512 && oz_ring(s, KC, t)) {
            nt[n] = t;
            path[n++] = 0;
        }
    const OzTwoPass tg = oz_gemm_geom(h, s);
    if (n < max && s <= 7 && oz_gemm_ring(s, tg.kcc, tg.resa ? tg.n_kc : 0)) {  // two-pass: 64-determinant tiles
        nt[n] = 64;
        path[n++] = 1;
    }
    return n;
}

void oz_set_config(fci_context *h, int s, int nt, int path) {
    if (s >= 2 && s <= 8) {
        h->oz_tuned_nt[s] = nt;
        h->oz_tuned_path[s] = nt ? path : 0;
    }
}
