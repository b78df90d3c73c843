// Split-precision sigma for complex spinor strings (the relativistic case of the paper's
// Results) with the contraction E = G D on the tcgen05 tensor cores, Ozaki style.
//
// The complex contraction over the n^2 spinor pairs is written as one real GEMM on the
// real embedding (index 2x = real part, 2x + 1 = imaginary part of complex index x):
//   [E_re; E_im] = [[G_re, -G_im]; [G_im, G_re]] [D_re; D_im],
// M = K = 2 n^2 rows (1,152 at 24 spinors), N = the determinants.  Neither operand fits in
// shared memory, so both are streamed: the G digit slices (prepared once) and the D digit
// slices (split from the fixed-point C by k_cz_split each sigma) are stored in HBM in the
// exact shared-memory layout of the MMA operands, tile by tile, and every K-chunk stage
// of the pipeline is filled by two cp.async.bulk copies that complete on an mbarrier.
//
// Digits are balanced base-128 (7 bits, [-64, 63], exact in f16).  A D column has at
// most 2 n_e (n - n_e + 1) nonzero entries (312 at 24 spinors / 12 electrons), so a level
// sum S_L = sum_{i+j=L} G_i D_j stays an integer below s * 312 * 2^12 < 2^24 for s <= 13:
// every FP32 accumulation in TMEM is exact.  The top s levels (L >= s - 1) are formed;
// the epilogue combines them in int64 (levels below L0 = max(s - 1, 2s - 7) rounded
// away), and the scatter sums in int64:
//   sigma_I = 2^{7 L0 - sh_G - sh_C} sum <I|E_x|K> E_int[x, K] + e_core C_I.
//
// Kernel layout (one persistent CTA per SM, 192 threads):
//   warp 0  lane 0 issues the bulk copies of each stage (G tile: s planes of 128 x 32,
//           D tile: s planes of 64 x 32, f16 core matrices);
//   warp 1  allocates TMEM; lane 0 issues the MMAs (M = 128, N = 64, K = 16) and commits;
//   warps 2-5 epilogue, one per TMEM lane quadrant.
// Work units are (N-tile, M-tile) pairs, N-tile outer and dealt round-robin, so the
// M-tiles of one D tile run at the same time and its reads hit L2.  All mbarrier waits
// are bounded in time (FCI_ERR_TIMEOUT in the status word on expiry).
#include <math.h>
#include <stdlib.h>

#include <algorithm>
#include <complex>
#include <vector>

#include "fci_internal.h"
#include "tc_ptx.cuh"

namespace {

using namespace tc;

constexpr int CZ_M = 128;   // rows of G per tile
constexpr int CZ_N = 64;    // determinants per tile
constexpr int CZ_KC = 32;   // K per pipeline stage (4 core matrices of 8)
constexpr int CZ_THREADS = 192;
constexpr int CZ_MAX_STAGES = 6;
constexpr int CZ_A_PLANE = CZ_M * CZ_KC * 2;  // 8 KB
constexpr int CZ_B_PLANE = CZ_N * CZ_KC * 2;  // 4 KB
constexpr size_t CZ_SMEM_MAX = 232448 - 1024;
constexpr int CZ_MAXS = 8;

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
    asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n\t}" ::"r"(bar),
                 "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void *src, uint32_t bytes, uint32_t bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
                 "l"(src), "r"(bytes), "r"(bar)
                 : "memory");
}

struct CzParams {
    int n_mt, n_kc, M_pad, ring;
    int64_t n_nt;
    const uint8_t *Gimg, *Dimg;
    int64_t *E;
    int *status;
    long long timeout_cycles;
};

struct CzShared {
    uint64_t full[CZ_MAX_STAGES], empty[CZ_MAX_STAGES];
    uint64_t acc_full[2], acc_empty[2];
    uint64_t drain;
    uint32_t tmem_base;
    int abort;
};

__device__ __forceinline__ bool cz_wait(uint32_t bar, uint32_t parity, volatile int *abort, int *status,
                                        long long timeout) {
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

__device__ __forceinline__ bool cz_wait_warp(uint32_t bar, uint32_t parity, volatile int *abort, int *status,
                                             long long timeout) {
    int ok = 0;
    if ((threadIdx.x & 31) == 0) ok = cz_wait(bar, parity, abort, status, timeout) ? 1 : 0;
    return __shfl_sync(0xFFFFFFFFu, ok, 0) != 0;
}

template <int S>
__global__ void __launch_bounds__(CZ_THREADS, 1) k_cz_gemm(const __grid_constant__ CzParams p) {
    constexpr int NBUF = (2 * S * CZ_N <= 512) ? 2 : 1;
    constexpr int L0 = (S - 1 > 2 * S - 7) ? S - 1 : 2 * S - 7;
    constexpr uint32_t STAGE_A = S * CZ_A_PLANE, STAGE_B = S * CZ_B_PLANE;
    extern __shared__ __align__(1024) uint8_t cz_smem_raw[];
    uint8_t *smem = (uint8_t *)(((uintptr_t)cz_smem_raw + 1023) & ~(uintptr_t)1023);
    const int R = p.ring;
    uint8_t *sA = smem;                              // R stages of S A-planes
    uint8_t *sB = sA + (size_t)R * STAGE_A;          // R stages of S B-planes
    CzShared *sh = (CzShared *)(sB + (size_t)R * STAGE_B);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        for (int r = 0; r < R; ++r) {
            mbar_init(smem_u32(&sh->full[r]), 1);
            mbar_init(smem_u32(&sh->empty[r]), 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(smem_u32(&sh->acc_full[b]), 1);
            mbar_init(smem_u32(&sh->acc_empty[b]), 4);
        }
        mbar_init(smem_u32(&sh->drain), 1);
        sh->abort = 0;
        fence_barrier_init();
    }
    if (warp == 1) {
        tmem_alloc(smem_u32(&sh->tmem_base), 512);
        tmem_relinquish();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = sh->tmem_base;
    volatile int *abort = &sh->abort;
    const int64_t n_units = p.n_nt * p.n_mt;

    if (warp == 0) {
        if (lane == 0) {
            // ------------------------------------------------------------ bulk copies
            uint32_t q = 0;
            for (int64_t u = blockIdx.x; u < n_units; u += gridDim.x) {
                const int64_t nt = u / p.n_mt;
                const int mt = (int)(u - nt * p.n_mt);
                const uint8_t *ga = p.Gimg + (size_t)mt * p.n_kc * STAGE_A;
                const uint8_t *gb = p.Dimg + (size_t)nt * p.n_kc * STAGE_B;
                bool ok = true;
                for (int kc = 0; kc < p.n_kc; ++kc, ++q) {
                    const int st = (int)(q % (uint32_t)R);
                    const uint32_t use = q / (uint32_t)R;
                    if (use > 0 && !cz_wait(smem_u32(&sh->empty[st]), (use - 1) & 1, abort, p.status,
                                            p.timeout_cycles)) {
                        ok = false;
                        break;
                    }
                    const uint32_t fb = smem_u32(&sh->full[st]);
                    mbar_expect_tx(fb, STAGE_A + STAGE_B);
                    bulk_g2s(smem_u32(sA + (size_t)st * STAGE_A), ga + (size_t)kc * STAGE_A, STAGE_A, fb);
                    bulk_g2s(smem_u32(sB + (size_t)st * STAGE_B), gb + (size_t)kc * STAGE_B, STAGE_B, fb);
                }
                if (!ok) break;
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            // ------------------------------------------------------------ MMA issuer
            const uint32_t idesc = idesc_f16(CZ_M, CZ_N);
            const uint64_t a0 = smem_desc(smem_u32(sA), 128, 4 * 128);
            const uint64_t b0 = smem_desc(smem_u32(sB), 128, 4 * 128);
            uint32_t q = 0, tau = 0;
            bool issued = false, ok = true;
            for (int64_t u = blockIdx.x; u < n_units && ok; u += gridDim.x, ++tau) {
                const int buf = NBUF == 2 ? (int)(tau & 1) : 0;
                if (tau >= (uint32_t)NBUF) {
                    const uint32_t par = NBUF == 2 ? ((tau >> 1) - 1) & 1 : (tau - 1) & 1;
                    if (!cz_wait(smem_u32(&sh->acc_empty[buf]), par, abort, p.status, p.timeout_cycles)) break;
                }
                tc_fence_after();
                const uint32_t dbase = tmem + (uint32_t)(buf * S * CZ_N);
                for (int kc = 0; kc < p.n_kc; ++kc, ++q) {
                    const int st = (int)(q % (uint32_t)R);
                    if (!cz_wait(smem_u32(&sh->full[st]), (q / (uint32_t)R) & 1, abort, p.status, p.timeout_cycles)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const uint64_t as = a0 + (uint64_t)((st * STAGE_A) >> 4);
                    const uint64_t bs = b0 + (uint64_t)((st * STAGE_B) >> 4);
#pragma unroll
                    for (int kk = 0; kk < CZ_KC / 16; ++kk) {
#pragma unroll
                        for (int j = S - 1; j >= 0; --j) {
                            const uint64_t b = bs + (uint64_t)((j * CZ_B_PLANE + kk * 256) >> 4);
                            const uint32_t acc_in = (kc != 0 || kk != 0 || j != S - 1) ? 1u : 0u;
#pragma unroll
                            for (int i = S - 1 - j; i < S; ++i)
                                mma_f16(dbase + (uint32_t)((i + j - (S - 1)) * CZ_N),
                                        as + (uint64_t)((i * CZ_A_PLANE + kk * 256) >> 4), b, idesc, acc_in);
                        }
                    }
                    issued = true;
                    mma_commit(smem_u32(&sh->empty[st]));
                }
                if (!ok) break;
                mma_commit(smem_u32(&sh->acc_full[buf]));
            }
            if (issued) {
                mma_commit(smem_u32(&sh->drain));
                const long long t0 = clock64();
                while (!mbar_try_wait(smem_u32(&sh->drain), 0)) {
                    if (clock64() - t0 > p.timeout_cycles) {
                        atomicExch(p.status, FCI_ERR_TIMEOUT);
                        break;
                    }
                }
            }
        }
    } else {
        // ---------------------------------------------------------------- epilogue
        const int qd = warp & 3;
        const int row = 32 * qd + lane;
        constexpr int lowshift = 7 * (L0 - (S - 1));
        uint32_t tau = 0;
        for (int64_t u = blockIdx.x; u < n_units; u += gridDim.x, ++tau) {
            const int64_t nt = u / p.n_mt;
            const int mt = (int)(u - nt * p.n_mt);
            const int buf = NBUF == 2 ? (int)(tau & 1) : 0;
            const uint32_t par = NBUF == 2 ? (tau >> 1) & 1 : tau & 1;
            if (!cz_wait_warp(smem_u32(&sh->acc_full[buf]), par, abort, p.status, p.timeout_cycles)) break;
            tc_fence_after();
            const uint32_t tl = tmem + ((uint32_t)(32 * qd) << 16) + (uint32_t)(buf * S * CZ_N);
            int64_t *dst_row = p.E + ((size_t)nt * p.M_pad + (size_t)mt * CZ_M + row) * CZ_N;
#pragma unroll 1
            for (int c0 = 0; c0 < CZ_N; c0 += 16) {
                int64_t acc[16];
#pragma unroll
                for (int c = 0; c < 16; ++c) acc[c] = 0;
#pragma unroll
                for (int L = S - 1; L <= 2 * S - 2; ++L) {
                    uint32_t v[16];
                    tmem_ld16(tl + (uint32_t)((L - (S - 1)) * CZ_N + c0), v);
                    tmem_ld_wait();
                    if (L < L0) {
#pragma unroll
                        for (int c = 0; c < 16; ++c)
                            acc[c] += (int64_t)__float2int_rn(__uint_as_float(v[c])) * ((int64_t)1 << (7 * (L - (S - 1))));
                    } else {
                        if (L == L0 && lowshift > 0) {
#pragma unroll
                            for (int c = 0; c < 16; ++c)
                                acc[c] = (acc[c] + ((int64_t)1 << (lowshift > 0 ? lowshift - 1 : 0))) >> lowshift;
                        }
#pragma unroll
                        for (int c = 0; c < 16; ++c)
                            acc[c] += (int64_t)__float2int_rn(__uint_as_float(v[c])) * ((int64_t)1 << (7 * (L - L0)));
                    }
                }
#pragma unroll
                for (int c = 0; c < 16; c += 2) __stcs((longlong2 *)(dst_row + c0 + c), make_longlong2(acc[c], acc[c + 1]));
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(smem_u32(&sh->acc_empty[buf]));
        }
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 1) tmem_dealloc(tmem, 512);
}

// ------------------------------------------------------------- helper kernels

__device__ __forceinline__ uint32_t cz_rank(uint32_t T, const uint64_t *__restrict__ binom) {
    uint32_t r = 0;
    int j = 1;
    while (T) {
        const int q = __ffs(T) - 1;
        r += (uint32_t)__ldg(binom + q * FCI_BINOM_LD + j);
        ++j;
        T &= T - 1;
    }
    return r;
}

__device__ __forceinline__ int cz_sign(uint32_t S, int a, int b) {
    const int lo = a < b ? a : b, hi = a < b ? b : a;
    const uint32_t between = (hi > lo + 1) ? (((1u << hi) - 1u) & ~((2u << lo) - 1u)) : 0u;
    return __popc(S & between) & 1;
}

__global__ void k_cz_absmax(const double *__restrict__ x, int64_t n, unsigned long long *__restrict__ out) {
    unsigned long long m = 0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        m = max(m, (unsigned long long)__double_as_longlong(x[i]) & 0x7FFFFFFFFFFFFFFFull);
    for (int o = 16; o; o >>= 1) m = max(m, __shfl_xor_sync(0xFFFFFFFFu, m, o));
    if ((threadIdx.x & 31) == 0 && m) atomicMax(out, m);
}

// C_int = round(C 2^{sh_C}) for real and imaginary parts, sh_C = 7 s - 3 - e_C with every
// |part| < 2^{e_C}: |C_int| < 2^{7s-3}, inside the range of s balanced base-128 digits.
__global__ void k_cz_to_fixed(const double *__restrict__ C, int64_t n2, int s,
                              const unsigned long long *__restrict__ maxbits, int64_t *__restrict__ Cint,
                              int *__restrict__ shC) {
    const unsigned long long mb = *maxbits;
    const int e = mb ? (int)((mb >> 52) & 0x7FF) - 1022 : 0;
    const int sh = 7 * s - 3 - e;
    if (blockIdx.x == 0 && threadIdx.x == 0) *shC = sh;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n2; i += (int64_t)gridDim.x * blockDim.x)
        Cint[i] = __double2ll_rn(scalbn(C[i], sh));
}

// Two balanced base-128 digits (bits 7j .. 7j+6 of the biased values) as an f16x2 word:
// 0x6400 | d encodes 1024 + d exactly, and one packed subtraction of 1024 + 64 leaves
// d - 64 in [-64, 63].
__device__ __forceinline__ uint32_t digits7_f16x2(uint64_t x, uint64_t y, int j) {
    const uint32_t lo = (uint32_t)(x >> (7 * j)) & 0x7Fu, hi = (uint32_t)(y >> (7 * j)) & 0x7Fu;
    const uint32_t w = (lo | (hi << 16)) | 0x64006400u;
    const __half2 h = __hsub2(*reinterpret_cast<const __half2 *>(&w),
                              __halves2half2(__ushort_as_half(0x6440), __ushort_as_half(0x6440)));
    return *reinterpret_cast<const uint32_t *>(&h);
}

// D digit image: block (N-tile nt, K-chunk kc) holds S planes of 64 determinants x 32
// real-embedded K, each in canonical K-major core matrices (8 rows x 16 bytes; core
// (row / 8, k / 8) at ((row / 8) * 4 + k / 8) * 128).  One CTA of 256 threads fills one
// block: thread t covers determinant t % 64 and core t / 64 (4 complex pairs = 8 reals).
template <int S>
__global__ void __launch_bounds__(256) k_cz_split(int n, int64_t ndet, int n_kc, int64_t n_blocks,
                                                  const uint64_t *__restrict__ str,
                                                  const uint64_t *__restrict__ binom,
                                                  const int64_t *__restrict__ Cint, uint8_t *__restrict__ Dimg) {
    uint64_t bias = 0;
#pragma unroll
    for (int j = 0; j < S; ++j) bias |= (uint64_t)64 << (7 * j);
    const int row = threadIdx.x & 63, cc = threadIdx.x >> 6;
    const int n2 = n * n;
    for (int64_t blk = blockIdx.x; blk < n_blocks; blk += gridDim.x) {
        const int64_t nt = blk / n_kc;
        const int kc = (int)(blk - nt * n_kc);
        const int64_t K = nt * CZ_N + row;
        uint64_t y[8];
        const uint32_t Sm = K < ndet ? (uint32_t)__ldg(str + K) : 0u;
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const int x = (kc * CZ_KC + cc * 8) / 2 + e;  // complex pair index
            int64_t vr = 0, vi = 0;
            if (K < ndet && x < n2) {
                const int a = x / n, b = x - a * n;
                if (((Sm >> a) & 1u) && (b == a || !((Sm >> b) & 1u))) {
                    const uint32_t T = (Sm & ~(1u << a)) | (1u << b);
                    const int64_t t = cz_rank(T, binom);
                    const int64_t cr = __ldg(Cint + 2 * t), ci = __ldg(Cint + 2 * t + 1);
                    const bool neg = cz_sign(Sm, a, b);
                    vr = neg ? -cr : cr;
                    vi = neg ? -ci : ci;
                }
            }
            y[2 * e] = (uint64_t)vr + bias;
            y[2 * e + 1] = (uint64_t)vi + bias;
        }
        uint8_t *base = Dimg + (size_t)blk * S * CZ_B_PLANE + ((row >> 3) * 4 + cc) * 128 + (row & 7) * 16;
#pragma unroll
        for (int j = 0; j < S; ++j) {
            uint4 w;
            w.x = digits7_f16x2(y[0], y[1], j);
            w.y = digits7_f16x2(y[2], y[3], j);
            w.z = digits7_f16x2(y[4], y[5], j);
            w.w = digits7_f16x2(y[6], y[7], j);
            *(uint4 *)(base + j * CZ_B_PLANE) = w;
        }
    }
}

// sigma_I = scale * sum over the replacements of I of sign * E_int[x, T] (complex parts in
// rows 2x and 2x + 1 of the tile-major E image) + e_core C_I.
__global__ void __launch_bounds__(128) k_cz_scatter(int n, int64_t ndet, int M_pad, const uint64_t *__restrict__ str,
                                                    const uint64_t *__restrict__ binom,
                                                    const int64_t *__restrict__ E, const double *__restrict__ C,
                                                    double e_core, int ushift, const int *__restrict__ shC,
                                                    const int *__restrict__ status, double *__restrict__ sigma) {
    const int64_t I = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (I >= ndet) return;
    const int u = ushift - *shC;
    const bool bad = *status != 0;
    const uint32_t Sm = (uint32_t)str[I];
    int64_t ar = 0, ai = 0;
    for (int a = 0; a < n; ++a) {
        if (!((Sm >> a) & 1u)) continue;
        for (int b = 0; b < n; ++b) {
            if (b != a && ((Sm >> b) & 1u)) continue;
            const uint32_t T = (Sm & ~(1u << a)) | (1u << b);
            const int64_t t = cz_rank(T, binom);
            const int x = a * n + b;
            const int64_t *e = E + ((t / CZ_N) * M_pad + 2 * x) * CZ_N + (t % CZ_N);
            const int64_t er = __ldg(e), ei = __ldg(e + CZ_N);
            if (cz_sign(Sm, a, b)) { ar -= er; ai -= ei; } else { ar += er; ai += ei; }
        }
    }
    const double cr = C[2 * I], ci = C[2 * I + 1];
    if (bad) {
        sigma[2 * I] = sigma[2 * I + 1] = __longlong_as_double(0x7FF8000000000000ll);
    } else {
        sigma[2 * I] = scalbn(__ll2double_rn(ar), u) + e_core * cr;
        sigma[2 * I + 1] = scalbn(__ll2double_rn(ai), u) + e_core * ci;
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

struct CzGeom {
    int M_real, M_pad, K_pad, n_mt, n_kc, ring;
    int64_t n_nt;
    size_t smem;
};

void cz_geom(const fci_context *h, int s, CzGeom &g) {
    const int n2 = h->n_orb * h->n_orb;
    g.M_real = 2 * n2;
    g.M_pad = (g.M_real + CZ_M - 1) / CZ_M * CZ_M;
    g.K_pad = (g.M_real + CZ_KC - 1) / CZ_KC * CZ_KC;
    g.n_mt = g.M_pad / CZ_M;
    g.n_kc = g.K_pad / CZ_KC;
    g.n_nt = (h->ndet + CZ_N - 1) / CZ_N;
    const size_t stage = (size_t)s * (CZ_A_PLANE + CZ_B_PLANE);
    const size_t fixed = 1024 + sizeof(CzShared) + 64;
    g.ring = (int)std::min<size_t>(CZ_MAX_STAGES, (CZ_SMEM_MAX - fixed) / stage);
    g.smem = fixed + (size_t)g.ring * stage;
}

int cz_num_sms(fci_context *h, int *nsm) {
    FCI_CUDA(h, cudaDeviceGetAttribute(nsm, cudaDevAttrMultiProcessorCount, h->device));
    return FCI_OK;
}

template <int S>
void (*cz_gemm_kernel())(const CzParams) { return k_cz_gemm<S>; }

}  // namespace

int cz_check(fci_context *h, int s) {
    if (h->mode != FCI_MODE_SPINOR) return fci_fail(h, FCI_ERR_UNSUPPORTED, "complex split path needs spinor strings");
    if (s < 2 || s > CZ_MAXS) return fci_fail(h, FCI_ERR_UNSUPPORTED, "the complex split path takes 2..%d slices", CZ_MAXS);
    if (h->n_orb > 32) return fci_fail(h, FCI_ERR_UNSUPPORTED, "more than 32 spinors");
    const int64_t nnz = 2 * (int64_t)h->na * (h->n_orb - h->na + 1);  // nonzeros of a real-embedded D column
    if ((int64_t)s * nnz * 4096 >= ((int64_t)1 << 24))
        return fci_fail(h, FCI_ERR_UNSUPPORTED, "%d slices x %lld nonzero terms could exceed 2^24 in a level sum", s,
                        (long long)nnz);
    CzGeom g;
    cz_geom(h, s, g);
    if (g.ring < 2) return fci_fail(h, FCI_ERR_UNSUPPORTED, "%d slices do not fit two pipeline stages", s);
    return FCI_OK;
}

// Real-embedded G digit image, tiles [M-tile][K-chunk][plane][128 x 32 core matrices].
static int cz_prepare_G(fci_context *h, int s) {
    if (h->Gs_slices == s && h->d_Gs) return FCI_OK;
    CzGeom g;
    cz_geom(h, s, g);
    const int n2 = h->n_orb * h->n_orb;
    std::vector<double> G((size_t)n2 * n2 * 2);
    if (cudaMemcpy(G.data(), h->d_G, G.size() * 8, cudaMemcpyDeviceToHost) != cudaSuccess)
        return fci_cuda_check(h, cudaGetLastError(), "G download");
    double gmax = 0.0;
    for (double v : G) gmax = std::max(gmax, fabs(v));
    int eG = 0;
    if (gmax > 0) frexp(gmax, &eG);
    const int shG = 7 * s - 2 - eG;
    uint64_t bias = 0;
    for (int j = 0; j < s; ++j) bias |= (uint64_t)64 << (7 * j);
    const size_t stageA = (size_t)s * CZ_A_PLANE;
    std::vector<uint16_t> img((size_t)g.n_mt * g.n_kc * stageA / 2, 0);
    for (int m = 0; m < g.M_pad; ++m) {
        const int mt = m / CZ_M, r = m % CZ_M;
        for (int k = 0; k < g.K_pad; ++k) {
            double v = 0.0;
            if (m < g.M_real && k < g.M_real) {
                const int x = m >> 1, u = m & 1, y = k >> 1, w = k & 1;  // complex row x, column y
                const double gr = G[2 * ((size_t)x * n2 + y)], gi = G[2 * ((size_t)x * n2 + y) + 1];
                v = (u == w) ? gr : (u == 0 ? -gi : gi);
            }
            const int64_t gi64 = llrint(ldexp(v, shG));
            const uint64_t yb = (uint64_t)gi64 + bias;
            const int kc = k / CZ_KC, kk = k % CZ_KC;
            const size_t off = ((size_t)mt * g.n_kc + kc) * stageA + ((r >> 3) * 4 + (kk >> 3)) * 128 + (r & 7) * 16 +
                               (kk & 7) * 2;
            for (int j = 0; j < s; ++j)
                img[(off + (size_t)j * CZ_A_PLANE) / 2] = half_bits_of_small_int((int)((yb >> (7 * j)) & 0x7F) - 64);
        }
    }
    fci_dev_free(h->d_Gs);
    h->d_Gs = nullptr;
    h->Gs_slices = 0;
    int rc = fci_dev_alloc(h, &h->d_Gs, img.size() * 2);
    if (rc) return rc;
    FCI_CUDA(h, cudaMemcpy(h->d_Gs, img.data(), img.size() * 2, cudaMemcpyHostToDevice));
    h->Gs_slices = s;
    h->G_exp = shG;
    return FCI_OK;
}

size_t cz_workspace_bytes(const fci_context *h, int s) {
    CzGeom g;
    cz_geom(h, s < 2 ? 2 : s, g);
    return al256((size_t)h->ndet * 16) + al256((size_t)g.n_nt * g.n_kc * s * CZ_B_PLANE) +
           al256((size_t)g.n_nt * g.M_pad * CZ_N * 8) + 256;
}

int cz_sigma(fci_context *h, const double *C, double *sigma, int s, void *ws, size_t ws_bytes, cudaStream_t st) {
    (void)ws_bytes;
    int rc = cz_check(h, s);
    if (!rc) rc = cz_prepare_G(h, s);
    if (rc) return rc;
    CzGeom g;
    cz_geom(h, s, g);
    char *p = (char *)ws;
    int64_t *Cint = (int64_t *)p;
    p += al256((size_t)h->ndet * 16);
    uint8_t *Dimg = (uint8_t *)p;
    p += al256((size_t)g.n_nt * g.n_kc * s * CZ_B_PLANE);
    int64_t *E = (int64_t *)p;
    p += al256((size_t)g.n_nt * g.M_pad * CZ_N * 8);
    unsigned long long *maxbits = (unsigned long long *)p;
    int *shC = (int *)(p + 8), *status = (int *)(p + 16);
    h->last_status = status;
    {
        phase_scope ps(h, st, FCI_PHASE_GATHER, 3);
        FCI_CUDA(h, cudaMemsetAsync(p, 0, 256, st));
        const unsigned nb = (unsigned)std::min<int64_t>(ceil_div(2 * h->ndet, 256), 152 * 8);
        k_cz_absmax<<<nb, 256, 0, st>>>(C, 2 * h->ndet, maxbits);
        k_cz_to_fixed<<<nb, 256, 0, st>>>(C, 2 * h->ndet, s, maxbits, Cint, shC);
        const int64_t nblk = g.n_nt * g.n_kc;
        const unsigned gb = (unsigned)std::min<int64_t>(nblk, 152 * 16);
        switch (s) {
#define CZ_SPLIT(S_) case S_: k_cz_split<S_><<<gb, 256, 0, st>>>(h->n_orb, h->ndet, g.n_kc, nblk, h->d_str_a, h->d_binom, Cint, Dimg); break;
            CZ_SPLIT(2) CZ_SPLIT(3) CZ_SPLIT(4) CZ_SPLIT(5) CZ_SPLIT(6) CZ_SPLIT(7) CZ_SPLIT(8)
#undef CZ_SPLIT
        }
        FCI_CUDA(h, cudaGetLastError());
    }
    {
        void (*kern)(const CzParams) = nullptr;
        switch (s) {
            case 2: kern = cz_gemm_kernel<2>(); break;
            case 3: kern = cz_gemm_kernel<3>(); break;
            case 4: kern = cz_gemm_kernel<4>(); break;
            case 5: kern = cz_gemm_kernel<5>(); break;
            case 6: kern = cz_gemm_kernel<6>(); break;
            case 7: kern = cz_gemm_kernel<7>(); break;
            case 8: kern = cz_gemm_kernel<8>(); break;
        }
        CzParams prm;
        prm.n_mt = g.n_mt;
        prm.n_kc = g.n_kc;
        prm.M_pad = g.M_pad;
        prm.ring = g.ring;
        prm.n_nt = g.n_nt;
        prm.Gimg = (const uint8_t *)h->d_Gs;
        prm.Dimg = Dimg;
        prm.E = E;
        prm.status = status;
        const char *to = getenv("FCI_WAIT_TIMEOUT_MS");
        prm.timeout_cycles = (long long)((to ? atof(to) : 2000.0) * 2.1e6);
        int nsm = 0;
        if ((rc = cz_num_sms(h, &nsm))) return rc;
        const int64_t units = g.n_nt * g.n_mt;
        FCI_CUDA(h, cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)g.smem));
        phase_scope ps(h, st, FCI_PHASE_CONTRACT, 1);
        kern<<<(unsigned)std::min<int64_t>(nsm, units), CZ_THREADS, g.smem, st>>>(prm);
        FCI_CUDA(h, cudaGetLastError());
    }
    {
        phase_scope ps(h, st, FCI_PHASE_SCATTER, 1);
        const int L0 = std::max(s - 1, 2 * s - 7);
        k_cz_scatter<<<(unsigned)ceil_div(h->ndet, 128), 128, 0, st>>>(h->n_orb, h->ndet, g.M_pad, h->d_str_a,
                                                                        h->d_binom, E, C, h->e_core,
                                                                        7 * L0 - h->G_exp, shC, status, sigma);
        FCI_CUDA(h, cudaGetLastError());
    }
    return FCI_OK;
}
