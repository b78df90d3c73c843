// Kernel layout (one persistent CTA per SM, 32 (1 + OZG_ISSUERS + 8 or 16) threads):
//   warp 0     lane 0 issues the two bulk copies of each pipeline stage (A tile: s planes
//              of 128 x 32, B tile: s planes of 64 x 32), completing on the stage's mbarrier;
//   warps 1 .. OZG_ISSUERS   lane 0 of each issues the MMAs (M = 128, N = 64, K = 16) of
//              its share of the s level accumulators and commits (warp 1 also allocates
//              TMEM): issuing threads on different SM sub-partitions, because one thread
//              issuing every MMA was measured at about 77 cycles per MMA against 48 for the
//              bare instruction stream; the levels are dealt so that every issuer issues
//              about as many MMAs (level l takes s - l products; ozg_issuer);
//   the rest   epilogue: 8 warps (two per TMEM lane quadrant, 32 columns each) when the
//              accumulators are double-buffered (s <= 4), else 16 (four per quadrant,
//              16 columns each), which read the levels three at a time and release each
//              group as soon as it is in registers.
// Level accumulators are double-buffered when 2 s x 64 TMEM columns fit in 512; otherwise
// the first K-chunk of a unit issues the MMAs of each level group once the epilogue has
// released it.  Work units
// are (N-tile, M-tile) pairs, N-tile outer and dealt round-robin, so the M-tiles of one
// B tile run at about the same time and its reads hit L2.  Every mbarrier wait is bounded
// in time (FCI_ERR_TIMEOUT in the status word on expiry; the kernel then waits, under a
// bound of its own, for the bulk copies and MMAs it issued, and frees TMEM before
// returning).
#include <stdlib.h>

#include <algorithm>
#include <type_traits>

#include "oz_gemm.cuh"
#include "tc_ptx.cuh"

namespace {

using namespace tc;

// Epilogue warps: 8 (two per TMEM lane quadrant, 32 columns each) when the level
// accumulators are double-buffered, 16 (four per quadrant, 16 columns each) otherwise.
__host__ __device__ constexpr int ozg_epi_warps(int s) { return 2 * s * OZG_N <= 512 ? 8 : 16; }
constexpr int OZG_ISSUERS = 2;
__host__ __device__ constexpr int ozg_threads(int s) { return 32 * (1 + OZG_ISSUERS + ozg_epi_warps(s)); }
// The MMA issuer of level l of s (level l takes s - l products): levels in order of their
// product counts, each to the issuer with the fewest products so far.
__host__ __device__ constexpr int ozg_issuer(int s, int l) {
    int load[OZG_ISSUERS] = {};
    int who = 0;
    for (int k = 0; k <= l; ++k) {
        int m = 0;
        for (int e = 1; e < OZG_ISSUERS; ++e)
            if (load[e] < load[m]) m = e;
        load[m] += s - k;
        who = m;
    }
    return who;
}
constexpr int OZG_MAX_STAGES = 6;
constexpr size_t OZG_SMEM_MAX = 232448 - 1024;

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

struct OzgParams {
    int n_mt, n_kc, M_pad, M_real, ring;
    int64_t n_nt;
    const uint8_t *Gimg, *Dimg;
    int64_t *E;
    int *status;
    long long timeout_cycles;
    int stall_test;  // test hook: the MMA thread issues nothing, so the producer's wait expires
};

struct OzgShared {
    uint64_t full[OZG_MAX_STAGES], empty[OZG_MAX_STAGES];
    uint64_t acc_full[2], acc_empty[OZG_MAXS];  // acc_empty: per buffer, or per level group (one buffer)
    uint64_t drain, a_full;
    uint32_t tmem_base;
    int abort;
};

template <bool FAST = false>
__device__ __forceinline__ bool ozg_wait(uint32_t bar, uint32_t parity, volatile int *abort, int *status,
                                        long long timeout) {
    if (FAST && mbar_test_wait(bar, parity)) return true;
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

// Wait for a phase that must complete (copies or MMAs already issued) before the CTA may
// leave: bounded like every other wait, but blind to the abort flag.
__device__ __forceinline__ bool ozg_drain_wait(uint32_t bar, uint32_t parity, int *status, long long timeout) {
    const long long t0 = clock64();
    while (!mbar_try_wait(bar, parity)) {
        if (clock64() - t0 > timeout) {
            atomicExch(status, FCI_ERR_TIMEOUT);
            return false;
        }
    }
    return true;
}

template <bool FAST = false>
__device__ __forceinline__ bool ozg_wait_warp(uint32_t bar, uint32_t parity, volatile int *abort, int *status,
                                             long long timeout) {
    int ok = 0;
    if ((threadIdx.x & 31) == 0) ok = ozg_wait<FAST>(bar, parity, abort, status, timeout) ? 1 : 0;
    return __shfl_sync(0xFFFFFFFFu, ok, 0) != 0;
}

// S slices, W-bit digits, KCC core matrices (8 K each) per pipeline stage, RESA: the whole
// A image (one M-tile) is loaded into shared memory once and only B tiles stream.
template <int S, int W, int KCC, bool RESA>
__global__ void __launch_bounds__(ozg_threads(S), 1) k_oz_gemm(const __grid_constant__ OzgParams p) {
    constexpr int NBUF = (2 * S * OZG_N <= 512) ? 2 : 1;
    // With one accumulator buffer the epilogue releases the levels in groups of GH as it
    // reads them, and the next unit's first K-chunk issues each group's MMAs once that
    // group is free.
    constexpr int GH = 3;
    constexpr int NG = NBUF == 1 ? (S + GH - 1) / GH : 1;
    constexpr int L0 = oz_gemm_L0(S, W);
    constexpr uint32_t A_PLANE = OZG_M * KCC * 16, B_PLANE = OZG_N * KCC * 16;
    constexpr uint32_t STAGE_A = S * A_PLANE, STAGE_B = S * B_PLANE;
    constexpr uint32_t STAGE_LOAD = RESA ? STAGE_B : STAGE_A + STAGE_B;
    extern __shared__ __align__(1024) uint8_t cz_smem_raw[];
    uint8_t *smem = (uint8_t *)(((uintptr_t)cz_smem_raw + 1023) & ~(uintptr_t)1023);
    const int R = p.ring;
    // RESA: A region = n_kc x STAGE_A (every K-chunk of the single M-tile); else R stages
    uint8_t *sA = smem;
    uint8_t *sB = sA + (RESA ? (size_t)p.n_kc * STAGE_A : (size_t)R * STAGE_A);  // R stages of S B-planes
    OzgShared *sh = (OzgShared *)(sB + (size_t)R * STAGE_B);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        for (int r = 0; r < R; ++r) {
            mbar_init(smem_u32(&sh->full[r]), 1);
            mbar_init(smem_u32(&sh->empty[r]), OZG_ISSUERS);  // every issuer's MMAs of the stage done
        }
        for (int b = 0; b < 2; ++b) mbar_init(smem_u32(&sh->acc_full[b]), OZG_ISSUERS);
        for (int b = 0; b < OZG_MAXS; ++b) mbar_init(smem_u32(&sh->acc_empty[b]), ozg_epi_warps(S));
        mbar_init(smem_u32(&sh->drain), OZG_ISSUERS);
        mbar_init(smem_u32(&sh->a_full), 1);
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
            if (RESA) {  // the whole A image, in pieces of at most 32 KB, on its own barrier
                const uint32_t total = (uint32_t)p.n_kc * STAGE_A, ab = smem_u32(&sh->a_full);
                mbar_expect_tx(ab, total);
                for (uint32_t o = 0; o < total; o += 32768u)
                    bulk_g2s(smem_u32(sA + o), p.Gimg + o, total - o < 32768u ? total - o : 32768u, ab);
            }
            uint32_t q = 0, st = 0, ph = 0;  // stage counter, its ring slot and the slot's use parity
            for (int64_t u = blockIdx.x; u < n_units; u += gridDim.x) {
                const int64_t nt = u / p.n_mt;
                const int mt = (int)(u - nt * p.n_mt);
                const uint8_t *ga = p.Gimg + (size_t)mt * p.n_kc * STAGE_A;
                const uint8_t *gb = p.Dimg + (size_t)nt * p.n_kc * STAGE_B;
                bool ok = true;
                for (int kc = 0; kc < p.n_kc; ++kc, ++q) {
                    if (q >= (uint32_t)R &&
                        !ozg_wait<true>(smem_u32(&sh->empty[st]), ph ^ 1, abort, p.status, p.timeout_cycles)) {
                        ok = false;
                        break;
                    }
                    const uint32_t fb = smem_u32(&sh->full[st]);
                    mbar_expect_tx(fb, STAGE_LOAD);
                    if (!RESA) bulk_g2s(smem_u32(sA + (size_t)st * STAGE_A), ga + (size_t)kc * STAGE_A, STAGE_A, fb);
                    bulk_g2s(smem_u32(sB + (size_t)st * STAGE_B), gb + (size_t)kc * STAGE_B, STAGE_B, fb);
                    if (++st == (uint32_t)R) {
                        st = 0;
                        ph ^= 1;
                    }
                }
                if (!ok) break;
            }
            // Every copy issued must land before the CTA leaves, also after an abort (the
            // copies of the stages the MMA thread never consumed are still in flight): wait
            // for the last use of each ring slot, and for the resident A image.
            const uint32_t used = q < (uint32_t)R ? q : (uint32_t)R;
            for (uint32_t k = 1; k <= used; ++k) {
                const uint32_t idx = q - k;
                ozg_drain_wait(smem_u32(&sh->full[idx % (uint32_t)R]), (idx / (uint32_t)R) & 1u, p.status,
                               p.timeout_cycles);
            }
            if (RESA) ozg_drain_wait(smem_u32(&sh->a_full), 0, p.status, p.timeout_cycles);
        }
    } else if (warp <= OZG_ISSUERS) {
        // ---------------------------------------------------------------- MMA issuers
        // ME (a compile-time copy of warp - 1): this thread issues the levels l with
        // ozg_issuer(S, l) == ME, so each issuer's instruction stream holds its MMAs only.
        auto issuer = [&](auto me_c) {
            constexpr int ME = decltype(me_c)::value;
            // The ring slot and its parity advance with each stage (no division on the
            // issue path), and each wait first tests the barrier without blocking.
            auto wait = [&](uint32_t bar, uint32_t par) -> bool {
                return ozg_wait<true>(bar, par, abort, p.status, p.timeout_cycles);
            };
            const uint32_t idesc = idesc_f16(OZG_M, OZG_N);
            const uint64_t a0 = smem_desc(smem_u32(sA), 128, KCC * 128);
            const uint64_t b0 = smem_desc(smem_u32(sB), 128, KCC * 128);
            uint32_t st = 0, ph = 0, tau = 0;  // ring slot, its use parity, unit counter
            bool issued = false, ok = !p.stall_test;
            if (ok && RESA && !wait(smem_u32(&sh->a_full), 0)) ok = false;
            for (int64_t u = blockIdx.x; u < n_units && ok; u += gridDim.x, ++tau) {
                const int buf = NBUF == 2 ? (int)(tau & 1) : 0;
                if (NBUF == 2 && tau >= 2) {
                    if (!wait(smem_u32(&sh->acc_empty[buf]), ((tau >> 1) - 1) & 1)) break;
                    tc_fence_after();
                }
                const uint32_t dbase = tmem + (uint32_t)(buf * S * OZG_N);
                for (int kc = 0; kc < p.n_kc; ++kc) {
                    if (!wait(smem_u32(&sh->full[st]), ph)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const uint64_t as = a0 + (uint64_t)(((RESA ? kc : (int)st) * STAGE_A) >> 4);
                    const uint64_t bs = b0 + (uint64_t)((st * STAGE_B) >> 4);
                    // the MMAs of this K-chunk whose level lies in [lo, hi)
                    auto issue = [&](int lo, int hi) {
#pragma unroll
                        for (int kk = 0; kk < KCC / 2; ++kk) {
#pragma unroll
                            for (int j = S - 1; j >= 0; --j) {
                                const uint64_t b = bs + (uint64_t)((j * B_PLANE + kk * 256) >> 4);
                                const uint32_t acc_in = (kc != 0 || kk != 0 || j != S - 1) ? 1u : 0u;
#pragma unroll
                                for (int i = S - 1 - j; i < S; ++i) {
                                    const int lv = i + j - (S - 1);
                                    if (lv >= lo && lv < hi && ozg_issuer(S, lv) == ME)
                                        mma_f16(dbase + (uint32_t)(lv * OZG_N),
                                                as + (uint64_t)((i * A_PLANE + kk * 256) >> 4), b, idesc, acc_in);
                                }
                            }
                        }
                    };
                    if (NBUF == 1 && kc == 0 && tau >= 1) {
                        bool freed = true;
#pragma unroll
                        for (int g = 0; g < NG; ++g) {
                            if (!wait(smem_u32(&sh->acc_empty[g]), (tau - 1) & 1)) {
                                freed = false;
                                break;
                            }
                            tc_fence_after();
                            issue(g * GH, g * GH + GH);
                        }
                        if (!freed) {
                            ok = false;
                            break;
                        }
                    } else {
                        issue(0, S);
                    }
                    issued = true;
                    mma_commit(smem_u32(&sh->empty[st]));
                    if (++st == (uint32_t)R) {
                        st = 0;
                        ph ^= 1;
                    }
                }
                if (!ok) break;
                mma_commit(smem_u32(&sh->acc_full[buf]));
            }
            // all MMAs issued must complete before TMEM is freed: each issuer arrives on the
            // drain barrier once its MMAs are done (at once if it issued none); if the first
            // budget expires (FCI_ERR_TIMEOUT recorded) a second one follows before the
            // deallocation goes ahead
            if (issued) mma_commit(smem_u32(&sh->drain));
            else mbar_arrive(smem_u32(&sh->drain));
            if (!ozg_drain_wait(smem_u32(&sh->drain), 0, p.status, p.timeout_cycles))
                ozg_drain_wait(smem_u32(&sh->drain), 0, p.status, p.timeout_cycles);
        };
        if (lane == 0) {
            if (warp == 1) issuer(std::integral_constant<int, 0>{});
            else if (OZG_ISSUERS == 2 || warp == 2) issuer(std::integral_constant<int, 1>{});
            else issuer(std::integral_constant<int, (OZG_ISSUERS > 2 ? 2 : 1)>{});
        }
    } else {
        // ---------------------------------------------------------------- epilogue
        // Warp (quadrant qd, part) owns lanes 32 qd .. 32 qd + 31 and 16 CH columns from
        // 16 CH part.  Single-buffered accumulators (s >= 5, CH = 1) are read GH levels at a
        // time; each group is handed back to the MMA warp as soon as it is in registers, so
        // the next unit's first K-chunk starts on it while the rest is read and combined.
        // Double-buffered accumulators (s <= 4, CH = 2) are combined level by level and
        // released at the end.
        constexpr int CH = OZG_N / (4 * ozg_epi_warps(S));  // 16-column chunks per warp: 2 or 1
        const int qd = warp & 3;
        const int cw = 16 * CH * ((warp - 1 - OZG_ISSUERS) >> 2);
        const int row = 32 * qd + lane;
        constexpr int lowshift = W * (L0 - (S - 1));
        uint32_t tau = 0;
        for (int64_t u = blockIdx.x; u < n_units; u += gridDim.x, ++tau) {
            const int64_t nt = u / p.n_mt;
            const int mt = (int)(u - nt * p.n_mt);
            const int buf = NBUF == 2 ? (int)(tau & 1) : 0;
            const uint32_t par = NBUF == 2 ? (tau >> 1) & 1 : tau & 1;
            if (!ozg_wait_warp(smem_u32(&sh->acc_full[buf]), par, abort, p.status, p.timeout_cycles)) break;
            tc_fence_after();
            const uint32_t tl0 = tmem + ((uint32_t)(32 * qd) << 16) + (uint32_t)(buf * S * OZG_N + cw);
            int64_t *dst0 = p.E + ((size_t)nt * p.M_pad + (size_t)mt * OZG_M + row) * OZG_N + cw;
            const bool keep = mt * OZG_M + row < p.M_real;  // rows past the operator's size are never read
            if (NBUF == 1) {  // CH == 1: group by group, each released as soon as it is read
                auto term = [](uint32_t x, int L) -> int64_t {
                    const int64_t v = (int64_t)__float2int_rn(__uint_as_float(x));
                    return L < L0 ? v * ((int64_t)1 << (W * (L - (S - 1)))) : v * ((int64_t)1 << (W * (L - L0)));
                };
                int64_t acc[16];
#pragma unroll
                for (int c = 0; c < 16; ++c) acc[c] = 0;
#pragma unroll
                for (int g = 0; g < NG; ++g) {
                    uint32_t v[GH][16];
#pragma unroll
                    for (int l = g * GH; l < g * GH + GH && l < S; ++l) tmem_ld16(tl0 + (uint32_t)(l * OZG_N), v[l - g * GH]);
                    tmem_ld_wait();
#pragma unroll
                    for (int l = g * GH; l < g * GH + GH && l < S; ++l) tmem_regs_ready(v[l - g * GH]);
                    tc_fence_before();
                    __syncwarp();
                    if (lane == 0) mbar_arrive(smem_u32(&sh->acc_empty[g]));
#pragma unroll
                    for (int l = g * GH; l < g * GH + GH && l < S; ++l) {
                        const int L = S - 1 + l;
#pragma unroll
                        for (int c = 0; c < 16; ++c) {
                            if (L == L0 && lowshift > 0)
                                acc[c] = (acc[c] + ((int64_t)1 << (lowshift > 0 ? lowshift - 1 : 0))) >> lowshift;
                            acc[c] += term(v[l - g * GH][c], L);
                        }
                    }
                }
                if (keep)
#pragma unroll
                    for (int c = 0; c < 16; c += 2) __stcs((longlong2 *)(dst0 + c), make_longlong2(acc[c], acc[c + 1]));
            } else {
                // double-buffered accumulators: combine level by level, release at the end
#pragma unroll 1
                for (int ch = 0; ch < CH; ++ch) {
                    int64_t acc[16];
#pragma unroll
                    for (int c = 0; c < 16; ++c) acc[c] = 0;
#pragma unroll
                    for (int L = S - 1; L <= 2 * S - 2; ++L) {
                        uint32_t v[16];
                        tmem_ld16(tl0 + (uint32_t)((L - (S - 1)) * OZG_N + 16 * ch), v);
                        tmem_ld_wait();
                        tmem_regs_ready(v);
                        if (L < L0) {
#pragma unroll
                            for (int c = 0; c < 16; ++c)
                                acc[c] += (int64_t)__float2int_rn(__uint_as_float(v[c])) * ((int64_t)1 << (W * (L - (S - 1))));
                        } else {
                            if (L == L0 && lowshift > 0) {
#pragma unroll
                                for (int c = 0; c < 16; ++c)
                                    acc[c] = (acc[c] + ((int64_t)1 << (lowshift > 0 ? lowshift - 1 : 0))) >> lowshift;
                            }
#pragma unroll
                            for (int c = 0; c < 16; ++c)
                                acc[c] += (int64_t)__float2int_rn(__uint_as_float(v[c])) * ((int64_t)1 << (W * (L - L0)));
                        }
                    }
                    if (keep)
#pragma unroll
                        for (int c = 0; c < 16; c += 2)
                            __stcs((longlong2 *)(dst0 + 16 * ch + c), make_longlong2(acc[c], acc[c + 1]));
                }
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(smem_u32(&sh->acc_empty[buf]));
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 1) tmem_dealloc(tmem, 512);
}


template <int W, int KCC, bool RESA>
void (*oz_gemm_kernel(int s))(const OzgParams) {
    switch (s) {
        case 2: return k_oz_gemm<2, W, KCC, RESA>;
        case 3: return k_oz_gemm<3, W, KCC, RESA>;
        case 4: return k_oz_gemm<4, W, KCC, RESA>;
        case 5: return k_oz_gemm<5, W, KCC, RESA>;
        case 6: return k_oz_gemm<6, W, KCC, RESA>;
        case 7: return k_oz_gemm<7, W, KCC, RESA>;
        case 8: return k_oz_gemm<8, W, KCC, RESA>;
        default: return nullptr;
    }
}

size_t oz_gemm_fixed() { return 1024 + sizeof(OzgShared) + 64; }

}  // namespace

int oz_gemm_ring(int s, int kcc, int resa_kc) {
    const size_t a_plane = (size_t)OZG_M * kcc * 16, b_plane = (size_t)OZG_N * kcc * 16;
    const size_t resident = resa_kc > 0 ? (size_t)resa_kc * s * a_plane : 0;
    const size_t stage = (size_t)s * ((resa_kc > 0 ? 0 : a_plane) + b_plane);
    const size_t fixed = oz_gemm_fixed() + resident;
    if (fixed >= OZG_SMEM_MAX) return 0;
    const size_t r = (OZG_SMEM_MAX - fixed) / stage;
    return r < 2 ? 0 : (int)std::min<size_t>(OZG_MAX_STAGES, r);
}

int oz_gemm_launch(fci_context *h, int s, int w, int kcc, bool resa, const oz_gemm_args &a, cudaStream_t st) {
    void (*kern)(const OzgParams) = nullptr;
    if (w == 7 && kcc == 4 && !resa) kern = oz_gemm_kernel<7, 4, false>(s);
    if (w == 8 && kcc == 2 && resa) kern = oz_gemm_kernel<8, 2, true>(s);
    if (w == 8 && kcc == 4 && !resa) kern = oz_gemm_kernel<8, 4, false>(s);
    if (resa && a.n_mt != 1) kern = nullptr;
    const int ring = oz_gemm_ring(s, kcc, resa ? a.n_kc : 0);
    if (!kern || !ring) return fci_fail(h, FCI_ERR_UNSUPPORTED, "split GEMM: %d slices of %d bits (K-chunk %d, resident %d)", s, w, 8 * kcc, (int)resa);
    OzgParams prm;
    prm.n_mt = a.n_mt;
    prm.n_kc = a.n_kc;
    prm.M_pad = a.M_pad;
    prm.M_real = a.M_real;
    prm.ring = ring;
    prm.n_nt = a.n_nt;
    prm.Gimg = (const uint8_t *)a.Gimg;
    prm.Dimg = (const uint8_t *)a.Dimg;
    prm.E = a.E;
    prm.status = a.status;
    const char *to = getenv("FCI_WAIT_TIMEOUT_MS");
    prm.timeout_cycles = (long long)((to ? atof(to) : 2000.0) * 2.1e6);
    const char *stall = getenv("FCI_TEST_STALL_PRODUCER");
    prm.stall_test = stall ? atoi(stall) : 0;
    int nsm = 0;
    FCI_CUDA(h, cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, h->device));
    const size_t a_plane = (size_t)OZG_M * kcc * 16, b_plane = (size_t)OZG_N * kcc * 16;
    const size_t smem = oz_gemm_fixed() + (resa ? (size_t)a.n_kc * s * a_plane : 0) +
                        (size_t)ring * s * ((resa ? 0 : a_plane) + b_plane);
    FCI_CUDA(h, cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    const int64_t units = a.n_nt * a.n_mt;
    phase_scope ps(h, st, FCI_PHASE_CONTRACT, 1);
    kern<<<(unsigned)std::max<int64_t>(1, std::min<int64_t>(nsm, units)), ozg_threads(s), smem, st>>>(prm);
    FCI_CUDA(h, cudaGetLastError());
    return FCI_OK;
}
