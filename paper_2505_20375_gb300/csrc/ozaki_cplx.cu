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
// The GEMM itself is the shared bulk-copy kernel (ozaki_gemm.cu) with 7-bit digits.
#include <math.h>
#include <stdlib.h>

#include <algorithm>
#include <complex>
#include <vector>

#include "fci_internal.h"
#include "oz_gemm.cuh"
#include "tc_ptx.cuh"

namespace {

using namespace tc;

constexpr int CZ_M = OZG_M;
constexpr int CZ_N = OZG_N;
constexpr int CZ_KC = OZG_KC;
constexpr int CZ_A_PLANE = OZG_A_PLANE;
constexpr int CZ_B_PLANE = OZG_B_PLANE;
constexpr int CZ_MAXS = OZG_MAXS;

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
            __stcs((uint4 *)(base + j * CZ_B_PLANE), w);  // streaming: keep C_int in L2
        }
    }
}

// sigma_I = scale * sum over the replacements of I of sign * E_int[x, T] (complex parts in
// rows 2x and 2x + 1 of the tile-major E image) + e_core C_I.
__global__ void __launch_bounds__(128) k_cz_scatter(int n, int64_t ndet, int M_pad, const uint64_t *__restrict__ str,
                                                    const uint64_t *__restrict__ binom,
                                                    const int64_t *__restrict__ E, const double *__restrict__ C,
                                                    double e_core, int ushift, const int *__restrict__ shC,
                                                    const int *__restrict__ status, int *__restrict__ sticky,
                                                    double *__restrict__ sigma) {
    const int64_t I = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (I >= ndet) return;
    const int u = ushift - *shC;
    const bool bad = *status != 0;
    if (bad && I == 0) atomicExch(sticky, *status);  // kept for fci_sync_status
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
    int M_real, M_pad, K_pad, n_mt, n_kc;
    int64_t n_nt;
};

void cz_geom(const fci_context *h, CzGeom &g) {
    const int n2 = h->n_orb * h->n_orb;
    g.M_real = 2 * n2;
    g.M_pad = (g.M_real + CZ_M - 1) / CZ_M * CZ_M;
    g.K_pad = (g.M_real + CZ_KC - 1) / CZ_KC * CZ_KC;
    g.n_mt = g.M_pad / CZ_M;
    g.n_kc = g.K_pad / CZ_KC;
    g.n_nt = (h->ndet + CZ_N - 1) / CZ_N;
}

}  // namespace

int cz_check(fci_context *h, int s) {
    if (h->mode != FCI_MODE_SPINOR) return fci_fail(h, FCI_ERR_UNSUPPORTED, "complex split path needs spinor strings");
    if (s < 2 || s > CZ_MAXS) return fci_fail(h, FCI_ERR_UNSUPPORTED, "the complex split path takes 2..%d slices", CZ_MAXS);
    if (h->n_orb > 32) return fci_fail(h, FCI_ERR_UNSUPPORTED, "more than 32 spinors");
    const int64_t nnz = 2 * (int64_t)h->na * (h->n_orb - h->na + 1);  // nonzeros of a real-embedded D column
    if ((int64_t)s * nnz * 4096 >= ((int64_t)1 << 24))
        return fci_fail(h, FCI_ERR_UNSUPPORTED, "%d slices x %lld nonzero terms could exceed 2^24 in a level sum", s,
                        (long long)nnz);
    if (!oz_gemm_ring(s, 4, 0)) return fci_fail(h, FCI_ERR_UNSUPPORTED, "%d slices do not fit two pipeline stages", s);
    return FCI_OK;
}

// Real-embedded G digit image, tiles [M-tile][K-chunk][plane][128 x 32 core matrices].
static int cz_prepare_G(fci_context *h, int s) {
    if (h->Gs_slices == s && h->d_Gs) return FCI_OK;
    CzGeom g;
    cz_geom(h, g);
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
    cz_geom(h, g);
    return al256((size_t)h->ndet * 16) + al256((size_t)g.n_nt * g.n_kc * s * CZ_B_PLANE) +
           al256((size_t)g.n_nt * g.M_pad * CZ_N * 8) + 256;
}

int cz_sigma(fci_context *h, const double *C, double *sigma, int s, void *ws, size_t ws_bytes, cudaStream_t st) {
    (void)ws_bytes;
    int rc = cz_check(h, s);
    if (!rc) rc = cz_prepare_G(h, s);
    if (rc) return rc;
    CzGeom g;
    cz_geom(h, g);
    char *p = (char *)ws;
    int64_t *Cint = (int64_t *)p;
    p += al256((size_t)h->ndet * 16);
    uint8_t *Dimg = (uint8_t *)p;
    p += al256((size_t)g.n_nt * g.n_kc * s * CZ_B_PLANE);
    int64_t *E = (int64_t *)p;
    p += al256((size_t)g.n_nt * g.M_pad * CZ_N * 8);
    unsigned long long *maxbits = (unsigned long long *)p;
    int *shC = (int *)(p + 8), *status = (int *)(p + 16);
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
        oz_gemm_args a;
        a.n_mt = g.n_mt;
        a.n_kc = g.n_kc;
        a.M_pad = g.M_pad;
        a.M_real = g.M_real;
        a.n_nt = g.n_nt;
        a.Gimg = h->d_Gs;
        a.Dimg = Dimg;
        a.E = E;
        a.status = status;
        if ((rc = oz_gemm_launch(h, s, 7, 4, false, a, st))) return rc;
    }
    {
        phase_scope ps(h, st, FCI_PHASE_SCATTER, 1);
        const int L0 = oz_gemm_L0(s, 7);
        k_cz_scatter<<<(unsigned)ceil_div(h->ndet, 128), 128, 0, st>>>(h->n_orb, h->ndet, g.M_pad, h->d_str_a,
                                                                        h->d_binom, E, C, h->e_core,
                                                                        7 * L0 - h->G_exp, shC, status, h->d_status,
                                                                        sigma);
        FCI_CUDA(h, cudaGetLastError());
    }
    return FCI_OK;
}
