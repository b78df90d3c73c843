// Complex (two-spinor) sigma build: one string of n spinors per determinant, complex
// Hermitian integrals (the relativistic case of the paper's Results; X2C two-spinors).
//   D[pq,K] = sum_J <K|E_pq|J> C_J      pq = p*n + q (no pair packing for complex g)
//   E = G D                             G = 1/2 g' ([n^2][n^2], complex FP64)
//   sigma_I = e_core C_I + sum_{pq,K} <I|E_pq|K> E[pq,K]
// Single replacements are regenerated from the string masks (ranking by popc over the
// set bits) instead of being stored: at 24 spinors / 12 electrons the stored list
// would be 3.4 GB.
#include <algorithm>

#include "fci_internal.h"

namespace {

__device__ __forceinline__ uint32_t rank_serial(uint32_t T, const uint64_t *__restrict__ binom) {
    uint32_t r = 0;
    int j = 1;
    while (T) {
        const int p = __ffs(T) - 1;
        r += (uint32_t)__ldg(binom + p * FCI_BINOM_LD + j);
        ++j;
        T &= T - 1;
    }
    return r;
}

__device__ __forceinline__ int sign_between(uint32_t S, int a, int b) {
    const int lo = a < b ? a : b, hi = a < b ? b : a;
    const uint32_t between = (hi > lo + 1) ? (((1u << hi) - 1u) & ~((2u << lo) - 1u)) : 0u;
    return __popc(S & between) & 1;
}

// Thread per determinant K; writes the full column D[:, K] (zeros included).
__global__ void __launch_bounds__(256) k_gather_spinor(int n, int64_t ns, const uint64_t *__restrict__ str,
                                                       const uint64_t *__restrict__ binom,
                                                       const double2 *__restrict__ C, double2 *__restrict__ D) {
    const int64_t K = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (K >= ns) return;
    const uint32_t S = (uint32_t)str[K];
    for (int a = 0; a < n; ++a) {
        const bool occ = (S >> a) & 1u;
        for (int b = 0; b < n; ++b) {
            double2 v = make_double2(0.0, 0.0);
            if (occ && (b == a || !((S >> b) & 1u))) {
                const uint32_t T = (S & ~(1u << a)) | (1u << b);
                const double2 c = __ldg(C + rank_serial(T, binom));
                v = sign_between(S, a, b) ? make_double2(-c.x, -c.y) : c;
            }
            D[(int64_t)(a * n + b) * ns + K] = v;
        }
    }
}

__global__ void __launch_bounds__(256) k_scatter_spinor(int n, int64_t ns, const uint64_t *__restrict__ str,
                                                        const uint64_t *__restrict__ binom,
                                                        const double2 *__restrict__ E,
                                                        const double2 *__restrict__ C, double e_core,
                                                        double2 *__restrict__ sigma) {
    const int64_t I = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (I >= ns) return;
    const uint32_t S = (uint32_t)str[I];
    double sx = 0.0, sy = 0.0;
    for (int a = 0; a < n; ++a) {
        if (!((S >> a) & 1u)) continue;
        for (int b = 0; b < n; ++b) {
            if (b != a && ((S >> b) & 1u)) continue;
            const uint32_t T = (S & ~(1u << a)) | (1u << b);
            const double2 e = __ldg(E + (int64_t)(a * n + b) * ns + rank_serial(T, binom));
            if (sign_between(S, a, b)) { sx -= e.x; sy -= e.y; } else { sx += e.x; sy += e.y; }
        }
    }
    const double2 c = C[I];
    sigma[I] = make_double2(sx + e_core * c.x, sy + e_core * c.y);
}

// Complex C[M x N] = A[M x K] B[K x N] (row-major, interleaved).  32 x 64 tiles, 256
// threads each owning 2 x 4 complex outputs.
constexpr int ZM = 32, ZN = 64, ZK = 8;
__global__ void __launch_bounds__(256) k_zgemm(int M, int64_t N, int K, const double2 *__restrict__ A,
                                               const double2 *__restrict__ B, int64_t ldb,
                                               double2 *__restrict__ Cm, int64_t ldc) {
    __shared__ double2 sA[ZK][ZM + 1];
    __shared__ double2 sB[ZK][ZN];
    const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
    const int m0 = blockIdx.y * ZM;
    const int64_t n0 = blockIdx.x * (int64_t)ZN;
    double2 acc[2][4];
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = make_double2(0.0, 0.0);
    for (int k0 = 0; k0 < K; k0 += ZK) {
        for (int i = threadIdx.x; i < ZK * ZM; i += 256) {
            int kk = i % ZK, mm = i / ZK;
            int gm = m0 + mm, gk = k0 + kk;
            sA[kk][mm] = (gm < M && gk < K) ? A[(int64_t)gm * K + gk] : make_double2(0.0, 0.0);
        }
        for (int i = threadIdx.x; i < ZK * ZN; i += 256) {
            int kk = i / ZN, nn = i % ZN;
            int64_t gn = n0 + nn;
            int gk = k0 + kk;
            sB[kk][nn] = (gn < N && gk < K) ? B[(int64_t)gk * ldb + gn] : make_double2(0.0, 0.0);
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < ZK; ++kk) {
            double2 a[2], b[4];
#pragma unroll
            for (int i = 0; i < 2; ++i) a[i] = sA[kk][ty * 2 + i];
#pragma unroll
            for (int j = 0; j < 4; ++j) b[j] = sB[kk][tx + 16 * j];
#pragma unroll
            for (int i = 0; i < 2; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    acc[i][j].x = fma(a[i].x, b[j].x, fma(-a[i].y, b[j].y, acc[i][j].x));
                    acc[i][j].y = fma(a[i].x, b[j].y, fma(a[i].y, b[j].x, acc[i][j].y));
                }
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 2; ++i) {
        int gm = m0 + ty * 2 + i;
        if (gm >= M) continue;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            int64_t gn = n0 + tx + 16 * j;
            if (gn < N) Cm[(int64_t)gm * ldc + gn] = acc[i][j];
        }
    }
}

__global__ void k_diag_spinor(int64_t ns, int n, const uint64_t *__restrict__ str, const double *__restrict__ hd,
                              const double *__restrict__ J, const double *__restrict__ K, double e_core,
                              double *__restrict__ diag) {
    for (int64_t I = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; I < ns; I += (int64_t)gridDim.x * blockDim.x) {
        const uint64_t S = str[I];
        double e = e_core;
        for (int p = 0; p < n; ++p) {
            if (!((S >> p) & 1)) continue;
            e += hd[p];
            for (int q = 0; q < n; ++q)
                if ((S >> q) & 1) e += 0.5 * (J[p * n + q] - K[p * n + q]);
        }
        diag[I] = e;
    }
}

}  // namespace

cudaError_t launch_gather_spinor(const fci_context *h, const double *C, double *D, cudaStream_t s) {
    k_gather_spinor<<<(unsigned)ceil_div(h->nsa, 128), 128, 0, s>>>(h->n_orb, h->nsa, h->d_str_a, h->d_binom,
                                                                  (const double2 *)C, (double2 *)D);
    return cudaGetLastError();
}

cudaError_t launch_scatter_spinor(const fci_context *h, const double *E, const double *C, double *sigma,
                                  cudaStream_t s) {
    k_scatter_spinor<<<(unsigned)ceil_div(h->nsa, 128), 128, 0, s>>>(h->n_orb, h->nsa, h->d_str_a, h->d_binom,
                                                                   (const double2 *)E, (const double2 *)C,
                                                                   h->e_core, (double2 *)sigma);
    return cudaGetLastError();
}

cudaError_t launch_zgemm(int M, int64_t N, int K, const double *A, const double *B, int64_t ldb, double *C,
                         int64_t ldc, cudaStream_t s) {
    if (M <= 0 || N <= 0) return cudaSuccess;
    dim3 grid((unsigned)ceil_div(N, ZN), (unsigned)ceil_div(M, ZM));
    k_zgemm<<<grid, 256, 0, s>>>(M, N, K, (const double2 *)A, (const double2 *)B, ldb, (double2 *)C, ldc);
    return cudaGetLastError();
}

cudaError_t launch_diag_spinor(const fci_context *h, double *diag, cudaStream_t s) {
    unsigned blocks = (unsigned)std::min<int64_t>(ceil_div(h->nsa, 256), 152 * 32);
    k_diag_spinor<<<blocks, 256, 0, s>>>(h->nsa, h->n_orb, h->d_str_a, h->d_hd, h->d_J, h->d_K, h->e_core, diag);
    return cudaGetLastError();
}
