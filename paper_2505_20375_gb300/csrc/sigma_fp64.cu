// FP64 sigma build for alpha/beta strings (real spin-free orbitals), unfused form:
//   gather  D[pq,K] = sum_J <K|E_pq|J> C_J                  (pair-packed pq)
//   GEMM    E = G D, G = 1/2 g' packed                        (FP64)
//   scatter sigma_I = e_core C_I + sum_{pq,K} <I|E_pq|K> E[pq,K]
// (Methods, Eqs. sigmaL, sigmaL1e, sigmaL2e; the one-electron term is folded into g').
//
// Layouts: C and sigma are [N_alpha][N_beta] row-major; D and E are pair-major
// [n_pair][N_det] so that consecutive threads (consecutive beta strings) touch
// consecutive addresses.  The dense pair tables are [n_pair][N_str]: entry
// (T << 1) | neg for the single replacement of the string that lands on pair pq, or -1.
// Because a string's list never holds both (a,b) and (b,a) for a != b, each packed
// pair has at most one entry per string and spin.
#include <algorithm>

#include "fci_internal.h"

namespace {

__global__ void __launch_bounds__(256) k_gather_fci_r64(int64_t nsa, int64_t nsb, int npair,
                                                        const int32_t *__restrict__ pairA,
                                                        const int32_t *__restrict__ pairB,
                                                        const double *__restrict__ C,
                                                        double *__restrict__ D) {
    const int64_t ndet = nsa * nsb;
    const int64_t ib = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (ib >= nsb) return;
    for (int64_t ia = blockIdx.y; ia < nsa; ia += gridDim.y) {
        const int64_t det = ia * nsb + ib;
        const double *Crow = C + ia * nsb;
        for (int pp = 0; pp < npair; ++pp) {
            double v = 0.0;
            const int32_t ea = __ldg(pairA + (int64_t)pp * nsa + ia);
            if (ea >= 0) {
                const double c = __ldg(C + (int64_t)(ea >> 1) * nsb + ib);
                v = (ea & 1) ? -c : c;
            }
            const int32_t eb = __ldg(pairB + (int64_t)pp * nsb + ib);
            if (eb >= 0) {
                const double c = __ldg(Crow + (eb >> 1));
                v += (eb & 1) ? -c : c;
            }
            D[(int64_t)pp * ndet + det] = v;
        }
    }
}

__global__ void __launch_bounds__(256) k_scatter_fci_r64(int64_t nsa, int64_t nsb, int npair,
                                                         const int32_t *__restrict__ pairA,
                                                         const int32_t *__restrict__ pairB,
                                                         const double *__restrict__ E,
                                                         const double *__restrict__ C, double e_core,
                                                         double *__restrict__ sigma) {
    const int64_t ndet = nsa * nsb;
    const int64_t ib = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (ib >= nsb) return;
    for (int64_t ia = blockIdx.y; ia < nsa; ia += gridDim.y) {
        const int64_t det = ia * nsb + ib;
        double acc = 0.0;
        for (int pp = 0; pp < npair; ++pp) {
            const double *Ep = E + (int64_t)pp * ndet;
            const int32_t ea = __ldg(pairA + (int64_t)pp * nsa + ia);
            if (ea >= 0) {
                const double e = __ldg(Ep + (int64_t)(ea >> 1) * nsb + ib);
                acc += (ea & 1) ? -e : e;
            }
            const int32_t eb = __ldg(pairB + (int64_t)pp * nsb + ib);
            if (eb >= 0) {
                const double e = __ldg(Ep + ia * nsb + (eb >> 1));
                acc += (eb & 1) ? -e : e;
            }
        }
        sigma[det] = acc + e_core * C[det];
    }
}

// C[M x N] = A[M x K] * B[K x N], all row-major FP64, N large.  64 x 64 tiles,
// 256 threads each owning a 4 x 4 block of outputs; K staged through shared memory in
// chunks of 16.  The FP64 pipe bounds this kernel on GB300.
constexpr int BM = 64, BN = 64, BK = 16;
__global__ void __launch_bounds__(256) k_dgemm(int M, int64_t N, int K, const double *__restrict__ A,
                                               const double *__restrict__ B, int64_t ldb,
                                               double *__restrict__ Cm, int64_t ldc) {
    __shared__ double sA[BK][BM + 1];
    __shared__ double sB[BK][BN];
    const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
    const int m0 = blockIdx.y * BM;
    const int64_t n0 = blockIdx.x * (int64_t)BN;
    double acc[4][4] = {};
    for (int k0 = 0; k0 < K; k0 += BK) {
        for (int i = threadIdx.x; i < BK * BM; i += 256) {
            int kk = i % BK, mm = i / BK;
            int gm = m0 + mm, gk = k0 + kk;
            sA[kk][mm] = (gm < M && gk < K) ? A[(int64_t)gm * K + gk] : 0.0;
        }
        for (int i = threadIdx.x; i < BK * BN; i += 256) {
            int kk = i / BN, nn = i % BN;
            int64_t gn = n0 + nn;
            int gk = k0 + kk;
            sB[kk][nn] = (gn < N && gk < K) ? B[(int64_t)gk * ldb + gn] : 0.0;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < BK; ++kk) {
            double a[4], b[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) a[i] = sA[kk][ty * 4 + i];
#pragma unroll
            for (int j = 0; j < 4; ++j) b[j] = sB[kk][tx + 16 * j];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        int gm = m0 + ty * 4 + i;
        if (gm >= M) continue;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            int64_t gn = n0 + tx + 16 * j;
            if (gn < N) Cm[(int64_t)gm * ldc + gn] = acc[i][j];
        }
    }
}

// H_II = sum_{p in a} h_pp + sum_{p in b} h_pp + 1/2 sum_{p,q in a} (J_pq - K_pq)
//      + 1/2 sum_{p,q in b} (J_pq - K_pq) + sum_{p in a, q in b} J_pq
// (Slater-Condon, the diagonal element).  The first four terms split into a per-string
// energy e(S) = sum_{p in S} h_pp + 1/2 sum_{p,q in S} (J_pq - K_pq), the last is the
// cross term X(a, b) = sum_{p in a} j_b(p) with j_S(p) = sum_{q in S} J_pq; both come from
// a table with one row per string (k_diag_strings), so a determinant costs O(n_el) adds.
// The cross term is taken as 1/2 (sum_{p in a} j_b(p) + sum_{p in b} j_a(p)) and the
// string energies are added as (e(a) + e(b)): H_II is then exactly symmetric under
// exchanging the alpha and beta strings, as the operator is.
__global__ void k_diag_strings(int64_t nsa, int64_t nsb, int n, const uint64_t *__restrict__ sa,
                               const uint64_t *__restrict__ sb, const double *__restrict__ hd,
                               const double *__restrict__ J, const double *__restrict__ K,
                               double *__restrict__ tab) {
    for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < nsa + nsb; s += (int64_t)gridDim.x * blockDim.x) {
        const uint64_t S = s < nsa ? sa[s] : sb[s - nsa];
        double *row = tab + s * (n + 1);
        double e = 0.0;
        for (int p = 0; p < n; ++p) {
            double jp = 0.0;
            for (int q = 0; q < n; ++q)
                if ((S >> q) & 1) jp += J[p * n + q];
            row[1 + p] = jp;
            if (!((S >> p) & 1)) continue;
            e += hd[p];
            for (int q = 0; q < n; ++q)
                if ((S >> q) & 1) e += 0.5 * (J[p * n + q] - K[p * n + q]);
        }
        row[0] = e;
    }
}

__global__ void k_diag_fci(int64_t nsa, int64_t nsb, int n, const uint64_t *__restrict__ sa,
                           const uint64_t *__restrict__ sb, const double *__restrict__ tab, double e_core,
                           double *__restrict__ diag) {
    const int64_t ndet = nsa * nsb;
    for (int64_t det = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; det < ndet;
         det += (int64_t)gridDim.x * blockDim.x) {
        const int64_t ia = det / nsb, ib = det - ia * nsb;
        diag[det] = diag_from_strings(sa[ia], sb[ib], tab + ia * (n + 1), tab + (nsa + ib) * (n + 1), e_core);
    }
}

inline dim3 det_grid(int64_t nsa, int64_t nsb, int threads) {
    unsigned gx = (unsigned)ceil_div(nsb, threads);
    unsigned gy = (unsigned)(nsa < 65535 ? nsa : 65535);
    return dim3(gx, gy);
}

}  // namespace

cudaError_t launch_gather_fci_r64(const fci_context *h, const double *C, double *D, cudaStream_t s) {
    const int threads = 128;
    k_gather_fci_r64<<<det_grid(h->nsa, h->nsb, threads), threads, 0, s>>>(
        h->nsa, h->nsb, h->npair, h->d_pair_a, h->d_pair_b, C, D);
    return cudaGetLastError();
}

cudaError_t launch_scatter_fci_r64(const fci_context *h, const double *E, const double *C,
                                   double *sigma, cudaStream_t s) {
    const int threads = 128;
    k_scatter_fci_r64<<<det_grid(h->nsa, h->nsb, threads), threads, 0, s>>>(
        h->nsa, h->nsb, h->npair, h->d_pair_a, h->d_pair_b, E, C, h->e_core, sigma);
    return cudaGetLastError();
}

cudaError_t launch_dgemm(int M, int64_t N, int K, const double *A, const double *B, int64_t ldb,
                         double *C, int64_t ldc, cudaStream_t s) {
    if (M <= 0 || N <= 0) return cudaSuccess;
    dim3 grid((unsigned)ceil_div(N, BN), (unsigned)ceil_div(M, BM));
    k_dgemm<<<grid, 256, 0, s>>>(M, N, K, A, B, ldb, C, ldc);
    return cudaGetLastError();
}

cudaError_t launch_diag_strings(const fci_context *h, cudaStream_t s) {
    const int64_t ns = h->nsa + h->nsb;
    k_diag_strings<<<(unsigned)std::max<int64_t>(1, std::min<int64_t>(ceil_div(ns, 128), 152 * 8)), 128, 0, s>>>(
        h->nsa, h->nsb, h->n_orb, h->d_str_a, h->d_str_b, h->d_hd, h->d_J, h->d_K, h->d_dstr);
    return cudaGetLastError();
}

cudaError_t launch_diag_fci(const fci_context *h, double *diag, cudaStream_t s) {
    cudaError_t e = launch_diag_strings(h, s);
    if (e != cudaSuccess) return e;
    const int64_t ndet = h->nsa * h->nsb;
    unsigned blocks = (unsigned)std::min<int64_t>(ceil_div(ndet, 256), 152 * 32);
    k_diag_fci<<<blocks, 256, 0, s>>>(h->nsa, h->nsb, h->n_orb, h->d_str_a, h->d_str_b, h->d_dstr, h->e_core, diag);
    return cudaGetLastError();
}
