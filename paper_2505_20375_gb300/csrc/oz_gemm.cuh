// Split-precision GEMM on the tcgen05 tensor cores with both operands streamed by
// cp.async.bulk from tile-ready digit images in HBM (shared by the complex spinor path
// and the two-pass alpha/beta path).
//
//   A image (G): tiles [M-tile][K-chunk][plane i < s][128 rows x 8 KCC K], f16 digits
//   B image (D): tiles [N-tile][K-chunk][plane j < s][ 64 rows x 8 KCC K], f16 digits
// each plane in canonical K-major core matrices (core (row / 8, k / 8) at
// ((row / 8) * KCC + k / 8) * 128 bytes, 8 rows x 16 bytes); KCC = 4 (32 K per chunk) or
// 2 (16 K).  With one M-tile the A image may instead stay resident in shared memory
// (loaded once per CTA), so that only the B tiles stream.  The top s digit levels
// L = i + j >= s - 1 are summed exactly in FP32 TMEM accumulators (the caller guarantees
// every level sum is an integer below 2^24); the epilogue combines them in int64 with
// base 2^W (W = 7 or 8 bit digits), rounding away the levels below
// L0 = max(s - 1, 2s - 2 - floor(38 / W)), and stores
//   E_int[N-tile][M_pad][64]   (row m of tile nt, determinant nt * 64 + c at column c).
#pragma once

#include <stdint.h>

#include "fci_internal.h"

constexpr int OZG_M = 128;                     // rows of A per tile
constexpr int OZG_N = 64;                      // determinants per tile
constexpr int OZG_KC = 32;                     // K per pipeline stage (KCC = 4)
constexpr int OZG_A_PLANE = OZG_M * OZG_KC * 2;  // 8 KB (KCC = 4)
constexpr int OZG_B_PLANE = OZG_N * OZG_KC * 2;  // 4 KB (KCC = 4)
constexpr int OZG_MAXS = 8;

struct oz_gemm_args {
    int n_mt, n_kc, M_pad, M_real;  // M_real: rows of the operator (rows past it are not stored)
    int64_t n_nt;
    const void *Gimg, *Dimg;
    int64_t *E;
    int *status;
};

__host__ __device__ constexpr int oz_gemm_L0(int s, int w) {
    return (s - 1 > 2 * s - 2 - 38 / w) ? s - 1 : 2 * s - 2 - 38 / w;
}

// Pipeline stages that fit for s slices, kcc cores per chunk, and (resa_kc > 0) a resident
// A image of resa_kc chunks (0: does not fit).
int oz_gemm_ring(int s, int kcc, int resa_kc);
// Launch over every (N-tile, M-tile) unit; w = digit bits.  Built forms: (w 7, kcc 4),
// (w 8, kcc 4), (w 8, kcc 2, resident A, one M-tile).
int oz_gemm_launch(fci_context *h, int s, int w, int kcc, bool resa, const oz_gemm_args &a, cudaStream_t st);
