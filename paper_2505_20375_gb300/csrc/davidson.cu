// Davidson eigensolver on the device (Results: the Ritz residual r = H C - E C is
// preconditioned and appended as the next expansion vector; Eq. sparsePreconditioner).
//
// Every vector operation runs here in FP64 (complex vectors as interleaved pairs):
// subspace projections V^H w, Ritz combinations, the residual, the preconditioner with
// its 1e-12 guard and eps * ||s|| threshold, two rounds of classical Gram-Schmidt and
// the projected eigenproblem (cyclic Jacobi in one thread block; complex Hermitian
// matrices through their real symmetric embedding [[A, -B], [B, A]]).  The host reads
// back a handful of scalars per iteration to decide convergence.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <chrono>
#include <new>
#include <vector>

#include "fci_internal.h"

namespace {

constexpr int RED_BLOCKS = 608;  // 4 x 152 SMs
constexpr int RED_THREADS = 256;
constexpr int KMAX = 32;
constexpr int JAC_THREADS = 256;  // the projected eigensolver's block

struct dav_scalars {      // device-resident scalars, read back each iteration
    double lam;           // lowest Ritz value (sigma carries e_core C, so e_core is included)
    double rnorm2, snorm2, maxdc;
    double ov_re, ov_im;  // <c_prev|c>
    double tnorm2;
    double pad;
};

// partial[b][i] (complex: 2 doubles) = sum over this block's slice of conj(V_i) x, for
// i < k <= KB: KB (a power of two, at least k) sizes the accumulator arrays, so a call
// with few vectors keeps few registers and many warps resident.
template <bool CPLX, int KB>
__global__ void __launch_bounds__(RED_THREADS) k_multidot(const double *__restrict__ V, int64_t ldv, int k,
                                                          const double *__restrict__ x, int64_t n,
                                                          double *__restrict__ partial) {
    __shared__ double red[RED_THREADS / 32][2 * KB];
    double acc_re[KB], acc_im[CPLX ? KB : 1];
#pragma unroll
    for (int i = 0; i < KB; ++i) acc_re[i] = 0.0;
#pragma unroll
    for (int i = 0; i < (CPLX ? KB : 1); ++i) acc_im[i] = 0.0;
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x) {
        if (CPLX) {
            const double xr = x[2 * j], xi = x[2 * j + 1];
#pragma unroll
            for (int i = 0; i < KB; ++i) {
                if (i < k) {
                    const double vr = V[i * 2 * ldv + 2 * j], vi = V[i * 2 * ldv + 2 * j + 1];
                    acc_re[i] = fma(vr, xr, fma(vi, xi, acc_re[i]));
                    acc_im[CPLX ? i : 0] = fma(vr, xi, fma(-vi, xr, acc_im[CPLX ? i : 0]));
                }
            }
        } else {
            const double xr = x[j];
#pragma unroll
            for (int i = 0; i < KB; ++i)
                if (i < k) acc_re[i] = fma(V[i * ldv + j], xr, acc_re[i]);
        }
    }
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int i = 0; i < KB; ++i) {
        if (i >= k) break;
        double a = acc_re[i], b = CPLX ? acc_im[CPLX ? i : 0] : 0.0;
        for (int o = 16; o; o >>= 1) {
            a += __shfl_xor_sync(0xFFFFFFFFu, a, o);
            if (CPLX) b += __shfl_xor_sync(0xFFFFFFFFu, b, o);
        }
        if (lane == 0) { red[wid][2 * i] = a; red[wid][2 * i + 1] = b; }
    }
    __syncthreads();
    if (threadIdx.x < 2 * k) {
        double s = 0.0;
        for (int w = 0; w < RED_THREADS / 32; ++w) s += red[w][threadIdx.x];
        partial[(int64_t)blockIdx.x * 2 * KMAX + threadIdx.x] = s;
    }
}

// Sum over the nb block partials of a reduction in a fixed order (lane l adds blocks l,
// l + 32, ..., then a butterfly over the lanes), so every result is reproducible.
__device__ __forceinline__ double warp_sum_blocks(const double *__restrict__ p, int64_t stride, int nb) {
    const int lane = threadIdx.x & 31;
    double a = 0.0;
    for (int b = lane; b < nb; b += 32) a += p[(int64_t)b * stride];
    for (int o = 16; o; o >>= 1) a += __shfl_xor_sync(0xFFFFFFFFu, a, o);
    return a;
}

// out[i] (complex) = sum_b partial[b][i], one warp per entry.
__global__ void k_reduce_partial(const double *__restrict__ partial, int nb, int k, double *__restrict__ out) {
    for (int i = threadIdx.x >> 5; i < 2 * k; i += blockDim.x >> 5) {
        const double a = warp_sum_blocks(partial + i, 2 * KMAX, nb);
        if ((threadIdx.x & 31) == 0) out[i] = a;
    }
}

// out = sum_i y_i V_i  (+ beta * out when accumulate), y complex as 2 doubles per entry.
template <bool CPLX>
__global__ void k_lincomb(const double *__restrict__ V, int64_t ldv, int k, const double *__restrict__ y,
                          double scale, int64_t n, double *__restrict__ out, int accumulate) {
    __shared__ double sy[2 * KMAX];
    if (threadIdx.x < 2 * k) sy[threadIdx.x] = y[threadIdx.x] * scale;
    __syncthreads();
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x) {
        if (CPLX) {
            double re = accumulate ? out[2 * j] : 0.0, im = accumulate ? out[2 * j + 1] : 0.0;
            for (int i = 0; i < k; ++i) {
                const double vr = V[i * 2 * ldv + 2 * j], vi = V[i * 2 * ldv + 2 * j + 1];
                re = fma(sy[2 * i], vr, fma(-sy[2 * i + 1], vi, re));
                im = fma(sy[2 * i], vi, fma(sy[2 * i + 1], vr, im));
            }
            out[2 * j] = re;
            out[2 * j + 1] = im;
        } else {
            double acc = accumulate ? out[j] : 0.0;
            for (int i = 0; i < k; ++i) acc = fma(sy[2 * i], V[i * ldv + j], acc);
            out[j] = acc;
        }
    }
}

// Phase-align (c, sc) to c_prev by the scalar ph = conj(ov)/|ov|, then
//   r = sc - lam c;  s_i = r_i / (lam - H_ii) if |lam - H_ii| >= 1e-12 else 0;  t = s.
// Partial sums: ||r||^2, ||s||^2; partial max |c - c_prev|.
template <bool CPLX>
__global__ void __launch_bounds__(RED_THREADS) k_residual(double *__restrict__ c, double *__restrict__ sc,
                                                          const double *__restrict__ cprev, int have_prev,
                                                          const double *__restrict__ diag,
                                                          const dav_scalars *__restrict__ sc_in, int64_t n,
                                                          double *__restrict__ t, double *__restrict__ partial) {
    const double lam = sc_in->lam;
    double pr = 1.0, pi = 0.0;
    if (have_prev) {
        const double ore = sc_in->ov_re, oim = sc_in->ov_im, m = sqrt(ore * ore + oim * oim);
        if (m > 0) { pr = ore / m; pi = -oim / m; }
    }
    double r2 = 0.0, s2 = 0.0, mdc = 0.0;
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x) {
        const double den = lam - diag[j];
        const bool ok = fabs(den) >= 1e-12;
        if (CPLX) {
            double cr = c[2 * j], ci = c[2 * j + 1], sr = sc[2 * j], si = sc[2 * j + 1];
            double a = cr * pr - ci * pi, b = cr * pi + ci * pr;
            cr = a; ci = b;
            a = sr * pr - si * pi; b = sr * pi + si * pr;
            sr = a; si = b;
            c[2 * j] = cr; c[2 * j + 1] = ci; sc[2 * j] = sr; sc[2 * j + 1] = si;
            const double rr = sr - lam * cr, ri = si - lam * ci;
            r2 += rr * rr + ri * ri;
            const double tr = ok ? rr / den : 0.0, ti = ok ? ri / den : 0.0;
            s2 += tr * tr + ti * ti;
            t[2 * j] = tr; t[2 * j + 1] = ti;
            if (have_prev) {
                const double dr = cr - cprev[2 * j], di = ci - cprev[2 * j + 1];
                mdc = fmax(mdc, sqrt(dr * dr + di * di));
            }
        } else {
            double cr = c[j] * pr, sr = sc[j] * pr;
            c[j] = cr; sc[j] = sr;
            const double rr = sr - lam * cr;
            r2 += rr * rr;
            const double tr = ok ? rr / den : 0.0;
            s2 += tr * tr;
            t[j] = tr;
            if (have_prev) mdc = fmax(mdc, fabs(cr - cprev[j]));
        }
    }
    __shared__ double red[3][RED_THREADS / 32];
    for (int o = 16; o; o >>= 1) {
        r2 += __shfl_xor_sync(0xFFFFFFFFu, r2, o);
        s2 += __shfl_xor_sync(0xFFFFFFFFu, s2, o);
        mdc = fmax(mdc, __shfl_xor_sync(0xFFFFFFFFu, mdc, o));
    }
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) { red[0][wid] = r2; red[1][wid] = s2; red[2][wid] = mdc; }
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0, b = 0, m = 0;
        for (int w = 0; w < RED_THREADS / 32; ++w) { a += red[0][w]; b += red[1][w]; m = fmax(m, red[2][w]); }
        partial[blockIdx.x * 4 + 0] = a;
        partial[blockIdx.x * 4 + 1] = b;
        partial[blockIdx.x * 4 + 2] = m;
    }
}

__global__ void k_reduce_residual(const double *__restrict__ partial, int nb, dav_scalars *__restrict__ out) {
    const int lane = threadIdx.x & 31;
    double a = 0, b = 0, m = 0;
    for (int i = lane; i < nb; i += 32) { a += partial[i * 4]; b += partial[i * 4 + 1]; m = fmax(m, partial[i * 4 + 2]); }
    for (int o = 16; o; o >>= 1) {
        a += __shfl_xor_sync(0xFFFFFFFFu, a, o);
        b += __shfl_xor_sync(0xFFFFFFFFu, b, o);
        m = fmax(m, __shfl_xor_sync(0xFFFFFFFFu, m, o));
    }
    if (lane == 0) {
        out->rnorm2 = a;
        out->snorm2 = b;
        out->maxdc = m;
    }
}

// Compression-compatible threshold: t_i = 0 where |t_i| < eps ||s||.
template <bool CPLX>
__global__ void k_threshold(double *__restrict__ t, int64_t n, const dav_scalars *__restrict__ s, double eps) {
    const double thr = eps * sqrt(s->snorm2);
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x) {
        if (CPLX) {
            const double a = t[2 * j], b = t[2 * j + 1];
            if (sqrt(a * a + b * b) < thr) { t[2 * j] = 0.0; t[2 * j + 1] = 0.0; }
        } else if (fabs(t[j]) < thr) {
            t[j] = 0.0;
        }
    }
}

// Squared norm partials of x (complex counted as 2n reals).
__global__ void __launch_bounds__(RED_THREADS) k_norm2(const double *__restrict__ x, int64_t nreal,
                                                       double *__restrict__ partial) {
    double a = 0.0;
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < nreal; j += (int64_t)gridDim.x * blockDim.x)
        a = fma(x[j], x[j], a);
    __shared__ double red[RED_THREADS / 32];
    for (int o = 16; o; o >>= 1) a += __shfl_xor_sync(0xFFFFFFFFu, a, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = a;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0;
        for (int w = 0; w < RED_THREADS / 32; ++w) s += red[w];
        partial[blockIdx.x] = s;
    }
}

__global__ void k_reduce_norm(const double *__restrict__ partial, int nb, double *__restrict__ out) {
    const double a = warp_sum_blocks(partial, 1, nb);
    if (threadIdx.x == 0) *out = a;
}

// x *= 1/sqrt(*n2) (or *scale directly when n2 == nullptr)
__global__ void k_scale(double *__restrict__ x, int64_t nreal, const double *__restrict__ n2) {
    const double f = 1.0 / sqrt(*n2);
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < nreal; j += (int64_t)gridDim.x * blockDim.x)
        x[j] *= f;
}

// Negate a complex coefficient vector (k entries).
__global__ void k_negate(double *__restrict__ y, int k) {
    if (threadIdx.x < 2 * k) y[threadIdx.x] = -y[threadIdx.x];
}

// Hsub column/row update: Hsub[i][k] = dots[i] for i <= k, Hsub[k][i] = conj(dots[i]).
__global__ void k_hsub_update(double *__restrict__ Hs, const double *__restrict__ dots, int k) {
    const int i = threadIdx.x;
    if (i > k) return;
    Hs[2 * (i * KMAX + k)] = dots[2 * i];
    Hs[2 * (i * KMAX + k) + 1] = dots[2 * i + 1];
    Hs[2 * (k * KMAX + i)] = dots[2 * i];
    Hs[2 * (k * KMAX + i) + 1] = -dots[2 * i + 1];
    if (i == k) Hs[2 * (k * KMAX + k) + 1] = 0.0;
}

// Lowest eigenpair of the k x k Hermitian Hs (leading dimension KMAX, complex entries)
// by Jacobi on the real symmetric embedding of size m = k (real) or 2k (complex), with the
// rotations of a sweep in round-robin order: each of the M - 1 rounds (M = m rounded up to
// even) pairs every index with one other (index M - 1 with r, and (r + i) with (r - i)
// modulo M - 1), so the M / 2 rotations of a round touch disjoint rows and columns and run
// at once: angles from the current A (the classical formula, tan of the angle the smaller
// root of t^2 + 2 theta t - 1 = 0, theta = (A_qq - A_pp) / (2 A_pq)), then the columns of A
// and Q, then the rows of A.  Sweeps stop once the off-diagonal mass is below 1e-30 of the
// total.  Writes y (complex, k entries) and lam.  One block of JAC_THREADS threads.
// root: 0 = lowest Ritz pair, 1 = second lowest (the real embedding of a complex Hermitian
// matrix has every eigenvalue twice, so there the selected entry is the (2 root)-th).
__global__ void __launch_bounds__(JAC_THREADS) k_jacobi(const double *__restrict__ Hs, int k, int cplx, int root,
                                                        double *__restrict__ y, dav_scalars *__restrict__ out) {
    extern __shared__ double jac_smem[];  // A and Q, each m x (m + 1)
    __shared__ double cs[KMAX][2];
    __shared__ int pr[KMAX][2];
    __shared__ double red[2][JAC_THREADS / 32];
    __shared__ int stop;
    const int m = cplx ? 2 * k : k;
    const int ld = m + 1;
    const int M = m + (m & 1), half = M / 2;
    double *Ab = jac_smem, *Qb = jac_smem + m * ld;
#define A(r, c) Ab[(r) * ld + (c)]
#define Q(r, c) Qb[(r) * ld + (c)]
    const int t = threadIdx.x, nt = blockDim.x;
    for (int i = t; i < m * m; i += nt) {
        const int r = i / m, c = i % m;
        double v;
        if (!cplx) {
            v = Hs[2 * (r * KMAX + c)];
        } else {
            const int rb = r / k, cb = c / k, rr = r % k, cc = c % k;
            const double re = Hs[2 * (rr * KMAX + cc)], im = Hs[2 * (rr * KMAX + cc) + 1];
            v = (rb == cb) ? re : (rb == 1 ? im : -im);
        }
        A(r, c) = v;
        Q(r, c) = (r == c) ? 1.0 : 0.0;
    }
    __syncthreads();
    for (int sweep = 0; sweep < 60 && m > 1; ++sweep) {
        double off = 0.0, tot = 0.0;
        for (int i = t; i < m * m; i += nt) {
            const int r = i / m, c = i % m;
            const double a2 = A(r, c) * A(r, c);
            tot += a2;
            if (r != c) off += a2;
        }
        for (int o = 16; o; o >>= 1) {
            off += __shfl_xor_sync(0xFFFFFFFFu, off, o);
            tot += __shfl_xor_sync(0xFFFFFFFFu, tot, o);
        }
        if ((t & 31) == 0) {
            red[0][t >> 5] = off;
            red[1][t >> 5] = tot;
        }
        __syncthreads();
        if (t == 0) {
            double o = 0.0, a = 0.0;
            for (int w = 0; w < nt / 32; ++w) {
                o += red[0][w];
                a += red[1][w];
            }
            stop = (o <= 1e-30 * a) || o == 0.0;
        }
        __syncthreads();
        if (stop) break;
        for (int r = 0; r < M - 1; ++r) {
            if (t < half) {
                int p, q;
                if (t == 0) {
                    p = M - 1;
                    q = r;
                } else {
                    p = (r + t) % (M - 1);
                    q = (r - t + (M - 1)) % (M - 1);
                }
                double c = 1.0, sn = 0.0;
                if (p < m && q < m) {
                    const double apq = A(p, q);
                    if (fabs(apq) > 1e-300) {
                        const double theta = (A(q, q) - A(p, p)) / (2.0 * apq);
                        const double tt = (theta >= 0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
                        c = 1.0 / sqrt(tt * tt + 1.0);
                        sn = tt * c;
                    }
                }
                pr[t][0] = p;
                pr[t][1] = q;
                cs[t][0] = c;
                cs[t][1] = sn;
            }
            __syncthreads();
            for (int i = t; i < half * m; i += nt) {  // columns p, q of A and Q
                const int j = i / m, row = i % m;
                const double sn = cs[j][1];
                if (sn == 0.0) continue;
                const double c = cs[j][0];
                const int p = pr[j][0], q = pr[j][1];
                const double ap = A(row, p), aq = A(row, q);
                A(row, p) = c * ap - sn * aq;
                A(row, q) = sn * ap + c * aq;
                const double qp = Q(row, p), qq = Q(row, q);
                Q(row, p) = c * qp - sn * qq;
                Q(row, q) = sn * qp + c * qq;
            }
            __syncthreads();
            for (int i = t; i < half * m; i += nt) {  // rows p, q of A
                const int j = i / m, col = i % m;
                const double sn = cs[j][1];
                if (sn == 0.0) continue;
                const double c = cs[j][0];
                const int p = pr[j][0], q = pr[j][1];
                const double ap = A(p, col), aq = A(q, col);
                A(p, col) = c * ap - sn * aq;
                A(q, col) = sn * ap + c * aq;
            }
            __syncthreads();
        }
    }
    if (t == 0) {
        // the (root * (cplx ? 2 : 1))-th smallest diagonal entry (ties: lowest index)
        const int want = root * (cplx ? 2 : 1);
        int best = 0;
        for (int r = 0; r <= want; ++r) {
            best = -1;
            for (int i = 0; i < m; ++i) {
                int rank = 0;  // entries before i in the ascending order
                for (int j = 0; j < m; ++j)
                    if (A(j, j) < A(i, i) || (A(j, j) == A(i, i) && j < i)) ++rank;
                if (rank == r) best = i;
            }
        }
        out->lam = A(best, best);
        double nrm = 0.0;
        for (int i = 0; i < k; ++i) {
            const double re = Q(i, best), im = cplx ? Q(k + i, best) : 0.0;
            y[2 * i] = re;
            y[2 * i + 1] = im;
            nrm += re * re + im * im;
        }
        nrm = 1.0 / sqrt(nrm);
        for (int i = 0; i < 2 * k; ++i) y[i] *= nrm;
    }
}
#undef A
#undef Q

// argmin of diag (lowest index on ties) -> unit vector
// Index of the smallest diagonal element (the lowest index among equal ones), in two
// passes: per block (value, index) into part, then one block over the nb block results.
__device__ __forceinline__ void argmin_merge(double &v, int64_t &i, double v2, int64_t i2) {
    if (v2 < v || (v2 == v && i2 < i)) { v = v2; i = i2; }
}
__device__ void argmin_block(double v, int64_t idx, double *bv, int64_t *bi) {
    for (int o = 16; o; o >>= 1)
        argmin_merge(v, idx, __shfl_xor_sync(0xFFFFFFFFu, v, o), __shfl_xor_sync(0xFFFFFFFFu, idx, o));
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) { bv[wid] = v; bi[wid] = idx; }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < (int)(blockDim.x >> 5); ++w) argmin_merge(v, idx, bv[w], bi[w]);
        bv[0] = v;
        bi[0] = idx;
    }
}
__global__ void __launch_bounds__(256) k_argmin_part(const double *__restrict__ d, int64_t n, double *__restrict__ part) {
    __shared__ double bv[8];
    __shared__ int64_t bi[8];
    double v = INFINITY;
    int64_t idx = INT64_MAX;
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x)
        if (d[j] < v) { v = d[j]; idx = j; }
    argmin_block(v, idx, bv, bi);
    if (threadIdx.x == 0) {
        part[2 * blockIdx.x] = bv[0];
        part[2 * blockIdx.x + 1] = __longlong_as_double((long long)bi[0]);
    }
}
__global__ void __launch_bounds__(256) k_argmin_final(const double *__restrict__ part, int nb, int64_t *__restrict__ out) {
    __shared__ double bv[8];
    __shared__ int64_t bi[8];
    double v = INFINITY;
    int64_t idx = INT64_MAX;
    for (int b = threadIdx.x; b < nb; b += blockDim.x)
        argmin_merge(v, idx, part[2 * b], (int64_t)__double_as_longlong(part[2 * b + 1]));
    argmin_block(v, idx, bv, bi);
    if (threadIdx.x == 0) *out = bi[0] == INT64_MAX ? 0 : bi[0];
}

// splitmix64 (Steele, Lea and Flood 2014, "Fast splittable pseudorandom number
// generators"): the published finaliser of a 64-bit counter.
__device__ __forceinline__ uint64_t splitmix64(uint64_t x) {
    uint64_t z = x + 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// Start vector: the unit vector at idx plus, if mix > 0, mix times a pseudo-random vector
// of norm about one (entries uniform in [-1, 1) from splitmix64 of the index, scaled by
// sqrt(3 / nreal)).  The admixture gives the start a component in every symmetry sector
// (a closed-shell unit vector alone is symmetric under alpha <-> beta exchange, and the
// iteration would stay in that sector).
__global__ void k_set_start(double *__restrict__ x, int64_t nreal, int cplx, const int64_t *__restrict__ idx,
                            double mix) {
    const int64_t at = (cplx ? 2 : 1) * (*idx);
    const double scale = mix * sqrt(3.0 / (double)nreal);
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < nreal; j += (int64_t)gridDim.x * blockDim.x) {
        double v = (j == at) ? 1.0 : 0.0;
        if (mix > 0.0) v += scale * (2.0 * (double)(splitmix64((uint64_t)j) >> 11) * 0x1.0p-53 - 1.0);
        x[j] = v;
    }
}

inline size_t al(size_t b) { return (b + 255) & ~(size_t)255; }

}  // namespace

// Davidson as a state machine: run_until_sigma() advances the iteration until the next
// sigma product is needed (it then exposes x and y = H x to the caller) or until the
// solve ends.  davidson_solve drives it with the library's own sigma; the step-wise C ABI
// (davidson_begin/advance/finish) lets a scheduler compute the sigma products of many
// solves together.
struct fci_davidson_state {
    enum { REQ_NONE = 0, REQ_INIT, REQ_SWITCH, REQ_APPEND };
    fci_context *h = nullptr;
    fci_davidson_opts o{};
    cudaStream_t s = nullptr;
    int64_t n = 0, nreal = 0, ldv = 0;
    bool cplx = false;
    size_t esz = 8, vec = 0;
    int ms = 0;
    double *V = nullptr, *S = nullptr, *c = nullptr, *sc = nullptr, *cp = nullptr, *scp = nullptr, *t = nullptr,
           *diag = nullptr;
    void *sig_ws = nullptr;
    size_t sig_bytes = 0;
    double *partial = nullptr, *Hs = nullptr, *dots = nullptr, *y = nullptr, *nrm = nullptr;
    dav_scalars *scal = nullptr;
    int64_t *argmin = nullptr;
    unsigned vb = 1;
    // iteration state
    int k = 0, it = 0, it_rec = 0, phase1_iters = 0, n_sigma = 0;
    int prec = FCI_PREC_FP64, slices = 0;
    bool final_phase = true, have_prev = false, converged = false, done = false;
    double E_prev = 0.0, lam_pending = 0.0;
    int request = REQ_NONE;
    double *req_x = nullptr, *req_y = nullptr;
    double *stage_x = nullptr, *stage_y = nullptr, *real_y = nullptr;  // staged sigma requests
    // gap bound (Results, Eq. gammaLowerBound): after convergence, the second Ritz pair
    bool gap_phase = false;
    int gap_iters = 0;
    double E1 = NAN, r1n = NAN, r0n = NAN, gap_lower = NAN, err_bound = NAN;
    std::chrono::steady_clock::time_point t_iter;
    std::vector<fci_davidson_iter> log;
    int status = FCI_OK;

    double *Vk(int i) { return (double *)((char *)V + (size_t)i * vec); }
    double *Sk(int i) { return (double *)((char *)S + (size_t)i * vec); }

    // vectors i0 .. i0 + kk - 1 of Vb into entries i0 .. of each block's partial row
    template <int KB>
    void multidot_kb(const double *Vb, int i0, int kk, const double *x) {
        const double *v0 = Vb + (size_t)i0 * (cplx ? 2 : 1) * ldv;
        if (cplx) k_multidot<true, KB><<<vb, RED_THREADS, 0, s>>>(v0, ldv, kk, x, n, partial + 2 * i0);
        else k_multidot<false, KB><<<vb, RED_THREADS, 0, s>>>(v0, ldv, kk, x, n, partial + 2 * i0);
    }
    // <V_i|x> for i < kk: up to 16 vectors per pass (more would cost occupancy)
    cudaError_t multidot(const double *Vb, int kk, const double *x, double *out) {
        if (kk <= 1) multidot_kb<1>(Vb, 0, kk, x);
        else if (kk <= 4) multidot_kb<4>(Vb, 0, kk, x);
        else if (kk <= 8) multidot_kb<8>(Vb, 0, kk, x);
        else if (kk <= 16) multidot_kb<16>(Vb, 0, kk, x);
        else {
            multidot_kb<16>(Vb, 0, 16, x);
            multidot_kb<16>(Vb, 16, kk - 16, x);
        }
        k_reduce_partial<<<1, 256, 0, s>>>(partial, vb, kk, out);
        return cudaGetLastError();
    }
    cudaError_t lincomb(const double *Vb, int kk, const double *yy, double scale, double *out, int acc) {
        if (cplx) k_lincomb<true><<<vb, RED_THREADS, 0, s>>>(Vb, ldv, kk, yy, scale, n, out, acc);
        else k_lincomb<false><<<vb, RED_THREADS, 0, s>>>(Vb, ldv, kk, yy, scale, n, out, acc);
        return cudaGetLastError();
    }
    cudaError_t normalize(double *x, double *n2out) {
        k_norm2<<<vb, RED_THREADS, 0, s>>>(x, nreal, partial);
        k_reduce_norm<<<1, 32, 0, s>>>(partial, vb, n2out);
        k_scale<<<vb, RED_THREADS, 0, s>>>(x, nreal, n2out);
        return cudaGetLastError();
    }
    // New subspace column kk: Hs[:, kk] = V^H S_kk.
    int add_column(int kk) {
        FCI_CUDA(h, multidot(V, kk + 1, Sk(kk), dots));
        k_hsub_update<<<1, 64, 0, s>>>(Hs, dots, kk);
        FCI_CUDA(h, cudaGetLastError());
        return FCI_OK;
    }
    int ask(int kind, double *x, double *yv) {
        request = kind;
        req_x = x;
        req_y = yv;
        ++n_sigma;
        if (o.staged_sigma) {  // the caller always sees the same two vectors
            FCI_CUDA(h, cudaMemcpyAsync(stage_x, x, (size_t)n * esz, cudaMemcpyDeviceToDevice, s));
            req_x = stage_x;
            req_y = stage_y;
            real_y = yv;
        }
        return FCI_OK;
    }

    int init(fci_context *hh, const fci_davidson_opts *oo, const void *guess, void *ws, cudaStream_t st) {
        h = hh;
        o = *oo;
        s = st;
        n = h->das_active ? h->das.n_det : h->ndet;
        cplx = h->dtype == FCI_C128;
        esz = cplx ? 16 : 8;
        nreal = cplx ? 2 * n : n;
        vec = al((size_t)n * esz);
        ms = o.max_subspace;
        char *p = (char *)ws;
        V = (double *)p; p += ms * vec;
        S = (double *)p; p += ms * vec;
        c = (double *)p; p += vec;
        sc = (double *)p; p += vec;
        cp = (double *)p; p += vec;
        scp = (double *)p; p += vec;
        t = (double *)p; p += vec;
        diag = (double *)p; p += al((size_t)n * 8);
        if (o.staged_sigma) {
            stage_x = (double *)p; p += vec;
            stage_y = (double *)p; p += vec;
        }
        sig_ws = p;
        size_t sig = sigma_ws_bytes(h, o.precision, o.n_slices);
        if (o.precision != FCI_PREC_FP64) sig = std::max(sig, sigma_ws_bytes(h, o.final_precision, o.final_slices));
        sig_bytes = al(sig);
        ldv = (int64_t)(vec / esz);
        double *small = h->d_small;
        partial = small;                           // RED_BLOCKS * 2 * KMAX
        Hs = partial + RED_BLOCKS * 2 * KMAX;      // 2 * KMAX * KMAX
        dots = Hs + 2 * KMAX * KMAX;               // 2 * KMAX
        y = dots + 2 * KMAX;                       // 2 * KMAX
        nrm = y + 2 * KMAX;                        // 4
        scal = (dav_scalars *)(nrm + 4);
        argmin = (int64_t *)(scal + 1);
        vb = (unsigned)std::min<int64_t>(RED_BLOCKS, std::max<int64_t>(1, ceil_div(n, RED_THREADS)));
        prec = o.precision;
        slices = o.n_slices;
        if (o.eps < 0.0) o.eps = 10.0 / sqrt((double)n);  // the paper's eps <~ 10 / sqrt(N_dets) rule
        final_phase = o.precision == FCI_PREC_FP64 || (o.precision == o.final_precision && o.n_slices == o.final_slices);
        FCI_CUDA(h, cudaFuncSetAttribute(k_jacobi, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         2 * (2 * KMAX) * (2 * KMAX + 1) * (int)sizeof(double)));
        if (h->das_active) FCI_CUDA(h, launch_diag_das(h, diag, s));
        else if (h->mode == FCI_MODE_SPINOR) FCI_CUDA(h, launch_diag_spinor(h, diag, s));
        else FCI_CUDA(h, launch_diag_fci(h, diag, s));
        if (guess) {
            FCI_CUDA(h, cudaMemcpyAsync(Vk(0), guess, (size_t)n * esz, cudaMemcpyDeviceToDevice, s));
        } else {
            k_argmin_part<<<vb, 256, 0, s>>>(diag, n, partial);
            k_argmin_final<<<1, 256, 0, s>>>(partial, (int)vb, argmin);
            k_set_start<<<vb, RED_THREADS, 0, s>>>(Vk(0), nreal, cplx, argmin, o.start_mix);
        }
        FCI_CUDA(h, normalize(Vk(0), nrm));
        return ask(REQ_INIT, Vk(0), Sk(0));
    }

    // The caller has written y = H x for the pending request.
    int consume_sigma() {
        int rc;
        if (o.staged_sigma && request != REQ_NONE)
            FCI_CUDA(h, cudaMemcpyAsync(real_y, stage_y, (size_t)n * esz, cudaMemcpyDeviceToDevice, s));
        switch (request) {
            case REQ_INIT:
                FCI_CUDA(h, cudaMemsetAsync(Hs, 0, 2 * KMAX * KMAX * 8, s));
                if ((rc = add_column(0))) return rc;
                k = 1;
                break;
            case REQ_SWITCH:
                FCI_CUDA(h, cudaMemsetAsync(Hs, 0, 2 * KMAX * KMAX * 8, s));
                if ((rc = add_column(0))) return rc;
                k = 1;
                FCI_CUDA(h, cudaMemcpyAsync(cp, c, (size_t)n * esz, cudaMemcpyDeviceToDevice, s));
                have_prev = true;
                E_prev = lam_pending;
                break;
            case REQ_APPEND:
                if ((rc = add_column(k))) return rc;
                ++k;
                break;
            default:
                return fci_fail(h, FCI_ERR_STATE, "no sigma product was requested");
        }
        request = REQ_NONE;
        return FCI_OK;
    }

    // Advance until the next sigma request (returns FCI_OK with request != REQ_NONE) or
    // until the solve ends (done = true).
    int run_until_sigma() {
        int rc;
        dav_scalars hs{};
        while (!done) {
            if (!gap_phase && it >= o.max_iter) {
                done = true;
                break;
            }
            if (!gap_phase) ++it;  // second-root passes have their own limit (max_iter of them)
            t_iter = std::chrono::steady_clock::now();
            {
                const int m = cplx ? 2 * k : k;
                k_jacobi<<<1, JAC_THREADS, 2 * m * (m + 1) * sizeof(double), s>>>(Hs, k, cplx ? 1 : 0, gap_phase ? 1 : 0, y,
                                                                          scal);
            }
            FCI_CUDA(h, lincomb(V, k, y, 1.0, c, 0));
            FCI_CUDA(h, lincomb(S, k, y, 1.0, sc, 0));
            if (have_prev) {
                FCI_CUDA(h, multidot(cp, 1, c, dots));  // <c_prev|c>
                FCI_CUDA(h, cudaMemcpyAsync(&scal->ov_re, dots, 16, cudaMemcpyDeviceToDevice, s));
            }
            if (cplx) k_residual<true><<<vb, RED_THREADS, 0, s>>>(c, sc, cp, have_prev, diag, scal, n, t, partial);
            else k_residual<false><<<vb, RED_THREADS, 0, s>>>(c, sc, cp, have_prev, diag, scal, n, t, partial);
            k_reduce_residual<<<1, 32, 0, s>>>(partial, vb, scal);
            FCI_CUDA(h, cudaGetLastError());
            FCI_CUDA(h, cudaMemcpyAsync(&hs, scal, sizeof hs, cudaMemcpyDeviceToHost, s));
            FCI_CUDA(h, cudaStreamSynchronize(s));
            const double lam = hs.lam, rn = sqrt(hs.rnorm2);
            const double dE = it > 1 ? lam - E_prev : 0.0;
            const auto t1 = std::chrono::steady_clock::now();
            fci_davidson_iter r;
            r.iteration = it;
            r.precision = prec;
            r.energy = lam;  // sigma carries e_core C
            r.delta_energy = dE;
            r.max_delta_c = have_prev ? hs.maxdc : 0.0;
            r.residual_norm = rn;
            r.seconds = std::chrono::duration<double>(t1 - t_iter).count();
            if (!gap_phase) log.push_back(r);
            if (!isfinite(lam) || !isfinite(rn)) return fci_fail(h, FCI_ERR_CUDA, "Davidson produced a non-finite value");
            if (!final_phase) {
                ++phase1_iters;
                if (rn <= o.switch_residual || phase1_iters >= o.max_iter / 2) {
                    // Residual correction: restart from the Ritz vector with the final precision.
                    final_phase = true;
                    prec = o.final_precision;
                    slices = o.final_slices;
                    FCI_CUDA(h, cudaMemcpyAsync(Vk(0), c, (size_t)n * esz, cudaMemcpyDeviceToDevice, s));
                    FCI_CUDA(h, normalize(Vk(0), nrm));
                    lam_pending = lam;
                    return ask(REQ_SWITCH, Vk(0), Sk(0));
                }
            } else if (gap_phase) {
                ++gap_iters;
                E1 = lam;
                r1n = rn;
                if (rn <= std::max(o.tol_residual, 0.25 * (lam - E_prev)) || gap_iters >= o.max_iter ||
                    (k >= ms && ms < 3)) {
                    if ((rc = finish_gap())) return rc;
                    done = true;
                    break;
                }
            } else if (rn <= o.tol_residual && it > 1 && fabs(dE) <= o.tol_energy) {
                converged = true;
                E_prev = lam;
                if (o.gap_bound && k >= 2) {
                    // keep the subspace and steer it to the second Ritz pair (root 0 stays in it)
                    gap_phase = true;
                    have_prev = false;
                    r0n = rn;
                    continue;  // the next pass re-diagonalises for root 1
                }
                done = true;
                break;
            }
            if (o.eps > 0.0) {
                if (cplx) k_threshold<true><<<vb, RED_THREADS, 0, s>>>(t, n, scal, o.eps);
                else k_threshold<false><<<vb, RED_THREADS, 0, s>>>(t, n, scal, o.eps);
            }
            if (k >= ms && !gap_phase) {
                // collapse to the current and previous Ritz vectors (sigma by linearity)
                // V_0 = c / ||c||, S_0 = sc / ||c||
                FCI_CUDA(h, cudaMemcpyAsync(Vk(0), c, (size_t)n * esz, cudaMemcpyDeviceToDevice, s));
                FCI_CUDA(h, cudaMemcpyAsync(Sk(0), sc, (size_t)n * esz, cudaMemcpyDeviceToDevice, s));
                k_norm2<<<vb, RED_THREADS, 0, s>>>(Vk(0), nreal, partial);
                k_reduce_norm<<<1, 32, 0, s>>>(partial, vb, nrm);
                k_scale<<<vb, RED_THREADS, 0, s>>>(Vk(0), nreal, nrm);
                k_scale<<<vb, RED_THREADS, 0, s>>>(Sk(0), nreal, nrm);
                int knew = 1;
                if (have_prev && ms > 2) {
                    // p = c_prev - <c|c_prev> c, S_p = sc_prev - <c|c_prev> sc, both / ||p||.
                    // Two Gram-Schmidt passes: c and c_prev are nearly parallel near
                    // convergence, and one pass leaves an orthogonality error of eps / ||p||
                    // that compounds over successive collapses.
                    FCI_CUDA(h, cudaMemcpyAsync(Vk(1), cp, (size_t)n * esz, cudaMemcpyDeviceToDevice, s));
                    FCI_CUDA(h, cudaMemcpyAsync(Sk(1), scp, (size_t)n * esz, cudaMemcpyDeviceToDevice, s));
                    for (int pass = 0; pass < 2; ++pass) {
                        FCI_CUDA(h, multidot(Vk(0), 1, Vk(1), dots));
                        k_negate<<<1, 64, 0, s>>>(dots, 1);
                        FCI_CUDA(h, lincomb(Vk(0), 1, dots, 1.0, Vk(1), 1));
                        FCI_CUDA(h, lincomb(Sk(0), 1, dots, 1.0, Sk(1), 1));
                    }
                    k_norm2<<<vb, RED_THREADS, 0, s>>>(Vk(1), nreal, partial);
                    k_reduce_norm<<<1, 32, 0, s>>>(partial, vb, nrm);
                    double pn2 = 0.0;
                    FCI_CUDA(h, cudaMemcpyAsync(&pn2, nrm, 8, cudaMemcpyDeviceToHost, s));
                    FCI_CUDA(h, cudaStreamSynchronize(s));
                    if (sqrt(pn2) > 1e-10) {
                        k_scale<<<vb, RED_THREADS, 0, s>>>(Vk(1), nreal, nrm);
                        k_scale<<<vb, RED_THREADS, 0, s>>>(Sk(1), nreal, nrm);
                        knew = 2;
                    }
                }
                FCI_CUDA(h, cudaMemsetAsync(Hs, 0, 2 * KMAX * KMAX * 8, s));
                for (int jj = 0; jj < knew; ++jj)
                    if ((rc = add_column(jj))) return rc;
                k = knew;
            }
            if (k >= ms && gap_phase) {
                // collapse to the ground-state Ritz vector (it must stay in the subspace for
                // the final E_0) and the current second Ritz vector orthogonalised against it;
                // c_prev / sc_prev are free in this phase and hold the ground state meanwhile
                {
                    const int m = cplx ? 2 * k : k;
                    k_jacobi<<<1, JAC_THREADS, 2 * m * (m + 1) * sizeof(double), s>>>(Hs, k, cplx ? 1 : 0, 0, y, scal);
                }
                FCI_CUDA(h, lincomb(V, k, y, 1.0, cp, 0));
                FCI_CUDA(h, lincomb(S, k, y, 1.0, scp, 0));
                FCI_CUDA(h, cudaMemcpyAsync(Vk(0), cp, (size_t)n * esz, cudaMemcpyDeviceToDevice, s));
                FCI_CUDA(h, cudaMemcpyAsync(Sk(0), scp, (size_t)n * esz, cudaMemcpyDeviceToDevice, s));
                k_norm2<<<vb, RED_THREADS, 0, s>>>(Vk(0), nreal, partial);
                k_reduce_norm<<<1, 32, 0, s>>>(partial, vb, nrm);
                k_scale<<<vb, RED_THREADS, 0, s>>>(Vk(0), nreal, nrm);
                k_scale<<<vb, RED_THREADS, 0, s>>>(Sk(0), nreal, nrm);
                FCI_CUDA(h, cudaMemcpyAsync(Vk(1), c, (size_t)n * esz, cudaMemcpyDeviceToDevice, s));
                FCI_CUDA(h, cudaMemcpyAsync(Sk(1), sc, (size_t)n * esz, cudaMemcpyDeviceToDevice, s));
                for (int pass = 0; pass < 2; ++pass) {
                    FCI_CUDA(h, multidot(Vk(0), 1, Vk(1), dots));
                    k_negate<<<1, 64, 0, s>>>(dots, 1);
                    FCI_CUDA(h, lincomb(Vk(0), 1, dots, 1.0, Vk(1), 1));
                    FCI_CUDA(h, lincomb(Sk(0), 1, dots, 1.0, Sk(1), 1));
                }
                k_norm2<<<vb, RED_THREADS, 0, s>>>(Vk(1), nreal, partial);
                k_reduce_norm<<<1, 32, 0, s>>>(partial, vb, nrm);
                k_scale<<<vb, RED_THREADS, 0, s>>>(Vk(1), nreal, nrm);
                k_scale<<<vb, RED_THREADS, 0, s>>>(Sk(1), nreal, nrm);
                FCI_CUDA(h, cudaGetLastError());
                FCI_CUDA(h, cudaMemsetAsync(Hs, 0, 2 * KMAX * KMAX * 8, s));
                for (int jj = 0; jj < 2; ++jj)
                    if ((rc = add_column(jj))) return rc;
                k = 2;
            }
            // two rounds of classical Gram-Schmidt against V[0..k)
            for (int round = 0; round < 2; ++round) {
                FCI_CUDA(h, multidot(V, k, t, dots));
                k_negate<<<1, 64, 0, s>>>(dots, k);
                FCI_CUDA(h, lincomb(V, k, dots, 1.0, t, 1));
            }
            k_norm2<<<vb, RED_THREADS, 0, s>>>(t, nreal, partial);
            k_reduce_norm<<<1, 32, 0, s>>>(partial, vb, nrm);
            double tn2 = 0.0;
            FCI_CUDA(h, cudaMemcpyAsync(&tn2, nrm, 8, cudaMemcpyDeviceToHost, s));
            if (!gap_phase) {
                FCI_CUDA(h, cudaMemcpyAsync(cp, c, (size_t)n * esz, cudaMemcpyDeviceToDevice, s));
                FCI_CUDA(h, cudaMemcpyAsync(scp, sc, (size_t)n * esz, cudaMemcpyDeviceToDevice, s));
            }
            FCI_CUDA(h, cudaStreamSynchronize(s));
            if (!gap_phase) {
                have_prev = true;
                E_prev = lam;
            }
            if (!(sqrt(tn2) >= 1e-10)) {  // new direction linearly dependent on the subspace
                if (gap_phase && (rc = finish_gap())) return rc;
                done = true;
                break;
            }
            k_scale<<<vb, RED_THREADS, 0, s>>>(t, nreal, nrm);
            FCI_CUDA(h, cudaMemcpyAsync(Vk(k), t, (size_t)n * esz, cudaMemcpyDeviceToDevice, s));
            return ask(REQ_APPEND, Vk(k), Sk(k));
        }
        return FCI_OK;
    }

    // Root 0 on the final subspace (its Ritz vector goes back to c), then the gap bound:
    // gamma_0^- = (E_1 - ||r_1||) - E_0 and |dE| <= ||r_0||^2 / gamma_0^- (gap theorem).
    int finish_gap() {
        dav_scalars hs{};
        const int m = cplx ? 2 * k : k;
        k_jacobi<<<1, JAC_THREADS, 2 * m * (m + 1) * sizeof(double), s>>>(Hs, k, cplx ? 1 : 0, 0, y, scal);
        FCI_CUDA(h, lincomb(V, k, y, 1.0, c, 0));
        FCI_CUDA(h, lincomb(S, k, y, 1.0, sc, 0));
        if (cplx) k_residual<true><<<vb, RED_THREADS, 0, s>>>(c, sc, cp, false, diag, scal, n, t, partial);
        else k_residual<false><<<vb, RED_THREADS, 0, s>>>(c, sc, cp, false, diag, scal, n, t, partial);
        k_reduce_residual<<<1, 32, 0, s>>>(partial, vb, scal);
        FCI_CUDA(h, cudaGetLastError());
        FCI_CUDA(h, cudaMemcpyAsync(&hs, scal, sizeof hs, cudaMemcpyDeviceToHost, s));
        FCI_CUDA(h, cudaStreamSynchronize(s));
        E_prev = hs.lam;
        r0n = sqrt(hs.rnorm2);
        gap_lower = (E1 - r1n) - E_prev;
        err_bound = gap_lower > 0.0 ? r0n * r0n / gap_lower : INFINITY;
        return FCI_OK;
    }

    int finish(void *C_out, double *energy, fci_davidson_log *lg) {
        if (C_out) FCI_CUDA(h, cudaMemcpyAsync(C_out, c, (size_t)n * esz, cudaMemcpyDeviceToDevice, s));
        FCI_CUDA(h, cudaStreamSynchronize(s));
        if (energy) *energy = E_prev;
        if (lg) {
            const int m = std::min<int>((int)log.size(), lg->capacity);
            if (lg->iters)
                for (int i = 0; i < m; ++i) lg->iters[i] = log[i];
            lg->n_iter = lg->iters ? m : 0;
            lg->converged = converged ? 1 : 0;
            lg->n_sigma = n_sigma;
            lg->e1 = E1;
            lg->r1_norm = r1n;
            lg->r0_norm = r0n;
            lg->gap_lower = gap_lower;
            lg->error_bound = err_bound;
            lg->gap_iterations = gap_iters;
        }
        if (!converged)
            return fci_fail(h, FCI_ERR_NOT_CONVERGED, "Davidson did not converge in %d iterations", o.max_iter);
        return FCI_OK;
    }
};

size_t davidson_ws_bytes(const fci_context *h, const fci_davidson_opts *o) {
    const int64_t n = h->das_active ? h->das.n_det : h->ndet;
    const size_t esz = h->dtype == FCI_C128 ? 16 : 8;
    const size_t vec = al((size_t)n * esz);
    size_t sig = sigma_ws_bytes(h, o->precision, o->n_slices);
    if (o->precision != FCI_PREC_FP64) sig = std::max(sig, sigma_ws_bytes(h, o->final_precision, o->final_slices));
    return 2 * (size_t)o->max_subspace * vec + (o->staged_sigma ? 7 : 5) * vec + al((size_t)n * 8) + al(sig);
}

int davidson_run(fci_context *h, const fci_davidson_opts *o, double *C_io, double *energy, fci_davidson_log *log,
                 void *ws, size_t ws_bytes, cudaStream_t s) {
    (void)ws_bytes;
    fci_davidson_state st;
    int rc = st.init(h, o, o->use_guess ? C_io : nullptr, ws, s);
    while (!rc) {
        rc = sigma_dispatch(h, st.req_x, st.req_y, st.prec, st.slices, st.sig_ws, st.sig_bytes, s);
        if (rc) break;
        if ((rc = st.consume_sigma())) break;
        if ((rc = st.run_until_sigma())) break;
        if (st.done) break;
    }
    if (rc) return rc;
    return st.finish(C_io, energy, log);
}

// ------------------------------------------------------------------ step-wise ABI

int davidson_state_begin(fci_context *h, const fci_davidson_opts *o, const void *guess, void *ws, cudaStream_t s,
                         fci_davidson_state **out) {
    fci_davidson_state *st = new (std::nothrow) fci_davidson_state();
    if (!st) return fci_fail(h, FCI_ERR_OOM, "host allocation failed");
    int rc = st->init(h, o, guess, ws, s);
    if (rc) {
        delete st;
        return rc;
    }
    *out = st;
    return FCI_OK;
}

int davidson_state_advance(fci_davidson_state *st, int *done) {
    int rc = st->consume_sigma();
    if (!rc) rc = st->run_until_sigma();
    *done = st->done ? 1 : 0;
    return rc;
}

void davidson_state_request(const fci_davidson_state *st, const void **x, void **y, int *prec, int *slices,
                            void **sig_ws, size_t *sig_bytes) {
    if (x) *x = st->req_x;
    if (y) *y = st->req_y;
    if (prec) *prec = st->prec;
    if (slices) *slices = st->slices;
    if (sig_ws) *sig_ws = st->sig_ws;
    if (sig_bytes) *sig_bytes = st->sig_bytes;
}

int davidson_state_finish(fci_davidson_state *st, void *C_out, double *energy, fci_davidson_log *log) {
    const int rc = st->finish(C_out, energy, log);
    delete st;
    return rc;
}

fci_context *davidson_state_handle(const fci_davidson_state *st) { return st->h; }
