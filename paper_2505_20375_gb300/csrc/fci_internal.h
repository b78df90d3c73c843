// Internal declarations of libfci (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/fci.h"

#define FCI_MAXORB 64
#define FCI_BINOM_LD 65  // binomial table row stride: binom[p * 65 + j] = C(p, j)

// Packed single-replacement entry (uint64):
//   bits  0-31 target string index, 32-39 a (created), 40-47 b (annihilated),
//   bit   48 sign (1 = negative), bits 49-63 pair index (packed n(n+1)/2 index for real
//   spin-free orbitals, a*n+b for spinors).
__host__ __device__ inline uint64_t rep_pack(uint32_t t, int a, int b, int neg, int pair) {
    return (uint64_t)t | ((uint64_t)(a & 0xFF) << 32) | ((uint64_t)(b & 0xFF) << 40) |
           ((uint64_t)(neg & 1) << 48) | ((uint64_t)(pair & 0x7FFF) << 49);
}
__host__ __device__ inline uint32_t rep_target(uint64_t e) { return (uint32_t)e; }
__host__ __device__ inline int rep_a(uint64_t e) { return (int)((e >> 32) & 0xFF); }
__host__ __device__ inline int rep_b(uint64_t e) { return (int)((e >> 40) & 0xFF); }
__host__ __device__ inline int rep_neg(uint64_t e) { return (int)((e >> 48) & 1); }

#ifdef __CUDACC__
// Diagonal element of the determinant of strings A (alpha) and B (beta) from their rows
// ta, tb of the per-string table (d_dstr: row[0] the string's own energy, row[1 + p] =
// sum_{q in string} J_pq): e_core + (e(A) + e(B)) + 1/2 (sum_{p in A} j_B(p) + sum_{p in B}
// j_A(p)), symmetric under exchanging A and B bit for bit.
__device__ __forceinline__ double diag_from_strings(uint64_t A, uint64_t B, const double *__restrict__ ta,
                                                    const double *__restrict__ tb, double e_core) {
    double x1 = 0.0, x2 = 0.0;
    for (uint64_t m = A; m; m &= m - 1) x1 += tb[__ffsll((long long)m)];  // row[1 + p], p = ffs - 1
    for (uint64_t m = B; m; m &= m - 1) x2 += ta[__ffsll((long long)m)];
    return e_core + ((ta[0] + tb[0]) + 0.5 * (x1 + x2));
}
#endif
__host__ __device__ inline int rep_pair(uint64_t e) { return (int)(e >> 49); }

// Packed index of the unordered orbital pair {a, b}.
__host__ __device__ inline int pair_index(int a, int b) {
    int hi = a > b ? a : b, lo = a > b ? b : a;
    return hi * (hi + 1) / 2 + lo;
}

struct fci_das_layout {
    int n_spaces = 0;
    int space_orbs[8] = {0};
    int space_off[8] = {0};
    int ref_a[8] = {0}, ref_b[8] = {0};
    int max_transfer = 0;
    // per-spin patterns (all patterns with excess <= max_transfer + 1)
    int n_pat_a = 0, n_pat_b = 0;
    std::vector<int> pat_a, pat_b;          // [n_pat][n_spaces]
    std::vector<int> exc_a, exc_b;          // excess per pattern
    std::vector<int64_t> pat_nstr_a, pat_nstr_b;
    // categories: target (excess <= T) then intermediate-only (excess == T+1)
    int n_cat = 0, n_cat_int = 0;
    std::vector<int> cat_pa, cat_pb;        // pattern ids
    std::vector<int64_t> cat_off;           // offsets in the intermediate space order
    int64_t n_det = 0, n_det_int = 0;
    // device arrays
    int32_t *d_cat_of_pair = nullptr;       // [n_pat_a * n_pat_b] -> category index or -1
    int32_t *d_loc_a = nullptr;             // [n_str_a]: local index of each global alpha string
    int32_t *d_pat_of_a = nullptr;          // [n_str_a]: pattern id (or -1 if excess > T+1)
    int32_t *d_loc_b = nullptr, *d_pat_of_b = nullptr;
    int64_t *d_pat_nstr_b = nullptr;        // [n_pat_b]
    int32_t *d_cat_pa = nullptr, *d_cat_pb = nullptr;  // [n_cat_int]
    int64_t *d_cat_off = nullptr;           // [n_cat_int + 1]
    int32_t *d_str_of_loc_a = nullptr;      // [n_pat_a][max local] -> global alpha index
    int32_t *d_str_of_loc_b = nullptr;
    int64_t *d_pat_locbase_a = nullptr, *d_pat_locbase_b = nullptr;  // offsets into str_of_loc
    // split-precision operands (built on first use): replacement tables that pack the
    // target string's pattern and local index, block offsets per pattern pair, and the
    // G digit slices in the layout of the MMA's B operand
    int32_t *d_dz_rep_a = nullptr, *d_dz_rep_b = nullptr;  // [n_pair_pad][n_str]
    int32_t *d_dz_base = nullptr;  // [target | intermediate block offset per pattern pair (-1: none) | n_str_b]
    void *d_dz_G = nullptr;
    int dz_slices = 0, dz_shG = 0;
    // the two-pass form (s >= 4): G digit slices in the A-tile layout of the bulk-copy GEMM
    void *d_dg_G = nullptr;
    int dg_slices = 0, dg_shG = 0;
    // kernel configuration chosen by the tuner for dz_tuned_slices (0: none)
    int dz_tuned_slices = 0, dz_tuned_kch = 0, dz_tuned_pw = 0;
};

struct fci_context {
    int device = 0;
    std::string err;

    // integrals
    int n_orb = 0;
    int dtype = -1;
    double e_core = 0.0;
    std::vector<double> h1, g2;  // host copies (interleaved complex for C128)

    // strings
    int mode = FCI_MODE_NONE;
    int na = 0, nb = 0;
    int64_t nsa = 0, nsb = 0, ndet = 0;
    int nent_a = 0, nent_b = 0;
    int npair = 0;
    int npair_pad = 0;  // rows of the dense pair tables: n_pair rounded up to 16 (extra rows = -1)

    uint64_t *d_binom = nullptr;   // [65*65]
    uint64_t *d_str_a = nullptr, *d_str_b = nullptr;
    uint64_t *d_rep_a = nullptr, *d_rep_b = nullptr;  // [ns * nent] packed entries
    int32_t *d_pair_a = nullptr, *d_pair_b = nullptr; // [npair][ns]: (target<<1)|neg or -1
    int32_t *d_pair_a_t = nullptr, *d_pair_b_t = nullptr;  // the same, string-major [ns][npair_pad]
                                                            // (built by the compressed sigma on first use)

    // contraction matrix G = 1/2 g' (packed real [npair x npair], or complex [n^2 x n^2])
    double *d_G = nullptr;
    // diagonal helpers: h_pp, J_pq = (pp|qq), K_pq = (pq|qp) (real parts)
    double *d_hd = nullptr, *d_J = nullptr, *d_K = nullptr;
    // per alpha and beta string (alpha strings first, n_orb + 1 doubles each): the string's
    // own one- and two-electron diagonal energy, then sum_{q in string} J_pq for every p;
    // filled by launch_diag_strings before each use of the diagonal (alpha/beta modes)
    double *d_dstr = nullptr;
    // Ozaki split of G (bf16 digit slices, canonical UMMA layout) and its scale
    void *d_Gs = nullptr;
    int Gs_slices = 0;
    double G_scale = 0.0;  // |G| <= 2^G_exp
    int G_exp = 0;
    int oz_tuned_nt[9] = {0};    // determinants per tile chosen by the tuner, per slice count (0: default)
    int oz_tuned_path[9] = {0};  // 1: two-pass path (D digit image + bulk-copy GEMM) chosen by the tuner
    void *d_Gt = nullptr;        // G digit image in the GEMM's A-tile layout (two-pass path)
    int Gt_slices = 0;

    fci_das_layout das;
    bool das_active = false;

    // phase timing (CUDA events around the sigma kernels)
    bool timing = false;
    std::vector<cudaEvent_t> ev_pool;
    struct ev_rec { cudaEvent_t a, b; int phase; int launches; };
    std::vector<ev_rec> ev_pending;
    size_t ev_used = 0;
    double phase_ms[FCI_N_PHASES] = {0, 0, 0, 0};
    int64_t phase_launches[FCI_N_PHASES] = {0, 0, 0, 0};

    // CUDA graphs of sigma builds, keyed by their arguments
    struct graph_rec {
        const void *C;
        void *sigma;
        int precision, n_slices;
        void *ws;
        cudaStream_t stream;
        cudaGraphExec_t exec;
    };
    std::vector<graph_rec> graphs;

    // device status word owned by the handle: a split-precision sigma whose bounded wait
    // expired records FCI_ERR_TIMEOUT here (through its scatter kernel); it stays set until
    // fci_sync_status reads and clears it, whatever happens to the caller's workspace
    int *d_status = nullptr;

    // scratch for reductions (small)
    double *d_small = nullptr;
    size_t small_bytes = 0;
};

// ---------------------------------------------------------------- helpers
int fci_fail(fci_context *h, int code, const char *fmt, ...);
int fci_cuda_check(fci_context *h, cudaError_t e, const char *what);
int fci_dev_alloc(fci_context *h, void **p, size_t bytes);
void fci_dev_free(void *p);
#define FCI_CUDA(h, call)                                            \
    do {                                                             \
        cudaError_t _e = (call);                                     \
        if (_e != cudaSuccess) return fci_cuda_check((h), _e, #call); \
    } while (0)

inline int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }

// Phase timing: phase_begin records an event before a group of kernel launches and
// phase_end one after; both are no-ops unless timing is enabled on the handle.
struct phase_scope {
    fci_context *h;
    cudaStream_t s;
    int phase, launches;
    cudaEvent_t a = nullptr;
    phase_scope(fci_context *h_, cudaStream_t s_, int phase_, int launches_);
    ~phase_scope();
};

// ------------------------------------------------------------- launchers
// strings.cu
cudaError_t launch_strings_unrank(int m, int ne, int64_t ns, const uint64_t *binom, uint64_t *out,
                                  cudaStream_t s);
cudaError_t launch_repl_table(int m, int ne, int64_t ns, const uint64_t *str, const uint64_t *binom,
                              int n_ent, int packed_pairs, uint64_t *rep, int32_t *pairtab,
                              int npair, cudaStream_t s);
cudaError_t launch_export_repl(int64_t ns, int n_ent, const uint64_t *rep, int32_t *dst, cudaStream_t s);

// sigma_fp64.cu
cudaError_t launch_gather_fci_r64(const fci_context *h, const double *C, double *D, cudaStream_t s);
cudaError_t launch_scatter_fci_r64(const fci_context *h, const double *E, const double *C,
                                   double *sigma, cudaStream_t s);
cudaError_t launch_dgemm(int M, int64_t N, int K, const double *A, const double *B, int64_t ldb,
                         double *C, int64_t ldc, cudaStream_t s);
// Per-string diagonal tables (d_dstr) from the current integrals.
cudaError_t launch_diag_strings(const fci_context *h, cudaStream_t s);
cudaError_t launch_diag_fci(const fci_context *h, double *diag, cudaStream_t s);

// spinor.cu
cudaError_t launch_gather_spinor(const fci_context *h, const double *C, double *D, cudaStream_t s);
cudaError_t launch_scatter_spinor(const fci_context *h, const double *E, const double *C,
                                  double *sigma, cudaStream_t s);
cudaError_t launch_zgemm(int M, int64_t N, int K, const double *A, const double *B, int64_t ldb,
                         double *C, int64_t ldc, cudaStream_t s);
cudaError_t launch_diag_spinor(const fci_context *h, double *diag, cudaStream_t s);

// das.cu
int das_build(fci_context *h, int n_spaces, const int *orbs, const int *ref_a, const int *ref_b,
              int max_transfer, cudaStream_t s);
void das_free(fci_context *h);
int das_sigma_fp64(fci_context *h, const double *C, double *sigma, void *ws, size_t ws_bytes,
                   cudaStream_t s);
int das_sigma_oz(fci_context *h, const double *C, double *sigma, int n_slices, void *ws,
                 size_t ws_bytes, cudaStream_t s);
size_t das_workspace_bytes(const fci_context *h, int precision, int n_slices);
cudaError_t launch_diag_das(const fci_context *h, double *diag, cudaStream_t s);
cudaError_t launch_das_export_address(const fci_context *h, int64_t *dst, cudaStream_t s);

// ozaki_das.cu
size_t dz_workspace_bytes(const fci_context *h, int n_slices);
int dz_sigma(fci_context *h, const double *C, double *sigma, int n_slices, void *ws, size_t ws_bytes,
             cudaStream_t s);
int dz_sigma_group(fci_context *const *hs, const double *const *Cs, double *const *sigmas, void *const *wss, int n,
                   int s, cudaStream_t st);
void dz_free(fci_das_layout &L);
int dz_tune_candidates(const fci_context *h, int n_slices, int *kch, int *pw, int max);  // fitting configurations
void dz_set_config(fci_context *h, int n_slices, int kch, int pw);                     // kch = 0: default
int dz_check(fci_context *h, int n_slices);  // FCI_OK if the DAS split path takes this problem
int das_split_check(fci_context *h, int n_slices);  // either DAS split form (s <= 3 fused, s >= 4 two-pass)
int dg_check(fci_context *h, int n_slices);         // the DAS two-pass split form (s = 4 .. 8)
size_t dg_workspace_bytes(const fci_context *h, int n_slices);
int dg_sigma(fci_context *h, const double *C, double *sigma, int n_slices, void *ws, cudaStream_t s);

// ozaki_cplx.cu (spinor strings, complex integrals)
int cz_check(fci_context *h, int n_slices);
size_t cz_workspace_bytes(const fci_context *h, int n_slices);
int cz_sigma(fci_context *h, const double *C, double *sigma, int n_slices, void *ws, size_t ws_bytes, cudaStream_t s);

// ozaki.cu
cudaError_t launch_to_fixed64(const double *C, int64_t n, int s, unsigned long long *maxbits, int64_t *Cint, int *shC,
                              cudaStream_t st);
int oz_prepare_G(fci_context *h, int n_slices);
int oz_tune_candidates(const fci_context *h, int n_slices, int *nt, int *path, int max);  // configurations that fit
void oz_set_config(fci_context *h, int n_slices, int nt, int path);                     // nt = 0: default
size_t oz_workspace_bytes(const fci_context *h, int n_slices);
int oz_sigma_fci(fci_context *h, const double *C, double *sigma, int n_slices, void *ws,
                 size_t ws_bytes, cudaStream_t s);
int oz_sigma_group(fci_context *const *hs, const double *const *Cs, double *const *sigmas, void *const *wss, int n,
                   int s, cudaStream_t st);

// davidson.cu
struct fci_davidson_state;
int davidson_state_begin(fci_context *h, const fci_davidson_opts *o, const void *guess, void *ws, cudaStream_t s,
                         fci_davidson_state **out);
int davidson_state_advance(fci_davidson_state *st, int *done);
void davidson_state_request(const fci_davidson_state *st, const void **x, void **y, int *prec, int *slices,
                            void **sig_ws, size_t *sig_bytes);
int davidson_state_finish(fci_davidson_state *st, void *C_out, double *energy, fci_davidson_log *log);
fci_context *davidson_state_handle(const fci_davidson_state *st);
int davidson_run(fci_context *h, const fci_davidson_opts *o, double *C_io, double *energy,
                 fci_davidson_log *log, void *ws, size_t ws_bytes, cudaStream_t s);
size_t davidson_ws_bytes(const fci_context *h, const fci_davidson_opts *o);

// fci_api.cu
int sigma_dispatch(fci_context *h, const void *C, void *sigma, int precision, int n_slices,
                   void *ws, size_t ws_bytes, cudaStream_t s);
size_t sigma_ws_bytes(const fci_context *h, int precision, int n_slices);
