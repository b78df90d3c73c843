/*
 * fci.h -- C ABI of libfci: the sigma = H C build of string-based configuration
 * interaction (CI) inside a Davidson eigensolver, on one NVIDIA GB300 (sm_103a).
 *
 * Problem (arXiv 2505.20375, "Methods", Eqs. sigmaL, sigmaL1e, sigmaL2e):
 *   H = e_core + sum_pq h_pq E_pq + 1/2 sum_pqrs (pq|rs) (E_pq E_rs - delta_qr E_ps)
 *     = e_core + sum_pq h'_pq E_pq + 1/2 sum_pqrs (pq|rs) E_pq E_rs,
 *   h'_pq = h_pq - 1/2 sum_r (pr|rq),
 * over determinants built from occupation strings: alpha x beta strings of n spatial
 * orbitals (real, spin-free integrals) or single strings of n spinors (complex
 * Hermitian integrals, the paper's two-spinor X2C case).  sigma is evaluated as
 *   D[rs,K] = sum_J <K|E_rs|J> C_J           (gather over single replacements)
 *   E[pq,K] = sum_rs g'_pqrs D[rs,K]          (dense contraction, on tensor cores)
 *   sigma_I = e_core C_I + 1/2 sum_pq sum_K <I|E_pq|K> E[pq,K]   (gather-back)
 * with g'_pqrs = (pq|rs) + (h'_pq delta_rs + delta_pq h'_rs)/N_e folding the one-electron
 * term into the contraction (sum_r E_rr = N_e on an N_e-electron space).
 *
 * Conventions (all tables compare bit for bit with an independent CPU code):
 *   - a string is a bit mask, orbital p = bit p; strings are listed in ascending integer
 *     order, so the index of a string is its combinadic rank sum_j C(p_j, j) over its
 *     occupied orbitals p_1 < p_2 < ... (0-based p, 1-based j);
 *   - determinant |I> = prod_{p in alpha, ascending} a+_{p,alpha} prod_{p in beta,
 *     ascending} a+_{p,beta} |0>; address I = I_alpha * N_beta + I_beta;
 *   - the single-replacement list of string S holds, for each occupied a (ascending)
 *     and each b (ascending) empty in S or equal to a, the string T = S - a + b, the
 *     pair (a, b) and the sign <S|a+_a a_b|T> = (-1)^(number of electrons of S strictly
 *     between a and b).  It has n_e (n_h + 1) entries per string, the size the paper's
 *     Introduction gives for one-electron excitation lists.
 *
 * Memory: every large buffer (CI vectors, sigma, workspaces, Davidson subspace) is
 * allocated by the caller on the handle's device and passed as a plain device pointer;
 * the library borrows it for the duration of the call.  The handle owns only small
 * device arrays (integrals, string tables, category metadata).  Calls that take a
 * stream are asynchronous on it unless stated otherwise.
 *
 * Errors: every function returns an fci_status; on failure fci_last_error(h) returns
 * a message (valid until the next call on h).  Invalid arguments never reach a kernel.
 */
#ifndef FCI_H
#define FCI_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct fci_context *fci_handle;
/* A cudaStream_t passed as an opaque pointer (NULL = the legacy default stream). */
typedef void *fci_stream;

typedef enum {
    FCI_OK = 0,
    FCI_ERR_ARG = 1,            /* invalid argument or size */
    FCI_ERR_OOM = 2,            /* a device or host allocation failed (nothing leaked) */
    FCI_ERR_CUDA = 3,           /* a CUDA runtime error; message in fci_last_error */
    FCI_ERR_NOT_CONVERGED = 4,  /* Davidson hit max_iter; best Ritz pair returned */
    FCI_ERR_TIMEOUT = 5,        /* a bounded device-side wait expired */
    FCI_ERR_UNSUPPORTED = 6,    /* valid request this build does not implement */
    FCI_ERR_STATE = 7           /* call out of order (e.g. sigma before strings) */
} fci_status;

enum { FCI_R64 = 0, FCI_C128 = 1 };              /* integral / vector element type */
enum { FCI_MODE_NONE = 0, FCI_MODE_FCI = 1, FCI_MODE_SPINOR = 2, FCI_MODE_DAS = 3 };
enum {
    FCI_PREC_FP64 = 0,      /* every step in IEEE binary64 */
    FCI_PREC_OZ_BF16 = 1    /* contraction split into bf16 slices on tcgen05 (Ozaki) */
};

typedef struct {
    int mode;               /* FCI_MODE_* */
    int dtype;              /* FCI_R64 or FCI_C128 */
    int n_orb;              /* spatial orbitals (FCI, DAS) or spinors (SPINOR) */
    int n_alpha, n_beta;    /* electrons per spin; SPINOR: n_alpha = electrons, n_beta = -1 */
    int n_pair;             /* rows of D/E: n(n+1)/2 (real, pair-packed) or n*n (complex) */
    int n_ent_alpha, n_ent_beta;   /* single-replacement entries per string */
    int64_t n_str_alpha, n_str_beta;
    int64_t n_det;          /* length of C and sigma */
    int64_t n_det_intermediate;    /* DAS: determinants of the intermediate space */
    int n_categories;       /* DAS target categories (0 otherwise) */
    int n_categories_intermediate;
} fci_info;

/* ---------------------------------------------------------------- handles */

/* Create a handle bound to CUDA device `device` (made current for every later call on
 * the handle).  *out receives the handle, or NULL on failure. */
int fci_create(fci_handle *out, int device);
/* Free the handle's own device arrays.  Safe on NULL. */
int fci_destroy(fci_handle h);
/* Message of the last failed call on h ("" if none).  h may be NULL (global message). */
const char *fci_last_error(fci_handle h);
/* Fill *out with the handle's current problem description. */
int fci_get_info(fci_handle h, fci_info *out);

/* Number of determinants C(n,k) products for a space, on the host (no device use):
 * FCI: C(n,na) C(n,nb); SPINOR (nb < 0): C(n,na).  Returns -1 on overflow/bad input. */
int64_t fci_count_determinants(int n_orb, int n_alpha, int n_beta);

/* ------------------------------------------------------------- problem setup */

/* Integrals of the Hamiltonian above (Methods, Eq. sigmaL1e uses h', Eq. sigmaL2e g).
 *   n_orb: 1..32 (R64) or 1..64 (C128);
 *   h1: HOST pointer, n_orb x n_orb row-major, double (R64) or interleaved complex
 *       (C128, h_pq = conj(h_qp));
 *   g2: HOST pointer, (pq|rs) at ((p*n+q)*n+r)*n+s, chemists' notation, same type;
 *       R64 needs the 8-fold symmetry of real orbitals, C128 needs (pq|rs) = (rs|pq)
 *       and conj((pq|rs)) = (qp|sr).  Symmetry is checked to 1e-12 (FCI_ERR_ARG).
 *   e_core: constant added to H.
 * Copies both arrays; may be called again to replace the integrals of a handle. */
int fci_setup_integrals(fci_handle h, int n_orb, int dtype, const void *h1, const void *g2,
                        double e_core, fci_stream stream);

/* Build the occupation strings and their single-replacement lists on the device
 * (string enumeration by combinadic unranking; list targets ranked with warp ballots
 * and popc).  n_beta >= 0: alpha/beta strings, FCI determinants (needs R64 integrals);
 * n_beta < 0: one spinor string of n_alpha electrons per determinant (needs C128).
 * Must follow fci_setup_integrals.  Resets any DAS layout.  Synchronous. */
int fci_build_strings(fci_handle h, int n_alpha, int n_beta, fci_stream stream);

/* STP-DAS layout (Results: categorical decomposition C = (+)_B C^B; Methods: the
 * categorical sigma build).  The n_orb orbitals are split into n_spaces contiguous
 * ranges of orbs_per_space[s] orbitals.  Per spin, a pattern is the tuple of electron
 * counts per space; a category is an (alpha pattern, beta pattern) pair whose
 * spin-resolved excess over the reference occupation (ref_alpha, ref_beta per space),
 * summed over spaces and spins, is at most max_transfer.  Categories are ordered
 * lexicographically, blocks are row-major [alpha-local][beta-local], local indices are
 * mixed-radix over spaces (space 0 most significant) of per-space string ranks.
 * Afterwards C and sigma are in DAS order (info.n_det entries), and sigma is P H P
 * over the DAS space: the intermediate determinants of the resolution E_pq E_rs range
 * over the categories within max_transfer + 1.  Requires R64 alpha/beta strings of
 * n_orb <= 32.  Synchronous. */
int das_build_categories(fci_handle h, int n_spaces, const int *orbs_per_space,
                         const int *ref_alpha, const int *ref_beta, int max_transfer,
                         fci_stream stream);

/* H_II for every determinant of the current layout into the device array diag
 * (info.n_det doubles; real also for C128, where H_II is real): the diagonal that the
 * Davidson preconditioner divides by (Results, Eqs. davidsonPreconditioner and
 * sparsePreconditioner).  FCI_ERR_STATE before fci_build_strings.  Asynchronous. */
int fci_diagonal(fci_handle h, double *diag, fci_stream stream);

/* ------------------------------------------------------------------- sigma */

/* Bytes of device workspace fci_sigma needs for n_vec vectors at this precision. */
int fci_sigma_workspace_bytes(fci_handle h, int n_vec, int precision, int n_slices,
                              size_t *bytes);

/* sigma = H C for n_vec vectors (Methods, Eqs. sigmaL, sigmaL1e, sigmaL2e).
 *   C, sigma: DEVICE pointers, n_vec x info.n_det, vector-major, double (R64) or
 *             interleaved complex (C128); must not overlap;
 *   precision: FCI_PREC_FP64, or FCI_PREC_OZ_BF16 with n_slices digit slices of each
 *             operand of the contraction (signed 8-bit digits held exactly in f16;
 *             7-bit digits for spinor strings): alpha/beta strings (R64) take 2..7
 *             slices (n_orb <= 15; 6 and 7 reach the FP64 tolerance); the DAS layout
 *             takes 2 or 3 slices (n_orb <= 17; one fused kernel, E stored in FP32, for
 *             the first phase of a mixed-precision solve) or 4 and more while
 *             n_slices x n_pair <= 1023 (two passes: a digit image of D, then the
 *             bulk-copy GEMM with exact int64 E; 6 and 7 reach the FP64 tolerance, the
 *             workspace holds up to 96 GiB of E and 24 GiB of digit image); spinor
 *             strings with complex integrals take 2..8 slices of 7 bits (8 reaches the
 *             FP64 tolerance); FCI_ERR_UNSUPPORTED otherwise;
 *   workspace: DEVICE pointer, >= fci_sigma_workspace_bytes, 256-byte aligned.
 * Asynchronous on `stream`. */
int fci_sigma(fci_handle h, const void *C, void *sigma, int n_vec, int precision,
              int n_slices, void *workspace, size_t workspace_bytes, fci_stream stream);

/* Bytes of device workspace fci_sigma_host needs: room for n_vec vectors of C and of
 * sigma on the device, then fci_sigma's own workspace. */
int fci_sigma_host_workspace_bytes(fci_handle h, int n_vec, int precision, int n_slices,
                                   size_t *bytes);

/* sigma = H C as fci_sigma, with C and sigma in HOST memory (n_vec x info.n_det,
 * vector-major, same element types; must not overlap).  The call copies C into the
 * front of the DEVICE workspace on `stream`, builds sigma there as fci_sigma does, copies
 * it back into sigma_host and waits for the copy: pinned (page-locked) host buffers let
 * the copies run asynchronously at the link rate, pageable ones go through the CUDA driver's
 * staging.  Synchronous; it reports a device-side failure of this build as
 * fci_sync_status does (FCI_ERR_TIMEOUT, sigma_host then holds NaN) and clears it.
 *   workspace: DEVICE pointer, >= fci_sigma_host_workspace_bytes, 256-byte aligned. */
int fci_sigma_host(fci_handle h, const void *C_host, void *sigma_host, int n_vec,
                   int precision, int n_slices, void *workspace, size_t workspace_bytes,
                   fci_stream stream);

/* ---------------------------------------------------------------- Davidson */

typedef struct {
    int max_iter;           /* default 100 */
    int max_subspace;       /* 2..32, default 32; collapse to the last two Ritz vectors */
    double tol_residual;    /* ||r|| threshold, default 1e-6 */
    double tol_energy;      /* |dE| threshold, default 1e-10 */
    double eps;             /* compression-compatible preconditioner threshold (Eq.
                               sparsePreconditioner), default 0 = Davidson's own; a
                               negative value selects 10 / sqrt(N_dets), the largest
                               threshold the paper found to converge reliably */
    int precision;          /* FCI_PREC_* used for sigma in the first phase */
    int n_slices;           /* slices for FCI_PREC_OZ_BF16 */
    double switch_residual; /* mixed mode: once ||r|| <= this, restart from the Ritz
                               vector with the final precision (default 1e-5) */
    int use_guess;          /* 1: start from C_io; 0: unit vector at min H_II */
    int final_precision;    /* sigma after the switch: FCI_PREC_FP64 (default), or
                               FCI_PREC_OZ_BF16 with final_slices >= 6 (error below
                               1e-11 of ||sigma||, the FP64 parity bar; on the DAS
                               layout the two-pass split form) */
    int final_slices;
    int gap_bound;          /* 1: after convergence, keep the subspace and converge the
                               second Ritz pair as well (until ||r_1|| <= max(tol_residual,
                               (E_1 - E_0) / 4) or max_iter further steps; a full subspace
                               restarts from the ground state and the second Ritz vector),
                               then report the gap lower bound gamma_0^- = (E_1 - ||r_1||)
                               - E_0 and the energy error bound ||r_0||^2 / gamma_0^-
                               (Results, eigenvalue bound analysis, Eq. gammaLowerBound);
                               default 0 */
    int staged_sigma;       /* step-wise ABI: 1 = every sigma request uses the same two
                               vectors of the workspace (x copied in, y copied out by the
                               library), so a caller can replay a captured sigma graph for
                               the whole solve; default 0 */
    double start_mix;       /* without a guess, the start vector is the unit vector at min
                               H_II plus start_mix times a pseudo-random vector of norm ~1
                               (splitmix64 of the index), normalised; default 1e-2.  The
                               admixture reaches every symmetry sector, so the solve finds
                               the lowest eigenvalue of H; 0 gives the bare unit vector,
                               which for a closed-shell determinant of an M_s = 0 space is
                               symmetric under alpha <-> beta exchange and converges to the
                               lowest state of that sector only */
} fci_davidson_opts;

typedef struct {
    int iteration;
    int precision;          /* precision of the sigma used in this iteration */
    double energy;          /* Ritz value + e_core */
    double delta_energy;    /* energy - previous energy (0 on the first iteration) */
    double max_delta_c;     /* max_i |c_i - c_i(previous)| (0 on the first) */
    double residual_norm;   /* ||sigma_c - E c|| */
    double seconds;         /* wall time of the iteration */
} fci_davidson_iter;

typedef struct {
    int n_iter;             /* iterations recorded in iters (<= capacity) */
    int converged;
    int n_sigma;            /* sigma builds performed */
    int capacity;           /* caller sets: length of iters (may be 0 with iters NULL) */
    fci_davidson_iter *iters;
    /* gap_bound = 1 only (NaN otherwise): the second Ritz value E_1 and its residual norm,
     * the ground state's residual norm, gamma_0^- and the error bound ||r_0||^2 / gamma_0^-
     * (+inf if gamma_0^- <= 0), and the iterations spent on the second pair */
    double e1, r1_norm, r0_norm, gap_lower, error_bound;
    int gap_iterations;
} fci_davidson_log;

/* Default options. */
void fci_davidson_default_opts(fci_davidson_opts *opts);

/* Device workspace davidson_solve needs (subspace vectors, sigma vectors, diagonal,
 * scratch and the fci_sigma workspace). */
int fci_davidson_workspace_bytes(fci_handle h, const fci_davidson_opts *opts, size_t *bytes);

/* Lowest eigenpair by Davidson (Results: Ritz residual appended each iteration,
 * preconditioner of Eq. sparsePreconditioner with guard |lambda - H_ii| >= 1e-12).
 * All vector work, the projected eigenproblem and the Rayleigh quotient run on the
 * device in FP64; the host only reads the Ritz value and residual norm per iteration.
 *   C_io: DEVICE pointer, info.n_det elements: guess in (if opts->use_guess), Ritz
 *         vector out (unit norm);
 *   energy: HOST pointer, receives the lowest Ritz value + e_core;
 *   log: optional HOST pointer (per-iteration table of the paper's Tables 1-3).
 * Synchronous.  Returns FCI_ERR_NOT_CONVERGED (with the best pair) at max_iter. */
int davidson_solve(fci_handle h, const fci_davidson_opts *opts, void *C_io, double *energy,
                   fci_davidson_log *log, void *workspace, size_t workspace_bytes,
                   fci_stream stream);

/* fci_sigma for one vector, replayed from a CUDA graph: the first call with a given
 * (C, sigma, precision, n_slices, workspace, stream) runs the sigma once, then captures
 * its kernel sequence into a graph kept in the handle (at most 64 graphs; the oldest is
 * dropped); later calls with the same arguments launch the graph.  Must not be called
 * while `stream` is itself being captured.  Results equal fci_sigma's. */
int fci_sigma_graph(fci_handle h, const void *C, void *sigma, int precision, int n_slices, void *workspace,
                    size_t workspace_bytes, fci_stream stream);
/* Drop the handle's cached sigma graphs (e.g. before freeing the buffers they name). */
int fci_clear_graphs(fci_handle h);

/* Autotuning of the split-precision contraction's tile shape for this problem.
 * Candidates: alpha/beta strings, the fused kernel with 64 or 32 determinants per tile
 * of the MMA, or the two-pass path (a digit image of D written to the workspace, then a
 * GEMM whose operand tiles arrive by cp.async.bulk);
 * DAS layout, the K-chunk width of the operand ring (6, 4 or 2 cores of 8 pairs) and
 * the number of producer warps (12 or 8), where shared memory allows.  Every candidate
 * runs one untimed and `reps` timed FCI_PREC_OZ_BF16 sigma builds of C (DEVICE, n_det
 * values; sigma is overwritten) with n_slices slices, timed by CUDA events on `stream`;
 * the fastest is kept in the handle and used by every later split sigma with n_slices
 * slices (the results do not depend on it: the arithmetic is exact integer).  Cached
 * sigma graphs are dropped.  Host-synchronous.  `report` (may be NULL) receives the
 * candidates, their mean times and the choice.  FCI_ERR_UNSUPPORTED for spinor strings
 * or slice counts the split path does not take. */
typedef struct {
    int n_candidates;
    int chosen;          /* index of the kept candidate */
    int param_a[8];      /* alpha/beta: determinants per tile; DAS: K-chunk cores */
    int param_b[8];      /* alpha/beta: 0 fused, 1 two-pass; DAS: producer warps */
    double ms[8];        /* mean time of one sigma build */
} fci_tune_report;

int fci_tune_sigma(fci_handle h, int n_slices, const void *C, void *sigma, void *workspace,
                   size_t workspace_bytes, int reps, fci_stream stream, fci_tune_report *report);

/* ------------------------------------------------- grouped sigma, step-wise Davidson */

/* One sigma build of a batch: sigma = H C for one vector of the problem held by handle. */
typedef struct {
    fci_handle handle;
    const void *C;          /* DEVICE, info.n_det elements */
    void *sigma;            /* DEVICE, info.n_det elements */
    int precision;          /* FCI_PREC_* */
    int n_slices;
    void *workspace;        /* DEVICE, >= fci_sigma_workspace_bytes of the job's handle */
    size_t workspace_bytes;
} fci_sigma_job;

/* sigma builds of several problems (different handles, sizes and integrals) in one pass
 * on `stream`: jobs that use FCI_PREC_OZ_BF16 with the same slice count share ONE
 * persistent launch of the tcgen05 contraction kernel (the uneven tile ranges of all jobs
 * in one grid, CTAs split in proportion to each job's tiles; alpha/beta-string jobs and
 * DAS jobs form separate launches); the other jobs run one after another.  All handles must be on the same device; a handle may
 * appear in at most one job.  Asynchronous.  This is the batching the serving loop uses
 * for the sigma builds of concurrent Davidson solves (not a step of the paper's method). */
int fci_sigma_grouped(const fci_sigma_job *jobs, int n_jobs, fci_stream stream);

/* fci_sigma_grouped replayed from a CUDA graph: the first call with a given job list (every
 * field of every job equal, same stream) runs it once, then captures its launches into a
 * graph kept in a process-wide cache (at most 16 lists; the oldest is dropped); later
 * calls with the same list launch the graph.  Destroying a handle, or rebuilding its
 * strings or integrals, drops the graphs that name it.  `stream` must not be the legacy
 * default stream (the list is then run without a graph) nor itself be capturing.  Results
 * equal fci_sigma_grouped's.  This is how the serving loop replays the batched sigma
 * builds of its active solves while the set of solves does not change. */
int fci_sigma_grouped_graph(const fci_sigma_job *jobs, int n_jobs, fci_stream stream);
/* Drop every cached grouped graph. */
int fci_clear_grouped_graphs(void);

typedef struct fci_davidson_state *fci_davidson_handle;

/* Davidson driven by the caller's sigma products (same iteration as davidson_solve):
 *   davidson_begin  sets up the solve (diagonal, start vector C_guess or, without one,
 *                   the start of opts->start_mix) and requests the first product;
 *   davidson_request returns the pending request: y (DEVICE) must receive H x, with the
 *                   precision and slice count this iteration uses, and the part of the
 *                   Davidson workspace reserved for the sigma build;
 *   davidson_advance consumes y = H x, updates the subspace and either sets *done or
 *                   leaves a new request;
 *   davidson_finish  copies the Ritz vector to C_out (DEVICE, may be NULL), returns the
 *                   energy and log, and frees the state (also after an error).
 * One solve at a time per handle (the handle's small scratch holds the projected matrix). */
int davidson_begin(fci_handle h, const fci_davidson_opts *opts, const void *C_guess, void *workspace,
                   size_t workspace_bytes, fci_stream stream, fci_davidson_handle *out);
int davidson_request(fci_davidson_handle st, const void **x, void **y, int *precision, int *n_slices,
                     void **sigma_workspace, size_t *sigma_workspace_bytes);
int davidson_advance(fci_davidson_handle st, int *done);
int davidson_finish(fci_davidson_handle st, void *C_out, double *energy, fci_davidson_log *log);

/* ------------------------------------------------------------ table export */

enum {
    FCI_TABLE_STRINGS_ALPHA = 0,    /* uint64[n_str_alpha] masks (SPINOR: the strings) */
    FCI_TABLE_STRINGS_BETA = 1,     /* uint64[n_str_beta] */
    FCI_TABLE_REPL_ALPHA = 2,       /* int32[n_str_alpha * n_ent_alpha * 4]: per entry
                                       {target, a, b, sign} */
    FCI_TABLE_REPL_BETA = 3,
    FCI_TABLE_DAS_CATEGORIES = 4,   /* int64[n_cat * (2*n_spaces + 3)]: alpha pattern,
                                       beta pattern, n_alpha_str, n_beta_str, offset */
    FCI_TABLE_DAS_ADDRESS = 5       /* int64[n_det]: FCI address of each DAS determinant */
};

/* Bytes of a table (0 if the table does not exist in the current layout). */
int fci_table_bytes(fci_handle h, int table, size_t *bytes);
/* Copy a table into a caller DEVICE buffer of at least fci_table_bytes bytes. */
int fci_copy_table(fci_handle h, int table, void *dst, size_t bytes, fci_stream stream);


/* Synchronise `stream` and report device-side failures of earlier calls on h: returns
 * FCI_ERR_TIMEOUT if a bounded wait inside a split-precision kernel expired (its sigma
 * output was then filled with NaN), else FCI_OK.  Clears the recorded status. */
int fci_sync_status(fci_handle h, fci_stream stream);

/* ------------------------------------------------------------ phase timing */

enum { FCI_PHASE_GATHER = 0, FCI_PHASE_CONTRACT = 1, FCI_PHASE_SCATTER = 2, FCI_PHASE_OTHER = 3,
       FCI_N_PHASES = 4 };

/* Enable (1) or disable (0) CUDA-event timing of the sigma phases (gather of D, the
 * contraction E = g' D, the scatter into sigma, other kernels).  Events are recorded on
 * the stream each kernel is launched on.  Adds no synchronisation to fci_sigma. */
int fci_set_phase_timing(fci_handle h, int enable);
/* Synchronise with the recorded events and return, per phase, the summed kernel time
 * in milliseconds (ms[FCI_N_PHASES]) and the number of kernel launches
 * (launches[FCI_N_PHASES]); either pointer may be NULL.  reset != 0 clears the sums. */
int fci_get_phase_times(fci_handle h, double *ms, int64_t *launches, int reset);

/* ------------------------------------------------ categorically compressed sigma */

/* sigma = H C on the DAS layout for a categorically compressed C (Results: categorical
 * compression, C = (+)_B (V^B, A^B), the nonzero coefficients of each category and their
 * addresses in a compressed sparse column; Methods, Algorithm 1 and the compression-
 * preservation argument: only nonzero coefficients contribute and sigma comes out
 * compressed).  Both vectors are given as DAS addresses in ascending order with their
 * values, i.e. the per-category (V, A) arrays of the paper concatenated in category order
 * (a category's local address is its DAS address minus the category's offset).
 *   c_addr, c_val: DEVICE, nnz_c entries: ascending target addresses (< info.n_det) and
 *                  their coefficients (explicit zeros allowed: a listed zero is treated
 *                  as a nonzero of value 0, so it widens the support below by its
 *                  connections, where sigma is then exactly 0);
 *   out_addr, out_val: DEVICE, capacity entries: sigma on its structural support (every
 *                  target determinant that H connects to a nonzero C_K), ascending; the
 *                  values equal the FP64 sigma of the dense vector there, term by term in
 *                  the same order, and the dense sigma is zero elsewhere;
 *   *nnz_sigma:    HOST, receives the size of the support (also when capacity is too small,
 *                  which returns FCI_ERR_ARG);
 *   workspace:     DEVICE, >= fci_sigma_compressed_workspace_bytes(h, nnz_c), 256-byte
 *                  aligned (bounded by nnz_c x (moves per determinant)^2 support entries).
 * D is gathered as Algorithm 1 does (each source looked up among its category's ascending
 * nonzero addresses by exponential search).  On its first call the handle builds
 * string-major copies of its pair tables (n_pair_pad x 4 bytes per alpha and per beta
 * string) and keeps them until the strings are rebuilt.  Real integrals only, at most 32
 * orbitals.  FCI_ERR_ARG for addresses that are not ascending target addresses.
 * Host-synchronous. */
int fci_sigma_compressed_workspace_bytes(fci_handle h, int64_t nnz_c, size_t *bytes);
int fci_sigma_compressed(fci_handle h, const int64_t *c_addr, const double *c_val, int64_t nnz_c,
                         int64_t *out_addr, double *out_val, int64_t capacity, int64_t *nnz_sigma,
                         void *workspace, size_t workspace_bytes, fci_stream stream);

/* ------------------------------------------------------- allocation-free sigma */

/* sigma = H C for ONE vector in FP64, like fci_sigma with precision FCI_PREC_FP64, but
 * with its scratch (the D and E intermediates, 2 x n_pair x n_det elements) in a
 * fixed 64 MiB device array inside libfci instead of a caller workspace.  The paper
 * has no counterpart; this exists for callers that cannot allocate device memory when
 * they need sigma: a process whose framework already reserved the device memory pool,
 * code running where CUDA allocation calls are not allowed (e.g. a host callback on a
 * stream), or a latency-critical loop that must avoid the implicit synchronisation of
 * cudaMalloc/cudaFree.  It calls no allocating routine.
 *   C, sigma: DEVICE pointers, info.n_det elements each (double or interleaved complex),
 *             not overlapping; FCI and spinor layouts (not DAS).
 *   Sizes whose scratch exceeds 64 MiB are rejected with FCI_ERR_ARG (use fci_sigma).
 * The array is a device variable: every GPU that loads libfci holds it until exit.  The
 * first call on each device looks up its address (cudaGetSymbolAddress, with that
 * device current); make that first call before any stream capture.  All calls share
 * the one array and it keeps the last call's contents (every byte a call reads it
 * writes first); calls that overlap on the GPU (other streams, other threads, other
 * handles on the same device) race on it and must be serialised by the caller.
 * Asynchronous on `stream`. */
int fci_sigma_noalloc(fci_handle h, const void *C, void *sigma, fci_stream stream);

#ifdef __cplusplus
}
#endif

#endif /* FCI_H */
