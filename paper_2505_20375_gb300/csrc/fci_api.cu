// C ABI of libfci: handles, argument checking, integral preparation and dispatch.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <complex>
#include <mutex>

#include "fci_internal.h"

static thread_local std::string g_err;  // message for calls without a usable handle
static std::atomic<long> g_alloc_count{0};

int fci_fail(fci_context *h, int code, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    if (h) h->err = buf; else g_err = buf;
    return code;
}

int fci_cuda_check(fci_context *h, cudaError_t e, const char *what) {
    if (e == cudaSuccess) return FCI_OK;
    if (e == cudaErrorMemoryAllocation) {
        cudaGetLastError();
        return fci_fail(h, FCI_ERR_OOM, "%s: %s", what, cudaGetErrorString(e));
    }
    return fci_fail(h, FCI_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

// Device allocation with host-side fault injection: FCI_FAULT_ALLOC_AT=n makes the n-th
// allocation (counting from 1) fail as if the device were out of memory, counting from
// the first allocation that sees the variable with its current value (setting it anew, or
// unsetting it, restarts the count).
int fci_dev_alloc(fci_context *h, void **p, size_t bytes) {
    *p = nullptr;
    {
        static std::mutex mu;
        static std::string seen;
        static long base = 0;
        std::lock_guard<std::mutex> lk(mu);
        const long k = ++g_alloc_count;
        const char *inj = getenv("FCI_FAULT_ALLOC_AT");
        const std::string now = inj ? inj : "";
        if (now != seen) {
            seen = now;
            base = k - 1;
        }
        if (inj && atol(inj) == k - base) return fci_fail(h, FCI_ERR_OOM, "injected allocation failure #%ld", k - base);
    }
    if (bytes == 0) bytes = 16;
    cudaError_t e = cudaMalloc(p, bytes);
    if (e != cudaSuccess) {
        *p = nullptr;
        cudaGetLastError();
        return fci_fail(h, e == cudaErrorMemoryAllocation ? FCI_ERR_OOM : FCI_ERR_CUDA,
                        "cudaMalloc(%zu): %s", bytes, cudaGetErrorString(e));
    }
    return FCI_OK;
}

void fci_dev_free(void *p) {
    if (p) cudaFree(p);
}

// ------------------------------------------------------------ phase timing

static cudaEvent_t take_event(fci_context *h) {
    if (h->ev_used == h->ev_pool.size()) {
        cudaEvent_t e;
        if (cudaEventCreate(&e) != cudaSuccess) { cudaGetLastError(); return nullptr; }
        h->ev_pool.push_back(e);
    }
    return h->ev_pool[h->ev_used++];
}

phase_scope::phase_scope(fci_context *h_, cudaStream_t s_, int phase_, int launches_)
    : h(h_), s(s_), phase(phase_), launches(launches_) {
    if (h->timing) {
        a = take_event(h);
        if (a) cudaEventRecord(a, s);
    }
}

phase_scope::~phase_scope() {
    if (!h->timing || !a) return;
    cudaEvent_t b = take_event(h);
    if (!b) return;
    cudaEventRecord(b, s);
    h->ev_pending.push_back({a, b, phase, launches});
}

static void drain_events(fci_context *h) {
    for (auto &r : h->ev_pending) {
        float ms = 0.f;
        if (cudaEventSynchronize(r.b) == cudaSuccess && cudaEventElapsedTime(&ms, r.a, r.b) == cudaSuccess) {
            h->phase_ms[r.phase] += ms;
            h->phase_launches[r.phase] += r.launches;
        }
    }
    cudaGetLastError();
    h->ev_pending.clear();
    h->ev_used = 0;
}

static int set_dev(fci_context *h) {
    FCI_CUDA(h, cudaSetDevice(h->device));
    return FCI_OK;
}

// Process-wide cache of grouped sigma graphs, keyed by the whole job list and the stream.
namespace {
struct grouped_graph_rec {
    std::vector<fci_sigma_job> jobs;
    cudaStream_t stream;
    int device;
    cudaGraphExec_t exec;
};
std::vector<grouped_graph_rec> g_grouped_graphs;
std::mutex g_grouped_mu;

bool same_jobs(const std::vector<fci_sigma_job> &a, const fci_sigma_job *b, int n) {
    if ((int)a.size() != n) return false;
    for (int i = 0; i < n; ++i)
        if (a[i].handle != b[i].handle || a[i].C != b[i].C || a[i].sigma != b[i].sigma ||
            a[i].precision != b[i].precision || a[i].n_slices != b[i].n_slices || a[i].workspace != b[i].workspace ||
            a[i].workspace_bytes != b[i].workspace_bytes)
            return false;
    return true;
}
}  // namespace

// Drops the grouped graphs that name h (its buffers or tables are about to change).
static void drop_grouped_graphs_of(const fci_context *h) {
    std::lock_guard<std::mutex> lk(g_grouped_mu);
    for (size_t i = 0; i < g_grouped_graphs.size();) {
        bool uses = false;
        for (const auto &j : g_grouped_graphs[i].jobs) uses |= j.handle == h;
        if (uses) {
            cudaGraphExecDestroy(g_grouped_graphs[i].exec);
            g_grouped_graphs.erase(g_grouped_graphs.begin() + i);
        } else {
            ++i;
        }
    }
}

static void drop_graphs(fci_context *h) {
    for (auto &g : h->graphs) cudaGraphExecDestroy(g.exec);
    h->graphs.clear();
    drop_grouped_graphs_of(h);
}

static void free_strings(fci_context *h) {
    drop_graphs(h);
    fci_dev_free(h->d_str_a); fci_dev_free(h->d_str_b);
    fci_dev_free(h->d_rep_a); fci_dev_free(h->d_rep_b);
    fci_dev_free(h->d_pair_a); fci_dev_free(h->d_pair_b);
    fci_dev_free(h->d_pair_a_t); fci_dev_free(h->d_pair_b_t);
    fci_dev_free(h->d_dstr);
    fci_dev_free(h->d_G); fci_dev_free(h->d_hd); fci_dev_free(h->d_J); fci_dev_free(h->d_K);
    fci_dev_free(h->d_Gs);
    fci_dev_free(h->d_Gt);
    h->d_str_a = h->d_str_b = nullptr;
    h->d_rep_a = h->d_rep_b = nullptr;
    h->d_pair_a = h->d_pair_b = nullptr;
    h->d_pair_a_t = h->d_pair_b_t = nullptr;
    h->d_dstr = nullptr;
    h->d_G = h->d_hd = h->d_J = h->d_K = nullptr;
    h->d_Gs = nullptr;
    h->Gs_slices = 0;
    h->d_Gt = nullptr;
    h->Gt_slices = 0;
    das_free(h);
    h->mode = FCI_MODE_NONE;
    h->nsa = h->nsb = h->ndet = 0;
}

static int64_t binom_host(int n, int k) {
    if (k < 0 || n < 0 || k > n) return 0;
    unsigned __int128 r = 1;
    for (int i = 1; i <= k; ++i) {
        r = r * (unsigned __int128)(n - k + i) / i;
        if (r > (unsigned __int128)INT64_MAX) return -1;
    }
    return (int64_t)r;
}

extern "C" {

int64_t fci_count_determinants(int n_orb, int n_alpha, int n_beta) {
    if (n_orb < 0 || n_orb > 128 || n_alpha < 0 || n_alpha > n_orb || n_beta > n_orb) return -1;
    int64_t a = binom_host(n_orb, n_alpha);
    if (a < 0) return -1;
    if (n_beta < 0) return a;
    int64_t b = binom_host(n_orb, n_beta);
    if (b < 0) return -1;
    if (a != 0 && b > INT64_MAX / a) return -1;
    return a * b;
}

int fci_create(fci_handle *out, int device) {
    if (!out) return fci_fail(nullptr, FCI_ERR_ARG, "out is NULL");
    *out = nullptr;
    int ndev = 0;
    cudaError_t e = cudaGetDeviceCount(&ndev);
    if (e != cudaSuccess) { cudaGetLastError(); return fci_fail(nullptr, FCI_ERR_CUDA, "cudaGetDeviceCount: %s", cudaGetErrorString(e)); }
    if (device < 0 || device >= ndev) return fci_fail(nullptr, FCI_ERR_ARG, "device %d out of range (%d devices)", device, ndev);
    fci_context *h = new (std::nothrow) fci_context();
    if (!h) return fci_fail(nullptr, FCI_ERR_OOM, "host allocation failed");
    h->device = device;
    int rc = set_dev(h);
    if (rc) { g_err = h->err; delete h; return rc; }
    // binomial table C(p, j), p, j in [0, 64]
    std::vector<uint64_t> bt(FCI_BINOM_LD * FCI_BINOM_LD, 0);
    for (int p = 0; p < FCI_BINOM_LD; ++p) {
        bt[p * FCI_BINOM_LD] = 1;
        for (int j = 1; j <= p; ++j)
            bt[p * FCI_BINOM_LD + j] = bt[(p - 1) * FCI_BINOM_LD + j - 1] + (j <= p - 1 ? bt[(p - 1) * FCI_BINOM_LD + j] : 0);
    }
    rc = fci_dev_alloc(h, (void **)&h->d_binom, bt.size() * 8);
    if (!rc) rc = fci_cuda_check(h, cudaMemcpy(h->d_binom, bt.data(), bt.size() * 8, cudaMemcpyHostToDevice), "binom upload");
    h->small_bytes = 1 << 20;
    if (!rc) rc = fci_dev_alloc(h, (void **)&h->d_small, h->small_bytes);
    if (!rc) rc = fci_dev_alloc(h, (void **)&h->d_status, 256);
    if (!rc) rc = fci_cuda_check(h, cudaMemset(h->d_status, 0, 256), "status word");
    if (rc) {
        g_err = h->err;
        fci_dev_free(h->d_binom);
        fci_dev_free(h->d_small);
        fci_dev_free(h->d_status);
        delete h;
        return rc;
    }
    *out = h;
    return FCI_OK;
}

int fci_set_phase_timing(fci_handle h, int enable) {
    if (!h) return fci_fail(nullptr, FCI_ERR_ARG, "NULL handle");
    h->timing = enable != 0;
    return FCI_OK;
}

int fci_get_phase_times(fci_handle h, double *ms, int64_t *launches, int reset) {
    if (!h) return fci_fail(nullptr, FCI_ERR_ARG, "NULL handle");
    int rc = set_dev(h);
    if (rc) return rc;
    drain_events(h);
    for (int i = 0; i < FCI_N_PHASES; ++i) {
        if (ms) ms[i] = h->phase_ms[i];
        if (launches) launches[i] = h->phase_launches[i];
        if (reset) { h->phase_ms[i] = 0.0; h->phase_launches[i] = 0; }
    }
    return FCI_OK;
}

int fci_sync_status(fci_handle h, fci_stream stream) {
    if (!h) return fci_fail(nullptr, FCI_ERR_ARG, "NULL handle");
    int rc = set_dev(h);
    if (rc) return rc;
    cudaStream_t s = (cudaStream_t)stream;
    FCI_CUDA(h, cudaStreamSynchronize(s));
    int st = 0;
    FCI_CUDA(h, cudaMemcpy(&st, h->d_status, sizeof st, cudaMemcpyDeviceToHost));
    FCI_CUDA(h, cudaMemset(h->d_status, 0, sizeof st));
    if (st == FCI_ERR_TIMEOUT) return fci_fail(h, FCI_ERR_TIMEOUT, "a bounded device wait expired; sigma was set to NaN");
    if (st) return fci_fail(h, st, "device status %d", st);
    return FCI_OK;
}

int fci_destroy(fci_handle h) {
    if (!h) return FCI_OK;
    cudaSetDevice(h->device);
    drain_events(h);
    for (auto e : h->ev_pool) cudaEventDestroy(e);
    drop_graphs(h);
    free_strings(h);
    fci_dev_free(h->d_binom);
    fci_dev_free(h->d_small);
    fci_dev_free(h->d_status);
    delete h;
    return FCI_OK;
}

const char *fci_last_error(fci_handle h) { return h ? h->err.c_str() : g_err.c_str(); }

int fci_get_info(fci_handle h, fci_info *o) {
    if (!h || !o) return fci_fail(h, FCI_ERR_ARG, "NULL argument");
    memset(o, 0, sizeof *o);
    o->mode = h->mode;
    o->dtype = h->dtype;
    o->n_orb = h->n_orb;
    o->n_alpha = h->na;
    o->n_beta = h->mode == FCI_MODE_SPINOR ? -1 : h->nb;
    o->n_pair = h->npair;
    o->n_ent_alpha = h->nent_a;
    o->n_ent_beta = h->nent_b;
    o->n_str_alpha = h->nsa;
    o->n_str_beta = h->nsb;
    o->n_det = h->das_active ? h->das.n_det : h->ndet;
    o->n_det_intermediate = h->das_active ? h->das.n_det_int : h->ndet;
    o->n_categories = h->das_active ? h->das.n_cat : 0;
    o->n_categories_intermediate = h->das_active ? h->das.n_cat_int : 0;
    return FCI_OK;
}

int fci_setup_integrals(fci_handle h, int n, int dtype, const void *h1, const void *g2, double e_core,
                        fci_stream stream) {
    (void)stream;
    if (!h) return fci_fail(nullptr, FCI_ERR_ARG, "NULL handle");
    if (!h1 || !g2) return fci_fail(h, FCI_ERR_ARG, "NULL integral pointer");
    if (dtype != FCI_R64 && dtype != FCI_C128) return fci_fail(h, FCI_ERR_ARG, "bad dtype %d", dtype);
    if (n < 1 || n > (dtype == FCI_R64 ? 32 : 64)) return fci_fail(h, FCI_ERR_ARG, "n_orb %d out of range", n);
    if (!isfinite(e_core)) return fci_fail(h, FCI_ERR_ARG, "e_core not finite");
    const int w = dtype == FCI_C128 ? 2 : 1;
    const size_t n2 = (size_t)n * n, n4 = n2 * n2;
    std::vector<double> hh((const double *)h1, (const double *)h1 + n2 * w);
    std::vector<double> gg((const double *)g2, (const double *)g2 + n4 * w);
    for (double v : hh) if (!isfinite(v)) return fci_fail(h, FCI_ERR_ARG, "h1 has a non-finite entry");
    for (double v : gg) if (!isfinite(v)) return fci_fail(h, FCI_ERR_ARG, "g2 has a non-finite entry");
    // symmetry checks
    auto H = [&](int p, int q) { return std::complex<double>(hh[(p * n + q) * w], w == 2 ? hh[(p * n + q) * w + 1] : 0.0); };
    auto Gv = [&](int p, int q, int r, int s) {
        size_t i = (((size_t)p * n + q) * n + r) * n + s;
        return std::complex<double>(gg[i * w], w == 2 ? gg[i * w + 1] : 0.0);
    };
    double gmax = 0.0;
    for (double v : gg) gmax = std::max(gmax, fabs(v));
    const double tol = 1e-12 * std::max(1.0, gmax);
    for (int p = 0; p < n; ++p)
        for (int q = 0; q < n; ++q)
            if (std::abs(H(p, q) - std::conj(H(q, p))) > tol) return fci_fail(h, FCI_ERR_ARG, "h1 is not Hermitian at (%d,%d)", p, q);
    for (int p = 0; p < n; ++p)
        for (int q = 0; q < n; ++q)
            for (int r = 0; r < n; ++r)
                for (int s = 0; s < n; ++s) {
                    auto v = Gv(p, q, r, s);
                    if (std::abs(v - Gv(r, s, p, q)) > tol ||
                        std::abs(std::conj(v) - Gv(q, p, s, r)) > tol)
                        return fci_fail(h, FCI_ERR_ARG, "g2 lacks (pq|rs)=(rs|pq)=conj(qp|sr) at (%d,%d,%d,%d)", p, q, r, s);
                    if (dtype == FCI_R64 && std::abs(v - Gv(q, p, r, s)) > tol)
                        return fci_fail(h, FCI_ERR_ARG, "real g2 lacks 8-fold symmetry at (%d,%d,%d,%d)", p, q, r, s);
                }
    int rc = set_dev(h);
    if (rc) return rc;
    free_strings(h);
    h->n_orb = n;
    h->dtype = dtype;
    h->e_core = e_core;
    h->h1.swap(hh);
    h->g2.swap(gg);
    return FCI_OK;
}

// G = 1/2 g', g'_pqrs = (pq|rs) + (h'_pq d_rs + d_pq h'_rs) / N_e, h' = h - 1/2 sum_r (pr|rq).
// Real: packed over unordered pairs (p>=q, r>=s), row-major [npair][npair].
// Complex: full [n^2][n^2], interleaved.
static int prepare_operator(fci_context *h, int n_el) {
    const int n = h->n_orb, w = h->dtype == FCI_C128 ? 2 : 1;
    const size_t n2 = (size_t)n * n;
    auto gidx = [&](int p, int q, int r, int s) { return (((size_t)p * n + q) * n + r) * n + s; };
    std::vector<std::complex<double>> hp(n2);
    for (int p = 0; p < n; ++p)
        for (int q = 0; q < n; ++q) {
            std::complex<double> v(h->h1[(p * n + q) * w], w == 2 ? h->h1[(p * n + q) * w + 1] : 0.0);
            for (int r = 0; r < n; ++r) {
                size_t i = gidx(p, r, r, q);
                v -= 0.5 * std::complex<double>(h->g2[i * w], w == 2 ? h->g2[i * w + 1] : 0.0);
            }
            hp[p * n + q] = v;
        }
    const double inv_ne = n_el > 0 ? 1.0 / n_el : 0.0;
    auto gp = [&](int p, int q, int r, int s) {
        size_t i = gidx(p, q, r, s);
        std::complex<double> v(h->g2[i * w], w == 2 ? h->g2[i * w + 1] : 0.0);
        if (n_el == 0) return std::complex<double>(0.0, 0.0);
        if (r == s) v += hp[p * n + q] * inv_ne;
        if (p == q) v += hp[r * n + s] * inv_ne;
        return 0.5 * v;
    };
    std::vector<double> G;
    if (h->dtype == FCI_R64) {
        const int np = n * (n + 1) / 2;
        h->npair = np;
        G.assign((size_t)np * np, 0.0);
        for (int p = 0; p < n; ++p)
            for (int q = 0; q <= p; ++q)
                for (int r = 0; r < n; ++r)
                    for (int s = 0; s <= r; ++s)
                        G[(size_t)pair_index(p, q) * np + pair_index(r, s)] = gp(p, q, r, s).real();
    } else {
        h->npair = (int)n2;
        G.assign(n2 * n2 * 2, 0.0);
        for (int p = 0; p < n; ++p)
            for (int q = 0; q < n; ++q)
                for (int r = 0; r < n; ++r)
                    for (int s = 0; s < n; ++s) {
                        auto v = gp(p, q, r, s);
                        size_t i = (size_t)(p * n + q) * n2 + (r * n + s);
                        G[2 * i] = v.real();
                        G[2 * i + 1] = v.imag();
                    }
    }
    int rc = fci_dev_alloc(h, (void **)&h->d_G, G.size() * 8);
    if (rc) return rc;
    FCI_CUDA(h, cudaMemcpy(h->d_G, G.data(), G.size() * 8, cudaMemcpyHostToDevice));
    // diagonal helpers (real parts; exact for Hermitian integrals)
    std::vector<double> hd(n), J(n2), K(n2);
    for (int p = 0; p < n; ++p) {
        hd[p] = h->h1[(p * n + p) * w];
        for (int q = 0; q < n; ++q) {
            J[p * n + q] = h->g2[gidx(p, p, q, q) * w];
            K[p * n + q] = h->g2[gidx(p, q, q, p) * w];
        }
    }
    rc = fci_dev_alloc(h, (void **)&h->d_hd, n * 8);
    if (!rc) rc = fci_dev_alloc(h, (void **)&h->d_J, n2 * 8);
    if (!rc) rc = fci_dev_alloc(h, (void **)&h->d_K, n2 * 8);
    if (rc) return rc;
    FCI_CUDA(h, cudaMemcpy(h->d_hd, hd.data(), n * 8, cudaMemcpyHostToDevice));
    FCI_CUDA(h, cudaMemcpy(h->d_J, J.data(), n2 * 8, cudaMemcpyHostToDevice));
    FCI_CUDA(h, cudaMemcpy(h->d_K, K.data(), n2 * 8, cudaMemcpyHostToDevice));
    return FCI_OK;
}

int fci_build_strings(fci_handle h, int n_alpha, int n_beta, fci_stream stream) {
    if (!h) return fci_fail(nullptr, FCI_ERR_ARG, "NULL handle");
    if (h->dtype < 0) return fci_fail(h, FCI_ERR_STATE, "fci_setup_integrals must come first");
    const int n = h->n_orb;
    const bool spinor = n_beta < 0;
    if (spinor && h->dtype != FCI_C128) return fci_fail(h, FCI_ERR_ARG, "spinor strings need C128 integrals");
    if (!spinor && h->dtype != FCI_R64) return fci_fail(h, FCI_ERR_ARG, "alpha/beta strings need R64 integrals");
    if (n_alpha < 0 || n_alpha > n || (!spinor && n_beta > n))
        return fci_fail(h, FCI_ERR_ARG, "electron counts (%d,%d) do not fit %d orbitals", n_alpha, n_beta, n);
    if (spinor && n > 32) return fci_fail(h, FCI_ERR_UNSUPPORTED, "spinor strings above 32 spinors are not built");
    cudaStream_t s = (cudaStream_t)stream;
    int rc = set_dev(h);
    if (rc) return rc;
    free_strings(h);
    const int64_t nsa = binom_host(n, n_alpha);
    const int64_t nsb = spinor ? 1 : binom_host(n, n_beta);
    if (nsa <= 0 || nsb <= 0 || nsa > (1ll << 31) || nsb > (1ll << 31))
        return fci_fail(h, FCI_ERR_UNSUPPORTED, "string count out of range");
    h->na = n_alpha;
    h->nb = spinor ? 0 : n_beta;
    h->nsa = nsa;
    h->nsb = nsb;
    h->ndet = nsa * nsb;
    h->nent_a = n_alpha * (n - n_alpha + 1);
    h->nent_b = spinor ? 0 : n_beta * (n - n_beta + 1);
    rc = prepare_operator(h, spinor ? n_alpha : n_alpha + n_beta);
    if (rc) { free_strings(h); return rc; }
    rc = fci_dev_alloc(h, (void **)&h->d_str_a, nsa * 8);
    if (!rc && !spinor) rc = fci_dev_alloc(h, (void **)&h->d_str_b, nsb * 8);
    if (rc) { free_strings(h); return rc; }
    FCI_CUDA(h, launch_strings_unrank(n, n_alpha, nsa, h->d_binom, h->d_str_a, s));
    if (!spinor) {
        FCI_CUDA(h, launch_strings_unrank(n, n_beta, nsb, h->d_binom, h->d_str_b, s));
        rc = fci_dev_alloc(h, (void **)&h->d_rep_a, (size_t)nsa * h->nent_a * 8);
        if (!rc) rc = fci_dev_alloc(h, (void **)&h->d_rep_b, (size_t)nsb * h->nent_b * 8);
        h->npair_pad = (h->npair + 15) / 16 * 16;
        if (!rc) rc = fci_dev_alloc(h, (void **)&h->d_pair_a, (size_t)nsa * h->npair_pad * 4);
        if (!rc) rc = fci_dev_alloc(h, (void **)&h->d_pair_b, (size_t)nsb * h->npair_pad * 4);
        if (!rc) rc = fci_dev_alloc(h, (void **)&h->d_dstr, (size_t)(nsa + nsb) * (n + 1) * 8);
        if (rc) { free_strings(h); return rc; }
        FCI_CUDA(h, launch_repl_table(n, n_alpha, nsa, h->d_str_a, h->d_binom, h->nent_a, 1, h->d_rep_a, h->d_pair_a, h->npair_pad, s));
        FCI_CUDA(h, launch_repl_table(n, n_beta, nsb, h->d_str_b, h->d_binom, h->nent_b, 1, h->d_rep_b, h->d_pair_b, h->npair_pad, s));
        h->mode = FCI_MODE_FCI;
    } else {
        // The list of every spinor string is kept only when it is small; the sigma kernels
        // regenerate entries from the string masks otherwise.
        if ((size_t)nsa * h->nent_a * 8 <= ((size_t)1 << 30)) {
            rc = fci_dev_alloc(h, (void **)&h->d_rep_a, (size_t)nsa * h->nent_a * 8);
            if (rc) { free_strings(h); return rc; }
            FCI_CUDA(h, launch_repl_table(n, n_alpha, nsa, h->d_str_a, h->d_binom, h->nent_a, 0, h->d_rep_a, nullptr, h->npair, s));
        }
        h->mode = FCI_MODE_SPINOR;
    }
    FCI_CUDA(h, cudaStreamSynchronize(s));
    return FCI_OK;
}

int das_build_categories(fci_handle h, int n_spaces, const int *orbs_per_space, const int *ref_alpha,
                         const int *ref_beta, int max_transfer, fci_stream stream) {
    if (!h) return fci_fail(nullptr, FCI_ERR_ARG, "NULL handle");
    if (h->mode != FCI_MODE_FCI && h->mode != FCI_MODE_DAS)
        return fci_fail(h, FCI_ERR_STATE, "DAS needs alpha/beta strings (fci_build_strings with n_beta >= 0)");
    if (!orbs_per_space || !ref_alpha || !ref_beta) return fci_fail(h, FCI_ERR_ARG, "NULL DAS argument");
    int rc = set_dev(h);
    if (rc) return rc;
    return das_build(h, n_spaces, orbs_per_space, ref_alpha, ref_beta, max_transfer, (cudaStream_t)stream);
}

int fci_diagonal(fci_handle h, double *diag, fci_stream stream) {
    if (!h || !diag) return fci_fail(h, FCI_ERR_ARG, "NULL argument");
    if (h->mode == FCI_MODE_NONE) return fci_fail(h, FCI_ERR_STATE, "no strings built");
    int rc = set_dev(h);
    if (rc) return rc;
    cudaStream_t s = (cudaStream_t)stream;
    if (h->das_active) FCI_CUDA(h, launch_diag_das(h, diag, s));
    else if (h->mode == FCI_MODE_SPINOR) FCI_CUDA(h, launch_diag_spinor(h, diag, s));
    else FCI_CUDA(h, launch_diag_fci(h, diag, s));
    return FCI_OK;
}

int fci_sigma_workspace_bytes(fci_handle h, int n_vec, int precision, int n_slices, size_t *bytes) {
    if (!h || !bytes) return fci_fail(h, FCI_ERR_ARG, "NULL argument");
    (void)n_vec;
    if (h->mode == FCI_MODE_NONE) return fci_fail(h, FCI_ERR_STATE, "no strings built");
    *bytes = sigma_ws_bytes(h, precision, n_slices);
    return FCI_OK;
}

int fci_sigma(fci_handle h, const void *C, void *sigma, int n_vec, int precision, int n_slices,
              void *ws, size_t ws_bytes, fci_stream stream) {
    if (!h) return fci_fail(nullptr, FCI_ERR_ARG, "NULL handle");
    if (h->mode == FCI_MODE_NONE) return fci_fail(h, FCI_ERR_STATE, "no strings built");
    if (!C || !sigma || n_vec < 0) return fci_fail(h, FCI_ERR_ARG, "bad C/sigma/n_vec");
    if (precision != FCI_PREC_FP64 && precision != FCI_PREC_OZ_BF16)
        return fci_fail(h, FCI_ERR_ARG, "unknown precision %d", precision);
    if (precision == FCI_PREC_OZ_BF16 && (n_slices < 2 || n_slices > 8))
        return fci_fail(h, FCI_ERR_ARG, "n_slices %d outside [2, 8]", n_slices);
    if (precision == FCI_PREC_OZ_BF16 && h->dtype != FCI_R64 && h->mode != FCI_MODE_SPINOR)
        return fci_fail(h, FCI_ERR_UNSUPPORTED, "split precision with complex integrals needs spinor strings");
    const size_t need = sigma_ws_bytes(h, precision, n_slices);
    if (ws_bytes < need || (need && !ws)) return fci_fail(h, FCI_ERR_ARG, "workspace %zu < %zu bytes", ws_bytes, need);
    if (((uintptr_t)ws & 255) != 0) return fci_fail(h, FCI_ERR_ARG, "workspace not 256-byte aligned");
    const int64_t nd = h->das_active ? h->das.n_det : h->ndet;
    const size_t esz = h->dtype == FCI_C128 ? 16 : 8;
    const char *c0 = (const char *)C, *s0 = (const char *)sigma;
    const size_t vb = (size_t)nd * esz * (size_t)n_vec;
    if (vb && c0 < s0 + vb && s0 < c0 + vb) return fci_fail(h, FCI_ERR_ARG, "C and sigma overlap");
    int rc = set_dev(h);
    if (rc) return rc;
    for (int v = 0; v < n_vec; ++v) {
        rc = sigma_dispatch(h, c0 + (size_t)v * nd * esz, (char *)sigma + (size_t)v * nd * esz, precision,
                            n_slices, ws, ws_bytes, (cudaStream_t)stream);
        if (rc) return rc;
    }
    return FCI_OK;
}

// Device bytes of n_vec vectors, rounded to the workspace alignment.
static size_t host_vec_bytes(const fci_context *h, int n_vec) {
    const int64_t nd = h->das_active ? h->das.n_det : h->ndet;
    const size_t esz = h->dtype == FCI_C128 ? 16 : 8;
    return ((size_t)nd * esz * (size_t)n_vec + 255) & ~(size_t)255;
}

int fci_sigma_host_workspace_bytes(fci_handle h, int n_vec, int precision, int n_slices, size_t *bytes) {
    if (!h || !bytes) return fci_fail(h, FCI_ERR_ARG, "NULL argument");
    if (h->mode == FCI_MODE_NONE) return fci_fail(h, FCI_ERR_STATE, "no strings built");
    if (n_vec < 0) return fci_fail(h, FCI_ERR_ARG, "bad n_vec");
    *bytes = 2 * host_vec_bytes(h, n_vec) + sigma_ws_bytes(h, precision, n_slices);
    return FCI_OK;
}

int fci_sigma_host(fci_handle h, const void *C_host, void *sigma_host, int n_vec, int precision, int n_slices,
                   void *ws, size_t ws_bytes, fci_stream stream) {
    if (!h) return fci_fail(nullptr, FCI_ERR_ARG, "NULL handle");
    if (h->mode == FCI_MODE_NONE) return fci_fail(h, FCI_ERR_STATE, "no strings built");
    if (!C_host || !sigma_host || n_vec < 0) return fci_fail(h, FCI_ERR_ARG, "bad C/sigma/n_vec");
    const size_t vb = host_vec_bytes(h, n_vec);
    const size_t need = 2 * vb + sigma_ws_bytes(h, precision, n_slices);
    if (!ws || ws_bytes < need) return fci_fail(h, FCI_ERR_ARG, "workspace %zu < %zu bytes", ws_bytes, need);
    if (((uintptr_t)ws & 255) != 0) return fci_fail(h, FCI_ERR_ARG, "workspace not 256-byte aligned");
    const int64_t nd = h->das_active ? h->das.n_det : h->ndet;
    const size_t bytes = (size_t)nd * (h->dtype == FCI_C128 ? 16 : 8) * (size_t)n_vec;
    const char *c0 = (const char *)C_host, *s0 = (const char *)sigma_host;
    if (bytes && c0 < s0 + bytes && s0 < c0 + bytes) return fci_fail(h, FCI_ERR_ARG, "C and sigma overlap");
    int rc = set_dev(h);
    if (rc) return rc;
    cudaStream_t s = (cudaStream_t)stream;
    char *Cd = (char *)ws, *Sd = Cd + vb;
    FCI_CUDA(h, cudaMemcpyAsync(Cd, C_host, bytes, cudaMemcpyHostToDevice, s));
    if ((rc = fci_sigma(h, Cd, Sd, n_vec, precision, n_slices, Sd + vb, ws_bytes - 2 * vb, stream))) {
        cudaStreamSynchronize(s);  // the copy in flight still reads C_host
        return rc;
    }
    FCI_CUDA(h, cudaMemcpyAsync(sigma_host, Sd, bytes, cudaMemcpyDeviceToHost, s));
    return fci_sync_status(h, stream);
}

void fci_davidson_default_opts(fci_davidson_opts *o) {
    if (!o) return;
    o->max_iter = 100;
    o->max_subspace = 32;
    o->tol_residual = 1e-6;
    o->tol_energy = 1e-10;
    o->eps = 0.0;
    o->precision = FCI_PREC_FP64;
    o->n_slices = 6;
    o->switch_residual = 1e-5;
    o->use_guess = 0;
    o->final_precision = FCI_PREC_FP64;
    o->final_slices = 0;
    o->staged_sigma = 0;
    o->gap_bound = 0;
    o->start_mix = 1e-2;
}

static int check_opts(fci_context *h, const fci_davidson_opts *o) {
    if (!o) return fci_fail(h, FCI_ERR_ARG, "NULL opts");
    if (o->max_iter < 1 || o->max_subspace < 2 || o->max_subspace > 32)
        return fci_fail(h, FCI_ERR_ARG, "max_iter >= 1 and max_subspace in [2, 32] required");
    if (!(o->tol_residual > 0) || !(o->tol_energy > 0) || !(o->eps == o->eps))
        return fci_fail(h, FCI_ERR_ARG, "tolerances must be positive, eps a number");
    if (!(o->start_mix >= 0.0 && o->start_mix <= 1.0))
        return fci_fail(h, FCI_ERR_ARG, "start_mix must lie in [0, 1]");
    if (o->precision != FCI_PREC_FP64 && o->precision != FCI_PREC_OZ_BF16)
        return fci_fail(h, FCI_ERR_ARG, "unknown precision %d", o->precision);
    if (o->precision == FCI_PREC_OZ_BF16 && (o->n_slices < 2 || o->n_slices > 8))
        return fci_fail(h, FCI_ERR_ARG, "n_slices %d outside [2, 8]", o->n_slices);
    if (o->final_precision != FCI_PREC_FP64 && o->final_precision != FCI_PREC_OZ_BF16)
        return fci_fail(h, FCI_ERR_ARG, "unknown final precision %d", o->final_precision);
    if (o->final_precision == FCI_PREC_OZ_BF16 && (o->final_slices < 6 || o->final_slices > 8))
        return fci_fail(h, FCI_ERR_ARG, "final_slices %d outside [6, 8]", o->final_slices);
    if (h->das_active) {  // the DAS split forms: 2 or 3 slices fused, 4 and more two-pass
        if (o->precision == FCI_PREC_OZ_BF16) {
            const int rc = das_split_check(h, o->n_slices);
            if (rc) return rc;
        }
        if (o->final_precision == FCI_PREC_OZ_BF16) {
            const int rc = das_split_check(h, o->final_slices);
            if (rc) return rc;
        }
    }
    return FCI_OK;
}

int fci_davidson_workspace_bytes(fci_handle h, const fci_davidson_opts *o, size_t *bytes) {
    if (!h || !bytes) return fci_fail(h, FCI_ERR_ARG, "NULL argument");
    int rc = check_opts(h, o);
    if (rc) return rc;
    if (h->mode == FCI_MODE_NONE) return fci_fail(h, FCI_ERR_STATE, "no strings built");
    *bytes = davidson_ws_bytes(h, o);
    return FCI_OK;
}

int davidson_solve(fci_handle h, const fci_davidson_opts *o, void *C_io, double *energy,
                   fci_davidson_log *log, void *ws, size_t ws_bytes, fci_stream stream) {
    if (!h) return fci_fail(nullptr, FCI_ERR_ARG, "NULL handle");
    int rc = check_opts(h, o);
    if (rc) return rc;
    if (h->mode == FCI_MODE_NONE) return fci_fail(h, FCI_ERR_STATE, "no strings built");
    if (!C_io || !energy) return fci_fail(h, FCI_ERR_ARG, "NULL C_io/energy");
    if ((o->precision == FCI_PREC_OZ_BF16 || o->final_precision == FCI_PREC_OZ_BF16) && h->dtype != FCI_R64 &&
        h->mode != FCI_MODE_SPINOR)
        return fci_fail(h, FCI_ERR_UNSUPPORTED, "split precision with complex integrals needs spinor strings");
    const size_t need = davidson_ws_bytes(h, o);
    if (ws_bytes < need || !ws) return fci_fail(h, FCI_ERR_ARG, "workspace %zu < %zu bytes", ws_bytes, need);
    if (((uintptr_t)ws & 255) != 0) return fci_fail(h, FCI_ERR_ARG, "workspace not 256-byte aligned");
    rc = set_dev(h);
    if (rc) return rc;
    return davidson_run(h, o, (double *)C_io, energy, log, ws, ws_bytes, (cudaStream_t)stream);
}

int fci_clear_graphs(fci_handle h) {
    if (!h) return fci_fail(nullptr, FCI_ERR_ARG, "NULL handle");
    cudaSetDevice(h->device);
    drop_graphs(h);
    return FCI_OK;
}

int fci_sigma_graph(fci_handle h, const void *C, void *sigma, int precision, int n_slices, void *ws, size_t ws_bytes,
                    fci_stream stream) {
    if (!h) return fci_fail(nullptr, FCI_ERR_ARG, "NULL handle");
    cudaStream_t s = (cudaStream_t)stream;
    for (auto &g : h->graphs) {
        if (g.C == C && g.sigma == sigma && g.precision == precision && g.n_slices == n_slices && g.ws == ws &&
            g.stream == s) {
            FCI_CUDA(h, cudaSetDevice(h->device));
            FCI_CUDA(h, cudaGraphLaunch(g.exec, s));
            return FCI_OK;
        }
    }
    // first call: a plain run (prepares integrals, kernel attributes), then the capture
    int rc = fci_sigma(h, C, sigma, 1, precision, n_slices, ws, ws_bytes, stream);
    if (rc) return rc;
    if (s == nullptr) return FCI_OK;  // the legacy default stream cannot be captured
    const bool timing = h->timing;
    h->timing = false;
    cudaGraph_t graph = nullptr;
    FCI_CUDA(h, cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
    rc = sigma_dispatch(h, C, sigma, precision, n_slices, ws, ws_bytes, s);
    cudaError_t e = cudaStreamEndCapture(s, &graph);
    h->timing = timing;
    if (rc) {
        if (graph) cudaGraphDestroy(graph);
        return rc;
    }
    if (e != cudaSuccess) return fci_cuda_check(h, e, "cudaStreamEndCapture");
    cudaGraphExec_t exec = nullptr;
    e = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) return fci_cuda_check(h, e, "cudaGraphInstantiate");
    if (h->graphs.size() >= 64) {
        cudaGraphExecDestroy(h->graphs.front().exec);
        h->graphs.erase(h->graphs.begin());
    }
    h->graphs.push_back({C, sigma, precision, n_slices, ws, s, exec});
    return FCI_OK;
}

int fci_tune_sigma(fci_handle h, int n_slices, const void *C, void *sigma, void *ws, size_t ws_bytes, int reps,
                   fci_stream stream, fci_tune_report *report) {
    if (!h) return fci_fail(nullptr, FCI_ERR_ARG, "NULL handle");
    if (h->mode == FCI_MODE_NONE) return fci_fail(h, FCI_ERR_STATE, "no strings built");
    if (h->mode == FCI_MODE_SPINOR || h->dtype != FCI_R64)
        return fci_fail(h, FCI_ERR_UNSUPPORTED, "split precision is built for real alpha/beta or DAS problems");
    if (!C || !sigma || reps < 1) return fci_fail(h, FCI_ERR_ARG, "bad C/sigma/reps");
    const size_t need = sigma_ws_bytes(h, FCI_PREC_OZ_BF16, n_slices);
    if (ws_bytes < need || !ws || ((uintptr_t)ws & 255)) return fci_fail(h, FCI_ERR_ARG, "workspace too small or misaligned");
    int rc = set_dev(h);
    if (rc) return rc;
    cudaStream_t s = (cudaStream_t)stream;
    int a[8] = {0}, b[8] = {0}, n = 0;
    if (h->das_active) {
        if (n_slices >= 4)
            return fci_fail(h, FCI_ERR_UNSUPPORTED, "the DAS two-pass split form (%d slices) has no tile choice", n_slices);
        if ((rc = dz_check(h, n_slices))) return rc;
        n = dz_tune_candidates(h, n_slices, a, b, 8);
    } else {
        if ((rc = oz_prepare_G(h, n_slices))) return rc;
        n = oz_tune_candidates(h, n_slices, a, b, 8);
    }
    if (n == 0) return fci_fail(h, FCI_ERR_UNSUPPORTED, "no kernel configuration fits %d slices", n_slices);
    drop_graphs(h);
    cudaEvent_t e0, e1;
    FCI_CUDA(h, cudaEventCreate(&e0));
    FCI_CUDA(h, cudaEventCreate(&e1));
    double ms[8];
    int best = 0;
    for (int i = 0; i < n; ++i) {
        if (h->das_active) dz_set_config(h, n_slices, a[i], b[i]);
        else oz_set_config(h, n_slices, a[i], b[i]);
        rc = sigma_dispatch(h, C, sigma, FCI_PREC_OZ_BF16, n_slices, ws, ws_bytes, s);  // untimed
        if (!rc) rc = fci_cuda_check(h, cudaEventRecord(e0, s), "event");
        for (int r = 0; r < reps && !rc; ++r) rc = sigma_dispatch(h, C, sigma, FCI_PREC_OZ_BF16, n_slices, ws, ws_bytes, s);
        if (!rc) rc = fci_cuda_check(h, cudaEventRecord(e1, s), "event");
        if (!rc) rc = fci_cuda_check(h, cudaEventSynchronize(e1), "sync");
        if (!rc) {
            int st = 0;
            rc = fci_cuda_check(h, cudaMemcpy(&st, h->d_status, sizeof(int), cudaMemcpyDeviceToHost), "status");
            if (!rc && st) {
                cudaMemset(h->d_status, 0, sizeof(int));
                rc = fci_fail(h, st, "split-precision kernel reported status %d while tuning", st);
            }
        }
        float t = 0.f;
        if (!rc) rc = fci_cuda_check(h, cudaEventElapsedTime(&t, e0, e1), "elapsed");
        if (rc) break;
        ms[i] = t / reps;
        if (ms[i] < ms[best]) best = i;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc) {  // leave the default configuration
        if (h->das_active) dz_set_config(h, n_slices, 0, 0);
        else oz_set_config(h, n_slices, 0, 0);
        return rc;
    }
    if (h->das_active) dz_set_config(h, n_slices, a[best], b[best]);
    else oz_set_config(h, n_slices, a[best], b[best]);
    if (report) {
        memset(report, 0, sizeof(*report));
        report->n_candidates = n;
        report->chosen = best;
        for (int i = 0; i < n; ++i) {
            report->param_a[i] = a[i];
            report->param_b[i] = b[i];
            report->ms[i] = ms[i];
        }
    }
    return FCI_OK;
}

int fci_sigma_grouped(const fci_sigma_job *jobs, int n_jobs, fci_stream stream) {
    if (!jobs || n_jobs < 0) return fci_fail(nullptr, FCI_ERR_ARG, "bad job list");
    if (n_jobs == 0) return FCI_OK;
    cudaStream_t s = (cudaStream_t)stream;
    // validate every job first
    for (int i = 0; i < n_jobs; ++i) {
        const fci_sigma_job &j = jobs[i];
        fci_context *h = j.handle;
        if (!h) return fci_fail(nullptr, FCI_ERR_ARG, "job %d has no handle", i);
        if (h->device != jobs[0].handle->device) return fci_fail(h, FCI_ERR_ARG, "jobs on different devices");
        for (int k = 0; k < i; ++k)
            if (jobs[k].handle == h) return fci_fail(h, FCI_ERR_ARG, "handle appears in jobs %d and %d", k, i);
        if (h->mode == FCI_MODE_NONE) return fci_fail(h, FCI_ERR_STATE, "job %d: no strings built", i);
        if (!j.C || !j.sigma) return fci_fail(h, FCI_ERR_ARG, "job %d: NULL vector", i);
        if (j.precision != FCI_PREC_FP64 && j.precision != FCI_PREC_OZ_BF16)
            return fci_fail(h, FCI_ERR_ARG, "job %d: unknown precision", i);
        if (j.precision == FCI_PREC_OZ_BF16 &&
            (j.n_slices < 2 || j.n_slices > 8 || (h->dtype != FCI_R64 && h->mode != FCI_MODE_SPINOR)))
            return fci_fail(h, FCI_ERR_ARG, "job %d: bad split-precision request", i);
        const size_t need = sigma_ws_bytes(h, j.precision, j.n_slices);
        if (j.workspace_bytes < need || !j.workspace || ((uintptr_t)j.workspace & 255))
            return fci_fail(h, FCI_ERR_ARG, "job %d: workspace too small or misaligned", i);
    }
    FCI_CUDA(jobs[0].handle, cudaSetDevice(jobs[0].handle->device));
    std::vector<char> done(n_jobs, 0);
    // split-precision FCI jobs, grouped by slice count: one contraction launch per group
    for (int i = 0; i < n_jobs; ++i) {
        const fci_sigma_job &j = jobs[i];
        if (done[i] || j.precision != FCI_PREC_OZ_BF16 || j.handle->mode != FCI_MODE_FCI || j.handle->das_active)
            continue;
        std::vector<fci_context *> hs;
        std::vector<const double *> Cs;
        std::vector<double *> ss;
        std::vector<void *> ws;
        for (int k = i; k < n_jobs; ++k) {
            const fci_sigma_job &q = jobs[k];
            if (done[k] || q.precision != FCI_PREC_OZ_BF16 || q.n_slices != j.n_slices ||
                q.handle->mode != FCI_MODE_FCI || q.handle->das_active)
                continue;
            hs.push_back(q.handle);
            Cs.push_back((const double *)q.C);
            ss.push_back((double *)q.sigma);
            ws.push_back(q.workspace);
            done[k] = 1;
        }
        int rc = oz_sigma_group(hs.data(), Cs.data(), ss.data(), ws.data(), (int)hs.size(), j.n_slices, s);
        if (rc) return rc;
    }
    // split-precision DAS jobs, grouped by slice count
    for (int i = 0; i < n_jobs; ++i) {
        const fci_sigma_job &j = jobs[i];
        if (done[i] || j.precision != FCI_PREC_OZ_BF16 || !j.handle->das_active || j.n_slices > 3) continue;
        std::vector<fci_context *> hs;
        std::vector<const double *> Cs;
        std::vector<double *> ss;
        std::vector<void *> ws;
        for (int k = i; k < n_jobs; ++k) {
            const fci_sigma_job &q = jobs[k];
            if (done[k] || q.precision != FCI_PREC_OZ_BF16 || q.n_slices != j.n_slices || !q.handle->das_active ||
                q.n_slices > 3)
                continue;
            hs.push_back(q.handle);
            Cs.push_back((const double *)q.C);
            ss.push_back((double *)q.sigma);
            ws.push_back(q.workspace);
            done[k] = 1;
        }
        int rc = dz_sigma_group(hs.data(), Cs.data(), ss.data(), ws.data(), (int)hs.size(), j.n_slices, s);
        if (rc) return rc;
    }
    for (int i = 0; i < n_jobs; ++i) {
        if (done[i]) continue;
        const fci_sigma_job &j = jobs[i];
        int rc = sigma_dispatch(j.handle, j.C, j.sigma, j.precision, j.n_slices, j.workspace, j.workspace_bytes, s);
        if (rc) return rc;
    }
    return FCI_OK;
}

int fci_clear_grouped_graphs(void) {
    std::lock_guard<std::mutex> lk(g_grouped_mu);
    for (auto &g : g_grouped_graphs) cudaGraphExecDestroy(g.exec);
    g_grouped_graphs.clear();
    return FCI_OK;
}

int fci_sigma_grouped_graph(const fci_sigma_job *jobs, int n_jobs, fci_stream stream) {
    if (!jobs || n_jobs <= 0) return fci_sigma_grouped(jobs, n_jobs, stream);
    cudaStream_t s = (cudaStream_t)stream;
    fci_context *h0 = jobs[0].handle;
    if (!h0) return fci_fail(nullptr, FCI_ERR_ARG, "job 0 has no handle");
    {
        std::lock_guard<std::mutex> lk(g_grouped_mu);
        for (auto &g : g_grouped_graphs)
            if (g.stream == s && g.device == h0->device && same_jobs(g.jobs, jobs, n_jobs)) {
                FCI_CUDA(h0, cudaSetDevice(h0->device));
                FCI_CUDA(h0, cudaGraphLaunch(g.exec, s));
                return FCI_OK;
            }
    }
    // first call with this list: a plain run (validates, prepares digit images and kernel
    // attributes), then the capture
    int rc = fci_sigma_grouped(jobs, n_jobs, stream);
    if (rc || s == nullptr) return rc;
    std::vector<char> timing(n_jobs);
    for (int i = 0; i < n_jobs; ++i) {
        timing[i] = jobs[i].handle->timing;
        jobs[i].handle->timing = false;
    }
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        rc = fci_sigma_grouped(jobs, n_jobs, stream);
        e = cudaStreamEndCapture(s, &graph);
    }
    for (int i = 0; i < n_jobs; ++i) jobs[i].handle->timing = timing[i];
    if (rc) {
        if (graph) cudaGraphDestroy(graph);
        return rc;
    }
    if (e != cudaSuccess) return fci_cuda_check(h0, e, "grouped sigma capture");
    cudaGraphExec_t exec = nullptr;
    e = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) return fci_cuda_check(h0, e, "cudaGraphInstantiate");
    std::lock_guard<std::mutex> lk(g_grouped_mu);
    if (g_grouped_graphs.size() >= 16) {
        cudaGraphExecDestroy(g_grouped_graphs.front().exec);
        g_grouped_graphs.erase(g_grouped_graphs.begin());
    }
    g_grouped_graphs.push_back({std::vector<fci_sigma_job>(jobs, jobs + n_jobs), s, h0->device, exec});
    return FCI_OK;
}

int davidson_begin(fci_handle h, const fci_davidson_opts *o, const void *C_guess, void *ws, size_t ws_bytes,
                   fci_stream stream, fci_davidson_handle *out) {
    if (!h || !out) return fci_fail(h, FCI_ERR_ARG, "NULL argument");
    *out = nullptr;
    int rc = check_opts(h, o);
    if (rc) return rc;
    if (h->mode == FCI_MODE_NONE) return fci_fail(h, FCI_ERR_STATE, "no strings built");
    if ((o->precision == FCI_PREC_OZ_BF16 || o->final_precision == FCI_PREC_OZ_BF16) && h->dtype != FCI_R64 &&
        h->mode != FCI_MODE_SPINOR)
        return fci_fail(h, FCI_ERR_UNSUPPORTED, "split precision with complex integrals needs spinor strings");
    const size_t need = davidson_ws_bytes(h, o);
    if (ws_bytes < need || !ws) return fci_fail(h, FCI_ERR_ARG, "workspace %zu < %zu bytes", ws_bytes, need);
    if (((uintptr_t)ws & 255) != 0) return fci_fail(h, FCI_ERR_ARG, "workspace not 256-byte aligned");
    rc = set_dev(h);
    if (rc) return rc;
    return davidson_state_begin(h, o, C_guess, ws, (cudaStream_t)stream, out);
}

int davidson_request(fci_davidson_handle st, const void **x, void **y, int *precision, int *n_slices, void **sws,
                     size_t *sws_bytes) {
    if (!st) return fci_fail(nullptr, FCI_ERR_ARG, "NULL Davidson state");
    davidson_state_request(st, x, y, precision, n_slices, sws, sws_bytes);
    return FCI_OK;
}

int davidson_advance(fci_davidson_handle st, int *done) {
    if (!st || !done) return fci_fail(nullptr, FCI_ERR_ARG, "NULL argument");
    fci_context *h = davidson_state_handle(st);
    int rc = set_dev(h);
    if (rc) return rc;
    return davidson_state_advance(st, done);
}

int davidson_finish(fci_davidson_handle st, void *C_out, double *energy, fci_davidson_log *log) {
    if (!st) return fci_fail(nullptr, FCI_ERR_ARG, "NULL Davidson state");
    fci_context *h = davidson_state_handle(st);
    set_dev(h);
    return davidson_state_finish(st, C_out, energy, log);
}

int fci_table_bytes(fci_handle h, int table, size_t *bytes) {
    if (!h || !bytes) return fci_fail(h, FCI_ERR_ARG, "NULL argument");
    *bytes = 0;
    switch (table) {
        case FCI_TABLE_STRINGS_ALPHA: *bytes = (size_t)h->nsa * 8; break;
        case FCI_TABLE_STRINGS_BETA: *bytes = h->mode == FCI_MODE_SPINOR ? 0 : (size_t)h->nsb * 8; break;
        case FCI_TABLE_REPL_ALPHA: *bytes = h->d_rep_a ? (size_t)h->nsa * h->nent_a * 16 : 0; break;
        case FCI_TABLE_REPL_BETA: *bytes = h->d_rep_b ? (size_t)h->nsb * h->nent_b * 16 : 0; break;
        case FCI_TABLE_DAS_CATEGORIES:
            *bytes = h->das_active ? (size_t)h->das.n_cat * (2 * h->das.n_spaces + 3) * 8 : 0; break;
        case FCI_TABLE_DAS_ADDRESS: *bytes = h->das_active ? (size_t)h->das.n_det * 8 : 0; break;
        default: return fci_fail(h, FCI_ERR_ARG, "unknown table %d", table);
    }
    return FCI_OK;
}

int fci_copy_table(fci_handle h, int table, void *dst, size_t bytes, fci_stream stream) {
    size_t need = 0;
    int rc = fci_table_bytes(h, table, &need);
    if (rc) return rc;
    if (need == 0) return fci_fail(h, FCI_ERR_STATE, "table %d does not exist in this layout", table);
    if (!dst || bytes < need) return fci_fail(h, FCI_ERR_ARG, "destination too small (%zu < %zu)", bytes, need);
    rc = set_dev(h);
    if (rc) return rc;
    cudaStream_t s = (cudaStream_t)stream;
    switch (table) {
        case FCI_TABLE_STRINGS_ALPHA: FCI_CUDA(h, cudaMemcpyAsync(dst, h->d_str_a, need, cudaMemcpyDeviceToDevice, s)); break;
        case FCI_TABLE_STRINGS_BETA: FCI_CUDA(h, cudaMemcpyAsync(dst, h->d_str_b, need, cudaMemcpyDeviceToDevice, s)); break;
        case FCI_TABLE_REPL_ALPHA: FCI_CUDA(h, launch_export_repl(h->nsa, h->nent_a, h->d_rep_a, (int32_t *)dst, s)); break;
        case FCI_TABLE_REPL_BETA: FCI_CUDA(h, launch_export_repl(h->nsb, h->nent_b, h->d_rep_b, (int32_t *)dst, s)); break;
        case FCI_TABLE_DAS_CATEGORIES: {
            const fci_das_layout &d = h->das;
            const int S = d.n_spaces;
            std::vector<int64_t> t((size_t)d.n_cat * (2 * S + 3));
            for (int c = 0; c < d.n_cat; ++c) {
                int64_t *r = &t[(size_t)c * (2 * S + 3)];
                for (int k = 0; k < S; ++k) {
                    r[k] = d.pat_a[d.cat_pa[c] * S + k];
                    r[S + k] = d.pat_b[d.cat_pb[c] * S + k];
                }
                r[2 * S] = d.pat_nstr_a[d.cat_pa[c]];
                r[2 * S + 1] = d.pat_nstr_b[d.cat_pb[c]];
                r[2 * S + 2] = d.cat_off[c];
            }
            FCI_CUDA(h, cudaMemcpyAsync(dst, t.data(), need, cudaMemcpyHostToDevice, s));
            FCI_CUDA(h, cudaStreamSynchronize(s));
            break;
        }
        case FCI_TABLE_DAS_ADDRESS: FCI_CUDA(h, launch_das_export_address(h, (int64_t *)dst, s)); break;
    }
    return FCI_OK;
}

}  // extern "C"

// ------------------------------------------------------------------ dispatch

size_t sigma_ws_bytes(const fci_context *h, int precision, int n_slices) {
    auto al = [](size_t b) { return (b + 255) & ~(size_t)255; };
    if (h->das_active) return das_workspace_bytes(h, precision, n_slices);
    if (precision == FCI_PREC_OZ_BF16 && h->mode == FCI_MODE_SPINOR) return cz_workspace_bytes(h, n_slices);
    if (precision == FCI_PREC_OZ_BF16) return oz_workspace_bytes(h, n_slices);
    const size_t esz = h->dtype == FCI_C128 ? 16 : 8;
    return 2 * al((size_t)h->npair * h->ndet * esz);
}

int sigma_dispatch(fci_context *h, const void *C, void *sigma, int precision, int n_slices, void *ws,
                   size_t ws_bytes, cudaStream_t s) {
    auto al = [](size_t b) { return (b + 255) & ~(size_t)255; };
    if (h->das_active) {
        return precision == FCI_PREC_FP64 ? das_sigma_fp64(h, (const double *)C, (double *)sigma, ws, ws_bytes, s)
                                          : das_sigma_oz(h, (const double *)C, (double *)sigma, n_slices, ws, ws_bytes, s);
    }
    if (precision == FCI_PREC_OZ_BF16 && h->mode == FCI_MODE_SPINOR)
        return cz_sigma(h, (const double *)C, (double *)sigma, n_slices, ws, ws_bytes, s);
    if (precision == FCI_PREC_OZ_BF16) return oz_sigma_fci(h, (const double *)C, (double *)sigma, n_slices, ws, ws_bytes, s);
    const size_t esz = h->dtype == FCI_C128 ? 16 : 8;
    double *D = (double *)ws;
    double *E = (double *)((char *)ws + al((size_t)h->npair * h->ndet * esz));
    const bool real = h->mode == FCI_MODE_FCI;
    {
        phase_scope ps(h, s, FCI_PHASE_GATHER, 1);
        FCI_CUDA(h, real ? launch_gather_fci_r64(h, (const double *)C, D, s)
                         : launch_gather_spinor(h, (const double *)C, D, s));
    }
    {
        phase_scope ps(h, s, FCI_PHASE_CONTRACT, 1);
        FCI_CUDA(h, real ? launch_dgemm(h->npair, h->ndet, h->npair, h->d_G, D, h->ndet, E, h->ndet, s)
                         : launch_zgemm(h->npair, h->ndet, h->npair, h->d_G, D, h->ndet, E, h->ndet, s));
    }
    {
        phase_scope ps(h, s, FCI_PHASE_SCATTER, 1);
        FCI_CUDA(h, real ? launch_scatter_fci_r64(h, E, (const double *)C, (double *)sigma, s)
                         : launch_scatter_spinor(h, E, (const double *)C, (double *)sigma, s));
    }
    return FCI_OK;
}
