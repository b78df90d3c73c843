// STP-DAS layout and the categorical sigma build (Results: C = (+)_B C^B over
// categories; Methods: Eqs. sigmaL1e/sigmaL2e sum over target, intermediate and source
// categories linked by one-electron excitation lists).
//
// Layout.  The orbitals are split into S contiguous distributed active spaces.  A
// per-spin pattern is the tuple of electrons per space; its excess is the number of
// electrons above the reference occupation, summed over spaces.  Target categories are
// (alpha pattern, beta pattern) pairs with total excess <= T, intermediate categories
// those with excess T + 1: one single replacement moves at most one electron, so every
// determinant reached by E_rs from the target space lies in target + intermediate, and
// sigma_I = 1/2 sum g' <I|E_pq|K><K|E_rs|J> C_J with K over that union is exactly
// P H P.  Determinant addresses: categories in lexicographic (alpha, beta) pattern
// order, target categories first, each block row-major [alpha-local][beta-local];
// a local string index is mixed radix over spaces (space 0 most significant) of the
// rank of the space's sub-string.  Fermion signs come from the global strings, which
// reproduces the paper's global phase factors P_mu_nu by construction.
//
// Sigma (FP64).  The intermediate space is processed in chunks of whole categories
// that fit the workspace: gather D[pq, K] = sum_J <K|E_pq|J> C_J for the chunk (J in
// the target space, zero elsewhere: the categorical skip of empty blocks), E = G D on
// the FP64 path, then every target determinant adds the terms <I|E_pq|K> E[pq, K]
// whose K lies in the chunk.
#include <math.h>

#include <stdlib.h>

#include <algorithm>
#include <functional>
#include <map>
#include <vector>

#include "das_dev.cuh"

namespace {

using das_dev::DasDev;
using das_dev::das_addr;
using das_dev::das_strings;
using das_dev::find_cat;
using das_dev::make_dev;

__global__ void __launch_bounds__(256) k_das_gather(DasDev d, int n_cat_int, int64_t a0, int64_t len,
                                                    const int32_t *__restrict__ pairA,
                                                    const int32_t *__restrict__ pairB,
                                                    const double *__restrict__ C, double *__restrict__ D) {
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < len; k += (int64_t)gridDim.x * blockDim.x) {
        int32_t A, B;
        int pb;
        das_strings(d, n_cat_int, a0 + k, A, B, pb);
        for (int pp = 0; pp < d.npair; ++pp) {
            double v = 0.0;
            const int32_t ea = __ldg(pairA + (int64_t)pp * d.nsa + A);
            if (ea >= 0) {
                const int64_t j = das_addr(d, ea >> 1, B);
                if (j >= 0 && j < d.n_det) {
                    const double c = __ldg(C + j);
                    v = (ea & 1) ? -c : c;
                }
            }
            const int32_t eb = __ldg(pairB + (int64_t)pp * d.nsb + B);
            if (eb >= 0) {
                const int64_t j = das_addr(d, A, eb >> 1);
                if (j >= 0 && j < d.n_det) {
                    const double c = __ldg(C + j);
                    v += (eb & 1) ? -c : c;
                }
            }
            D[(int64_t)pp * len + k] = v;
        }
    }
}

__global__ void __launch_bounds__(256) k_das_scatter(DasDev d, int64_t a0, int64_t len,
                                                     const int32_t *__restrict__ pairA,
                                                     const int32_t *__restrict__ pairB,
                                                     const double *__restrict__ E, const double *__restrict__ C,
                                                     double e_core, int first, double *__restrict__ sigma) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < d.n_det; i += (int64_t)gridDim.x * blockDim.x) {
        int32_t A, B;
        int pb;
        das_strings(d, d.n_cat, i, A, B, pb);
        double acc = 0.0;
        for (int pp = 0; pp < d.npair; ++pp) {
            const double *Ep = E + (int64_t)pp * len;
            const int32_t ea = __ldg(pairA + (int64_t)pp * d.nsa + A);
            if (ea >= 0) {
                const int64_t k = das_addr(d, ea >> 1, B) - a0;
                if (k >= 0 && k < len) {
                    const double e = __ldg(Ep + k);
                    acc += (ea & 1) ? -e : e;
                }
            }
            const int32_t eb = __ldg(pairB + (int64_t)pp * d.nsb + B);
            if (eb >= 0) {
                const int64_t k = das_addr(d, A, eb >> 1) - a0;
                if (k >= 0 && k < len) {
                    const double e = __ldg(Ep + k);
                    acc += (eb & 1) ? -e : e;
                }
            }
        }
        sigma[i] = first ? fma(e_core, C[i], acc) : sigma[i] + acc;  // one rounding for the e_core term
    }
}

__global__ void k_das_diag(DasDev d, int n, int64_t nsa, const uint64_t *__restrict__ sa,
                           const uint64_t *__restrict__ sb, const double *__restrict__ tab, double e_core,
                           double *__restrict__ diag) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < d.n_det; i += (int64_t)gridDim.x * blockDim.x) {
        int32_t Ai, Bi;
        int pb;
        das_strings(d, d.n_cat, i, Ai, Bi, pb);
        diag[i] = diag_from_strings(sa[Ai], sb[Bi], tab + (int64_t)Ai * (n + 1), tab + (nsa + Bi) * (n + 1), e_core);
    }
}

__global__ void k_das_address(DasDev d, int64_t *__restrict__ out) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < d.n_det; i += (int64_t)gridDim.x * blockDim.x) {
        int32_t A, B;
        int pb;
        das_strings(d, d.n_cat, i, A, B, pb);
        out[i] = (int64_t)A * d.nsb + B;
    }
}

unsigned grid_for(int64_t n) { return (unsigned)std::max<int64_t>(1, std::min<int64_t>(ceil_div(n, 256), 152 * 16)); }

inline size_t al(size_t b) { return (b + 255) & ~(size_t)255; }

int64_t binom64(int n, int k) {
    if (k < 0 || k > n) return 0;
    int64_t r = 1;
    for (int i = 1; i <= k; ++i) r = r * (n - k + i) / i;
    return r;
}

// All patterns (n_0..n_{S-1}), 0 <= n_s <= m_s, sum = ne, lexicographic.
void gen_patterns(const std::vector<int> &m, int ne, std::vector<std::vector<int>> &out) {
    const int S = (int)m.size();
    std::vector<int> cur(S, 0);
    std::function<void(int, int)> rec = [&](int s, int left) {
        if (s == S) {
            if (left == 0) out.push_back(cur);
            return;
        }
        for (int k = 0; k <= m[s]; ++k) {
            cur[s] = k;
            rec(s + 1, left - k);
        }
    };
    rec(0, ne);
}

}  // namespace

void das_free(fci_context *h) {
    fci_das_layout &L = h->das;
    void *ptrs[] = {L.d_cat_of_pair, L.d_loc_a, L.d_pat_of_a, L.d_loc_b, L.d_pat_of_b, L.d_pat_nstr_b,
                    L.d_cat_pa, L.d_cat_pb, L.d_cat_off, L.d_str_of_loc_a, L.d_str_of_loc_b,
                    L.d_pat_locbase_a, L.d_pat_locbase_b};
    for (void *p : ptrs) fci_dev_free(p);
    dz_free(L);
    L = fci_das_layout();
    h->das_active = false;
    if (h->mode == FCI_MODE_DAS) h->mode = FCI_MODE_FCI;
}

int das_build(fci_context *h, int S, const int *orbs, const int *ref_a, const int *ref_b, int T, cudaStream_t st) {
    if (S < 1 || S > 8) return fci_fail(h, FCI_ERR_ARG, "n_spaces %d outside [1, 8]", S);
    if (T < 0) return fci_fail(h, FCI_ERR_ARG, "max_transfer must be >= 0");
    int tot = 0, ra = 0, rb = 0;
    for (int s = 0; s < S; ++s) {
        if (orbs[s] < 1) return fci_fail(h, FCI_ERR_ARG, "space %d has no orbitals", s);
        if (ref_a[s] < 0 || ref_a[s] > orbs[s] || ref_b[s] < 0 || ref_b[s] > orbs[s])
            return fci_fail(h, FCI_ERR_ARG, "reference occupation of space %d out of range", s);
        tot += orbs[s];
        ra += ref_a[s];
        rb += ref_b[s];
    }
    if (tot != h->n_orb) return fci_fail(h, FCI_ERR_ARG, "spaces hold %d orbitals, the problem has %d", tot, h->n_orb);
    if (ra != h->na || rb != h->nb)
        return fci_fail(h, FCI_ERR_ARG, "reference occupation holds (%d,%d) electrons, strings have (%d,%d)", ra, rb,
                        h->na, h->nb);
    das_free(h);
    fci_das_layout &L = h->das;
    L.n_spaces = S;
    std::vector<int> m(orbs, orbs + S);
    int off = 0;
    for (int s = 0; s < S; ++s) {
        L.space_orbs[s] = orbs[s];
        L.space_off[s] = off;
        off += orbs[s];
        L.ref_a[s] = ref_a[s];
        L.ref_b[s] = ref_b[s];
    }
    L.max_transfer = T;
    // patterns with excess <= T + 1
    auto excess = [&](const std::vector<int> &p, const int *ref) {
        int e = 0;
        for (int s = 0; s < S; ++s) e += std::max(0, p[s] - ref[s]);
        return e;
    };
    std::vector<std::vector<int>> all_a, all_b, pa, pb;
    gen_patterns(m, h->na, all_a);
    gen_patterns(m, h->nb, all_b);
    for (auto &p : all_a) if (excess(p, ref_a) <= T + 1) pa.push_back(p);
    for (auto &p : all_b) if (excess(p, ref_b) <= T + 1) pb.push_back(p);
    L.n_pat_a = (int)pa.size();
    L.n_pat_b = (int)pb.size();
    auto nstr = [&](const std::vector<int> &p) {
        int64_t r = 1;
        for (int s = 0; s < S; ++s) r *= binom64(m[s], p[s]);
        return r;
    };
    for (auto &p : pa) {
        for (int s = 0; s < S; ++s) L.pat_a.push_back(p[s]);
        L.exc_a.push_back(excess(p, ref_a));
        L.pat_nstr_a.push_back(nstr(p));
    }
    for (auto &p : pb) {
        for (int s = 0; s < S; ++s) L.pat_b.push_back(p[s]);
        L.exc_b.push_back(excess(p, ref_b));
        L.pat_nstr_b.push_back(nstr(p));
    }
    // categories: target (excess <= T) then intermediate-only (excess == T + 1)
    std::vector<int32_t> cat_of((size_t)L.n_pat_a * L.n_pat_b, -1);
    for (int pass = 0; pass < 2; ++pass) {
        for (int a = 0; a < L.n_pat_a; ++a)
            for (int b = 0; b < L.n_pat_b; ++b) {
                const int e = L.exc_a[a] + L.exc_b[b];
                if ((pass == 0 && e <= T) || (pass == 1 && e == T + 1)) {
                    cat_of[(size_t)a * L.n_pat_b + b] = (int32_t)L.cat_pa.size();
                    L.cat_pa.push_back(a);
                    L.cat_pb.push_back(b);
                }
            }
        if (pass == 0) L.n_cat = (int)L.cat_pa.size();
    }
    L.n_cat_int = (int)L.cat_pa.size();
    if (L.n_cat == 0) return fci_fail(h, FCI_ERR_ARG, "no category within the transfer limit");
    int64_t o = 0;
    for (int c = 0; c < L.n_cat_int; ++c) {
        L.cat_off.push_back(o);
        o += L.pat_nstr_a[L.cat_pa[c]] * L.pat_nstr_b[L.cat_pb[c]];
    }
    L.cat_off.push_back(o);
    L.n_det_int = o;
    L.n_det = L.cat_off[L.n_cat];
    // per-string pattern and local index
    auto string_maps = [&](uint64_t *d_str, int64_t ns, const std::vector<std::vector<int>> &pats,
                           std::vector<int32_t> &pat_of, std::vector<int32_t> &loc_of, std::vector<int32_t> &str_of_loc,
                           std::vector<int64_t> &locbase) -> int {
        std::vector<uint64_t> strs(ns);
        if (cudaMemcpy(strs.data(), d_str, ns * 8, cudaMemcpyDeviceToHost) != cudaSuccess)
            return fci_cuda_check(h, cudaGetLastError(), "string download");
        std::map<std::vector<int>, int> pid;
        for (int i = 0; i < (int)pats.size(); ++i) pid[pats[i]] = i;
        locbase.assign(pats.size() + 1, 0);
        for (size_t i = 0; i < pats.size(); ++i) locbase[i + 1] = locbase[i] + nstr(pats[i]);
        str_of_loc.assign(locbase.back(), -1);
        pat_of.assign(ns, -1);
        loc_of.assign(ns, 0);
        std::vector<int> occ(S);
        for (int64_t i = 0; i < ns; ++i) {
            const uint64_t x = strs[i];
            int64_t loc = 0;
            for (int s = 0; s < S; ++s) {
                const uint64_t sub = (x >> L.space_off[s]) & ((((uint64_t)1) << m[s]) - 1);
                occ[s] = __builtin_popcountll(sub);
                // combinadic rank of the sub-string inside its space
                int64_t r = 0;
                int j = 1;
                for (int q = 0; q < m[s]; ++q)
                    if ((sub >> q) & 1) r += binom64(q, j++);
                loc = loc * binom64(m[s], occ[s]) + r;
            }
            auto it = pid.find(occ);
            if (it == pid.end()) continue;
            pat_of[i] = it->second;
            loc_of[i] = (int32_t)loc;
            str_of_loc[locbase[it->second] + loc] = (int32_t)i;
        }
        return FCI_OK;
    };
    std::vector<int32_t> pat_of_a, loc_a, sol_a, pat_of_b, loc_b, sol_b;
    std::vector<int64_t> lb_a, lb_b;
    int rc = string_maps(h->d_str_a, h->nsa, pa, pat_of_a, loc_a, sol_a, lb_a);
    if (!rc) rc = string_maps(h->d_str_b, h->nsb, pb, pat_of_b, loc_b, sol_b, lb_b);
    if (rc) { das_free(h); return rc; }
    auto up = [&](void **dst, const void *src, size_t bytes) -> int {
        int r = fci_dev_alloc(h, dst, bytes);
        if (r) return r;
        FCI_CUDA(h, cudaMemcpy(*dst, src, bytes, cudaMemcpyHostToDevice));
        return FCI_OK;
    };
    std::vector<int32_t> cpa(L.cat_pa.begin(), L.cat_pa.end()), cpb(L.cat_pb.begin(), L.cat_pb.end());
    rc = up((void **)&L.d_cat_of_pair, cat_of.data(), cat_of.size() * 4);
    if (!rc) rc = up((void **)&L.d_pat_of_a, pat_of_a.data(), pat_of_a.size() * 4);
    if (!rc) rc = up((void **)&L.d_loc_a, loc_a.data(), loc_a.size() * 4);
    if (!rc) rc = up((void **)&L.d_pat_of_b, pat_of_b.data(), pat_of_b.size() * 4);
    if (!rc) rc = up((void **)&L.d_loc_b, loc_b.data(), loc_b.size() * 4);
    if (!rc) rc = up((void **)&L.d_pat_nstr_b, L.pat_nstr_b.data(), L.pat_nstr_b.size() * 8);
    if (!rc) rc = up((void **)&L.d_cat_pa, cpa.data(), cpa.size() * 4);
    if (!rc) rc = up((void **)&L.d_cat_pb, cpb.data(), cpb.size() * 4);
    if (!rc) rc = up((void **)&L.d_cat_off, L.cat_off.data(), L.cat_off.size() * 8);
    if (!rc) rc = up((void **)&L.d_str_of_loc_a, sol_a.data(), std::max<size_t>(1, sol_a.size()) * 4);
    if (!rc) rc = up((void **)&L.d_str_of_loc_b, sol_b.data(), std::max<size_t>(1, sol_b.size()) * 4);
    if (!rc) rc = up((void **)&L.d_pat_locbase_a, lb_a.data(), lb_a.size() * 8);
    if (!rc) rc = up((void **)&L.d_pat_locbase_b, lb_b.data(), lb_b.size() * 8);
    if (rc) { das_free(h); return rc; }
    (void)st;
    h->das_active = true;
    h->mode = FCI_MODE_DAS;
    return FCI_OK;
}

// Chunk of the intermediate space processed per pass: whole categories, D and E both
// resident; at most 16 GiB of workspace so very large spaces run in several passes.
// FCI_DAS_FP64_CHUNK_DETS=n lowers the cap to n determinants (never below the largest
// category), so that small problems can run the several-pass form too.
static int64_t das_chunk_len(const fci_context *h) {
    const int64_t cap_bytes = (int64_t)16 << 30;
    const int64_t per_det = 2 * 8 * (int64_t)h->npair;
    const fci_das_layout &L = h->das;
    int64_t maxcat = 0;
    for (int c = 0; c < L.n_cat_int; ++c) maxcat = std::max(maxcat, L.cat_off[c + 1] - L.cat_off[c]);
    int64_t cap = std::min(L.n_det_int, cap_bytes / per_det);
    if (const char *env = getenv("FCI_DAS_FP64_CHUNK_DETS")) {
        const long long v = atoll(env);
        if (v > 0) cap = std::min<int64_t>(cap, v);
    }
    return std::max(maxcat, cap);
}

size_t das_workspace_bytes(const fci_context *h, int precision, int n_slices) {
    if (precision == FCI_PREC_OZ_BF16) return dz_workspace_bytes(h, n_slices);
    const int64_t len = das_chunk_len(h);
    return 2 * al((size_t)h->npair * len * 8);
}

int das_sigma_fp64(fci_context *h, const double *C, double *sigma, void *ws, size_t ws_bytes, cudaStream_t s) {
    (void)ws_bytes;
    const fci_das_layout &L = h->das;
    const DasDev d = make_dev(h);
    const int64_t cap = das_chunk_len(h);
    double *D = (double *)ws;
    double *E = (double *)((char *)ws + al((size_t)h->npair * cap * 8));
    int c0 = 0;
    bool first = true;
    while (c0 < L.n_cat_int) {
        int c1 = c0;
        while (c1 < L.n_cat_int && L.cat_off[c1 + 1] - L.cat_off[c0] <= cap) ++c1;
        const int64_t a0 = L.cat_off[c0], len = L.cat_off[c1] - a0;
        {
            phase_scope ps(h, s, FCI_PHASE_GATHER, 1);
            k_das_gather<<<grid_for(len), 256, 0, s>>>(d, L.n_cat_int, a0, len, h->d_pair_a, h->d_pair_b, C, D);
            FCI_CUDA(h, cudaGetLastError());
        }
        {
            phase_scope ps(h, s, FCI_PHASE_CONTRACT, 1);
            FCI_CUDA(h, launch_dgemm(h->npair, len, h->npair, h->d_G, D, len, E, len, s));
        }
        {
            phase_scope ps(h, s, FCI_PHASE_SCATTER, 1);
            k_das_scatter<<<grid_for(L.n_det), 256, 0, s>>>(d, a0, len, h->d_pair_a, h->d_pair_b, E, C, h->e_core,
                                                           first ? 1 : 0, sigma);
            FCI_CUDA(h, cudaGetLastError());
        }
        first = false;
        c0 = c1;
    }
    return FCI_OK;
}

int das_sigma_oz(fci_context *h, const double *C, double *sigma, int n_slices, void *ws, size_t ws_bytes,
                 cudaStream_t s) {
    return dz_sigma(h, C, sigma, n_slices, ws, ws_bytes, s);
}

cudaError_t launch_diag_das(const fci_context *h, double *diag, cudaStream_t s) {
    cudaError_t e = launch_diag_strings(h, s);
    if (e != cudaSuccess) return e;
    k_das_diag<<<grid_for(h->das.n_det), 256, 0, s>>>(make_dev(h), h->n_orb, h->nsa, h->d_str_a, h->d_str_b,
                                                      h->d_dstr, h->e_core, diag);
    return cudaGetLastError();
}

cudaError_t launch_das_export_address(const fci_context *h, int64_t *dst, cudaStream_t s) {
    k_das_address<<<grid_for(h->das.n_det), 256, 0, s>>>(make_dev(h), dst);
    return cudaGetLastError();
}
