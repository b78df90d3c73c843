// Device-side view of an STP-DAS layout (categories, per-string pattern and local
// index) and the address arithmetic shared by the FP64 and split-precision kernels.
#pragma once

#include "fci_internal.h"

namespace das_dev {

struct DasDev {
    int S;
    int64_t nsa, nsb;
    int npair;
    int n_pat_b;
    const int32_t *pat_of_a, *loc_of_a, *pat_of_b, *loc_of_b;
    const int32_t *cat_of;      // [n_pat_a * n_pat_b] -> category or -1
    const int64_t *cat_off;     // [n_cat_int + 1]
    const int32_t *cat_pa, *cat_pb;
    const int64_t *nstr_b;      // [n_pat_b]
    const int32_t *str_of_loc_a, *str_of_loc_b;
    const int64_t *locbase_a, *locbase_b;
    int n_cat;                  // target categories
    int64_t n_det;
};

__device__ __forceinline__ int find_cat(const int64_t *__restrict__ off, int n, int64_t addr) {
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (off[mid] <= addr) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// Address of the determinant (alpha string A, beta string B) in the intermediate
// space, or -1 if it is outside target + intermediate.
__device__ __forceinline__ int64_t das_addr(const DasDev &d, int32_t A, int32_t B) {
    const int pa = d.pat_of_a[A], pb = d.pat_of_b[B];
    if (pa < 0 || pb < 0) return -1;
    const int c = d.cat_of[pa * d.n_pat_b + pb];
    if (c < 0) return -1;
    return d.cat_off[c] + (int64_t)d.loc_of_a[A] * d.nstr_b[pb] + d.loc_of_b[B];
}

__device__ __forceinline__ void das_strings(const DasDev &d, int n_cat_range, int64_t addr, int32_t &A, int32_t &B,
                                            int &pb) {
    const int c = find_cat(d.cat_off, n_cat_range, addr);
    const int pa = d.cat_pa[c];
    pb = d.cat_pb[c];
    const int64_t r = addr - d.cat_off[c], nb = d.nstr_b[pb];
    const int64_t la = r / nb, lb = r - la * nb;
    A = d.str_of_loc_a[d.locbase_a[pa] + la];
    B = d.str_of_loc_b[d.locbase_b[pb] + lb];
}


inline DasDev make_dev(const fci_context *h) {

    const fci_das_layout &L = h->das;
    DasDev d;
    d.S = L.n_spaces;
    d.nsa = h->nsa;
    d.nsb = h->nsb;
    d.npair = h->npair;
    d.n_pat_b = L.n_pat_b;
    d.pat_of_a = L.d_pat_of_a;
    d.loc_of_a = L.d_loc_a;
    d.pat_of_b = L.d_pat_of_b;
    d.loc_of_b = L.d_loc_b;
    d.cat_of = L.d_cat_of_pair;
    d.cat_off = L.d_cat_off;
    d.cat_pa = L.d_cat_pa;
    d.cat_pb = L.d_cat_pb;
    d.nstr_b = L.d_pat_nstr_b;
    d.str_of_loc_a = L.d_str_of_loc_a;
    d.str_of_loc_b = L.d_str_of_loc_b;
    d.locbase_a = L.d_pat_locbase_a;
    d.locbase_b = L.d_pat_locbase_b;
    d.n_cat = L.n_cat;
    d.n_det = L.n_det;
    return d;
}


}  // namespace das_dev
