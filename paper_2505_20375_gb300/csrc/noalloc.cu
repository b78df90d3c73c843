// fci_sigma_noalloc: the FP64 sigma build with its scratch in a fixed device array.
//
// fci_sigma needs D and E intermediates (2 x n_pair x n_det elements) in a workspace
// the caller allocates.  Some callers cannot allocate device memory when they need a
// sigma vector: a process whose framework has already reserved the whole device
// memory pool for its own caching allocator, code running where CUDA allocation calls
// are not allowed (for example inside a host callback enqueued on a stream), or a
// latency-critical loop that must not risk the implicit device synchronisation that
// cudaMalloc and cudaFree can cause.  This entry point serves them: it uses a
// file-scope device array of FCI_NOALLOC_SCRATCH_BYTES instead of a workspace and calls
// no allocating routine.
//
// The array is a __device__ variable: every GPU that loads libfci holds it until the
// process exits.  In host code its name is only a host-side stand-in, so the device
// address is looked up once per device with cudaGetSymbolAddress (with that device
// current) and passed to the kernels.
#include <mutex>

#include "fci_internal.h"

namespace {

constexpr size_t FCI_NOALLOC_SCRATCH_BYTES = (size_t)64 << 20;  // 64 MiB
constexpr int FCI_NOALLOC_MAX_DEVICES = 64;

static __device__ __align__(256) unsigned char g_fci_noalloc_scratch[FCI_NOALLOC_SCRATCH_BYTES];

std::mutex g_noalloc_mu;
void *g_noalloc_ptr[FCI_NOALLOC_MAX_DEVICES] = {nullptr};

inline size_t al(size_t b) { return (b + 255) & ~(size_t)255; }

}  // namespace

extern "C" int fci_sigma_noalloc(fci_handle h, const void *C, void *sigma, fci_stream stream) {
    if (!h) return fci_fail(nullptr, FCI_ERR_ARG, "NULL handle");
    if (h->mode != FCI_MODE_FCI && h->mode != FCI_MODE_SPINOR)
        return fci_fail(h, FCI_ERR_UNSUPPORTED, "fci_sigma_noalloc covers FCI and spinor layouts (build strings first)");
    if (!C || !sigma) return fci_fail(h, FCI_ERR_ARG, "NULL C or sigma");
    const size_t esz = h->dtype == FCI_C128 ? 16 : 8;
    const size_t half = al((size_t)h->npair * h->ndet * esz);
    const size_t need = 2 * half;
    if (need > FCI_NOALLOC_SCRATCH_BYTES)
        return fci_fail(h, FCI_ERR_ARG,
                        "fci_sigma_noalloc needs %zu bytes of scratch (2 x n_pair x n_det elements), above its "
                        "static maximum of %zu bytes; use fci_sigma with a caller workspace",
                        need, FCI_NOALLOC_SCRATCH_BYTES);
    const char *c0 = (const char *)C, *s0 = (const char *)sigma;
    const size_t vb = (size_t)h->ndet * esz;
    if (c0 < s0 + vb && s0 < c0 + vb) return fci_fail(h, FCI_ERR_ARG, "C and sigma overlap");
    FCI_CUDA(h, cudaSetDevice(h->device));
    if (h->device < 0 || h->device >= FCI_NOALLOC_MAX_DEVICES)
        return fci_fail(h, FCI_ERR_UNSUPPORTED, "device index %d above %d", h->device, FCI_NOALLOC_MAX_DEVICES);
    void *scratch = nullptr;
    {
        // One-time set-up per device, with that device current (made current above).
        std::lock_guard<std::mutex> lock(g_noalloc_mu);
        if (!g_noalloc_ptr[h->device]) {
            void *p = nullptr;
            cudaError_t e = cudaGetSymbolAddress(&p, g_fci_noalloc_scratch);
            if (e != cudaSuccess || !p) {
                cudaGetLastError();
                return fci_fail(h, FCI_ERR_CUDA, "cudaGetSymbolAddress of the static scratch failed: %s",
                                cudaGetErrorString(e));
            }
            g_noalloc_ptr[h->device] = p;
        }
        scratch = g_noalloc_ptr[h->device];
    }
    // D and E are written in full by the gather and the contraction before they are
    // read, so the shared array needs no clearing between calls.
    double *D = (double *)scratch;
    double *E = (double *)((char *)scratch + half);
    cudaStream_t s = (cudaStream_t)stream;
    if (h->mode == FCI_MODE_FCI) {
        FCI_CUDA(h, launch_gather_fci_r64(h, (const double *)C, D, s));
        FCI_CUDA(h, launch_dgemm(h->npair, h->ndet, h->npair, h->d_G, D, h->ndet, E, h->ndet, s));
        FCI_CUDA(h, launch_scatter_fci_r64(h, E, (const double *)C, (double *)sigma, s));
    } else {
        FCI_CUDA(h, launch_gather_spinor(h, (const double *)C, D, s));
        FCI_CUDA(h, launch_zgemm(h->npair, h->ndet, h->npair, h->d_G, D, h->ndet, E, h->ndet, s));
        FCI_CUDA(h, launch_scatter_spinor(h, E, (const double *)C, (double *)sigma, s));
    }
    return FCI_OK;
}
