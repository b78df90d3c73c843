// Split-precision (Ozaki) contraction on tcgen05 tensor cores (filled in below).
#include "fci_internal.h"

int oz_prepare_G(fci_context *h, int) { return fci_fail(h, FCI_ERR_UNSUPPORTED, "split precision not built yet"); }
size_t oz_workspace_bytes(const fci_context *, int) { return 0; }
int oz_sigma_fci(fci_context *h, const double *, double *, int, void *, size_t, cudaStream_t) {
    return fci_fail(h, FCI_ERR_UNSUPPORTED, "split precision not built yet");
}
