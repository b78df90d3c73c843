// STP-DAS categories and the categorical sigma build (filled in below).
#include "fci_internal.h"

int das_build(fci_context *h, int, const int *, const int *, const int *, int, cudaStream_t) {
    return fci_fail(h, FCI_ERR_UNSUPPORTED, "DAS layout not built yet");
}
void das_free(fci_context *h) { h->das_active = false; }
int das_sigma_fp64(fci_context *h, const double *, double *, void *, size_t, cudaStream_t) {
    return fci_fail(h, FCI_ERR_UNSUPPORTED, "DAS sigma not built yet");
}
int das_sigma_oz(fci_context *h, const double *, double *, int, void *, size_t, cudaStream_t) {
    return fci_fail(h, FCI_ERR_UNSUPPORTED, "DAS sigma not built yet");
}
size_t das_workspace_bytes(const fci_context *, int, int) { return 0; }
cudaError_t launch_diag_das(const fci_context *, double *, cudaStream_t) { return cudaErrorNotSupported; }
cudaError_t launch_das_export_address(const fci_context *, int64_t *, cudaStream_t) { return cudaErrorNotSupported; }
