// npm_tc.cu -- tensor-core (tcgen05, BF16) path of the NPM forward pass.
#include "npm_handle.h"
#include "npm_kernels.h"

namespace npm {

struct TcState {
    int unused;
};

npm_status tc_create(npm_handle* h) {
    (void)h;
    return NPM_ERR_UNSUPPORTED;
}

void tc_destroy(npm_handle* h) {
    delete h->tc;
    h->tc = nullptr;
}

cudaError_t tc_refresh_weights(npm_handle* h, cudaStream_t st) {
    (void)h;
    (void)st;
    return cudaSuccess;
}

npm_status tc_query(npm_handle* h, int64_t n, int64_t ld, const float* pos, const float* aux,
                    const float* uin, float ufrac, bool sample, float* dir_out, float* pdf_out,
                    float* mix_out, cudaStream_t st) {
    (void)h, (void)n, (void)ld, (void)pos, (void)aux, (void)uin, (void)ufrac, (void)sample;
    (void)dir_out, (void)pdf_out, (void)mix_out, (void)st;
    return NPM_ERR_UNSUPPORTED;
}

}  // namespace npm
