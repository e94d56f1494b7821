// 2.5D CNN denoising agents (Sec. IV) and their training step (Sec. V).
// Placeholder entry points: the tcgen05 implementation lands in this file.
#include "common.cuh"

struct msf_cnn {
    int64_t max_pixels;
};

extern "C" size_t msf_cnn_param_count(void) {
    // W1 [64][5][3][3] + b1, W2..W9 [64][64][3][3] + b, W10 [1][64][3][3] + b10,
    // then gamma, beta, running mean, running var for layers 2..9
    return (size_t)64 * 5 * 9 + 64 + 8 * ((size_t)64 * 64 * 9 + 64) + 64 * 9 + 1 + 8 * 4 * 64;
}

extern "C" msf_status msf_cnn_create(int64_t, msf_cnn** out) {
    if (out) *out = nullptr;
    return msf::fail(MSF_ERR_UNSUPPORTED, "msf_cnn_create: not built yet");
}
extern "C" void msf_cnn_destroy(msf_cnn* c) { delete c; }
extern "C" msf_status msf_cnn_set_params(msf_cnn*, const float*, size_t) {
    return msf::fail(MSF_ERR_UNSUPPORTED, "msf_cnn_set_params: not built yet");
}
extern "C" msf_status msf_cnn_get_params(msf_cnn*, float*, size_t) {
    return msf::fail(MSF_ERR_UNSUPPORTED, "msf_cnn_get_params: not built yet");
}
extern "C" msf_status msf_denoise(msf_cnn*, msf_orient, const msf_vol*, const float*, float*, void*) {
    return msf::fail(MSF_ERR_UNSUPPORTED, "msf_denoise: not built yet");
}
extern "C" msf_status msf_train_step(msf_cnn*, const float*, const float*, int, int, int, float, float*, void*) {
    return msf::fail(MSF_ERR_UNSUPPORTED, "msf_train_step: not built yet");
}
