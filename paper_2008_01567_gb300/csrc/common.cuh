// Shared internals of libmsf: error reporting, launch helpers, deterministic
// FP64 block reductions.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <stdio.h>

#include "msf.h"

namespace msf {

// Records a printf-style message as this thread's last error and returns `st`.
msf_status fail(msf_status st, const char* fmt, ...);

inline cudaStream_t as_stream(void* s) { return reinterpret_cast<cudaStream_t>(s); }

// Checks the device is usable for the kernels of this library (sm_103).
msf_status check_device();

// The volume a projector plan was built for, and its sinogram size (rays).
const msf_vol* projector_volume(const msf_projector* p);
size_t projector_sino_size(const msf_projector* p);
void projector_detector(const msf_projector* p, int* nu, int* nv);
// Advances whenever the plan's launch shapes change (autotune, set_tuning), so
// that a captured graph of launches with the old shapes is re-captured.
uint64_t projector_tuning_gen(const msf_projector* p);

// Device status word of a data-agent workspace: 0, or MSF_ERR_NUMERIC once a
// CG or ICD scalar was non-finite (sticky).
int* dataprox_status(msf_dataprox* d);

// CNN handle state used by the MACE orchestration: a counter that changes with
// the parameters, and the out-of-stream set-up done before a graph capture.
uint64_t cnn_generation(const msf_cnn* c);
msf_status cnn_prepare(msf_cnn* c, cudaStream_t st);

}  // namespace msf

#define MSF_TRY_CUDA(call)                                                                  \
    do {                                                                                    \
        cudaError_t e_ = (call);                                                            \
        if (e_ != cudaSuccess)                                                              \
            return msf::fail(MSF_ERR_CUDA, "%s:%d: %s: %s", __FILE__, __LINE__, #call,      \
                             cudaGetErrorString(e_));                                       \
    } while (0)

#define MSF_LAUNCH_CHECK()                                                                  \
    do {                                                                                    \
        cudaError_t e_ = cudaGetLastError();                                                \
        if (e_ != cudaSuccess)                                                              \
            return msf::fail(MSF_ERR_CUDA, "%s:%d: launch: %s", __FILE__, __LINE__,         \
                             cudaGetErrorString(e_));                                       \
    } while (0)

#define MSF_REQUIRE(cond, ...)                                                              \
    do {                                                                                    \
        if (!(cond)) return msf::fail(MSF_ERR_ARG, __VA_ARGS__);                            \
    } while (0)

#define MSF_TRY(expr)                                                                       \
    do {                                                                                    \
        msf_status s_ = (expr);                                                             \
        if (s_ != MSF_OK) return s_;                                                        \
    } while (0)

// Block-wide sum of a double; result valid in linear thread 0.  The block size
// must be a multiple of 32 and at most 1024.  The order of additions is fixed,
// so results are reproducible run to run.
__device__ __forceinline__ double block_sum_f64(double v) {
    __shared__ double warp_part[32];
    const int tid = threadIdx.x + blockDim.x * (threadIdx.y + blockDim.y * threadIdx.z);
    const int nwarps = (blockDim.x * blockDim.y * blockDim.z) >> 5;
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if ((tid & 31) == 0) warp_part[tid >> 5] = v;
    __syncthreads();
    double r = 0.0;
    if (tid < 32) {
        r = (tid < nwarps) ? warp_part[tid] : 0.0;
        for (int o = 16; o > 0; o >>= 1) r += __shfl_down_sync(0xffffffffu, r, o);
    }
    __syncthreads();
    return r;
}

namespace msf {

// RAII launch timer: when profiling is enabled, records an event pair on
// `stream` around the scope (one kernel launch) under `name`.
class ProfScope {
  public:
    ProfScope(const char* name, cudaStream_t stream);
    ~ProfScope();

  private:
    int slot_ = -1;
    cudaStream_t stream_;
};

}  // namespace msf

#define MSF_PROF(name, stream) msf::ProfScope msf_prof_scope_(name, stream)
