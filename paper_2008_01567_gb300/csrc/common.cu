// Error reporting, version, device check and measurement conditioning.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>

#include <mutex>
#include <string>
#include <vector>

#include "common.cuh"

namespace msf {

static thread_local char g_last_error[1024] = "";

msf_status fail(msf_status st, const char* fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_last_error, sizeof(g_last_error), fmt, ap);
    va_end(ap);
    return st;
}

msf_status check_device() {
    int dev = 0;
    MSF_TRY_CUDA(cudaGetDevice(&dev));
    int major = 0, minor = 0;
    MSF_TRY_CUDA(cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev));
    MSF_TRY_CUDA(cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev));
    if (major != 10 || minor != 3)
        return fail(MSF_ERR_UNSUPPORTED, "libmsf is built for sm_103a only; device %d is sm_%d%d",
                    dev, major, minor);
    return MSF_OK;
}

// y = -ln(max(n,1)/I0) and Lambda = c exp(-y): Sec. II, the weight matrix
// Lambda_n = diag{c exp(-y_n)} of the Gaussian approximation to Poisson noise.
__global__ void weights_kernel(const float* __restrict__ counts, float* __restrict__ y,
                               float* __restrict__ lam, size_t m, float log_i0, float c) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < m;
         i += (size_t)gridDim.x * blockDim.x) {
        float n = fmaxf(counts[i], 1.0f);
        float yi = log_i0 - logf(n);
        if (y) y[i] = yi;
        if (lam) lam[i] = c * expf(-yi);
    }
}

// ------------------------------------------------------------------ profiler

struct ProfRecord {
    int name;
    cudaEvent_t a, b;
};

static std::mutex g_prof_mu;
static bool g_prof_on = false;
static std::vector<const char*> g_prof_names;
static std::vector<int64_t> g_prof_count;
static std::vector<double> g_prof_ms;
static std::vector<ProfRecord> g_prof_pending;
static std::vector<cudaEvent_t> g_prof_pool;

static cudaEvent_t prof_event() {
    if (!g_prof_pool.empty()) {
        cudaEvent_t e = g_prof_pool.back();
        g_prof_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

static void prof_drain() {   // caller holds g_prof_mu
    for (ProfRecord& r : g_prof_pending) {
        float ms = 0.0f;
        cudaEventSynchronize(r.b);
        if (cudaEventElapsedTime(&ms, r.a, r.b) == cudaSuccess) {
            g_prof_ms[r.name] += ms;
            g_prof_count[r.name] += 1;
        }
        g_prof_pool.push_back(r.a);
        g_prof_pool.push_back(r.b);
    }
    g_prof_pending.clear();
}

ProfScope::ProfScope(const char* name, cudaStream_t stream) : stream_(stream) {
    if (!g_prof_on) return;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(stream, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) return;
    std::lock_guard<std::mutex> lk(g_prof_mu);
    int id = -1;
    for (size_t i = 0; i < g_prof_names.size(); ++i)
        if (g_prof_names[i] == name || std::string(g_prof_names[i]) == name) id = (int)i;
    if (id < 0) {
        id = (int)g_prof_names.size();
        g_prof_names.push_back(name);
        g_prof_count.push_back(0);
        g_prof_ms.push_back(0.0);
    }
    ProfRecord r{id, prof_event(), prof_event()};
    cudaEventRecord(r.a, stream_);
    g_prof_pending.push_back(r);
    slot_ = (int)g_prof_pending.size() - 1;
}

ProfScope::~ProfScope() {
    if (slot_ < 0) return;
    std::lock_guard<std::mutex> lk(g_prof_mu);
    cudaEventRecord(g_prof_pending[slot_].b, stream_);
    if (g_prof_pending.size() > 4096) prof_drain();
}

}  // namespace msf

extern "C" void msf_profile_enable(int on) { msf::g_prof_on = on != 0; }

extern "C" void msf_profile_reset(void) {
    std::lock_guard<std::mutex> lk(msf::g_prof_mu);
    msf::prof_drain();
    for (size_t i = 0; i < msf::g_prof_names.size(); ++i) {
        msf::g_prof_count[i] = 0;
        msf::g_prof_ms[i] = 0.0;
    }
}

extern "C" int msf_profile_read(int i, const char** name, int64_t* launches, double* total_ms) {
    std::lock_guard<std::mutex> lk(msf::g_prof_mu);
    msf::prof_drain();
    const int n = (int)msf::g_prof_names.size();
    if (i >= 0 && i < n) {
        if (name) *name = msf::g_prof_names[i];
        if (launches) *launches = msf::g_prof_count[i];
        if (total_ms) *total_ms = msf::g_prof_ms[i];
    }
    return n;
}

extern "C" const char* msf_last_error(void) { return msf::g_last_error; }

extern "C" const char* msf_version(void) { return "msf-gb300 0.1 (sm_103a)"; }

extern "C" msf_status msf_weights(const float* d_counts, float* d_y, float* d_lambda, size_t m,
                                  double I0, double c, void* stream) {
    MSF_REQUIRE(d_counts != nullptr, "msf_weights: d_counts is NULL");
    MSF_REQUIRE(I0 > 0 && c > 0, "msf_weights: I0 and c must be positive");
    if (m == 0) return MSF_OK;
    int blocks = (int)((m + 255) / 256);
    if (blocks > 152 * 16) blocks = 152 * 16;
    MSF_PROF("weights", msf::as_stream(stream));
    msf::weights_kernel<<<blocks, 256, 0, msf::as_stream(stream)>>>(d_counts, d_y, d_lambda, m,
                                                                    (float)log(I0), (float)c);
    MSF_LAUNCH_CHECK();
    return MSF_OK;
}
