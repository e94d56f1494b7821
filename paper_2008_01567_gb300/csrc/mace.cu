// MACE consensus and the partial-update Mann iteration (Sec. III, Algorithm 1).
//
//   X <- F~(W; X)           (data agent L~ by warm-started CG or grouped ICD, prior agents H_k)
//   Z <- G(2X - W)          (Eqs. (8)-(9): weighted average, replicated)
//   W <- W + 2 rho (Z - X)
//
// The consensus update is one pass over the K+1 stacked states that also forms
// the FP64 partial sums of the consensus spread of X.  With the q-GGMRF prior
// the data agent and the prior agent run concurrently on two forked streams.
// One iteration can be captured once into a CUDA graph and replayed; a batch of
// independent problems runs on forked streams inside one captured graph.
#include <math.h>
#include <string.h>

#include <vector>

#include "common.cuh"

struct msf_mace {
    msf_mace_desc desc;
    msf_dataprox* dp = nullptr;
    double* d_partial = nullptr;   // [2][nblocks]
    double* d_sums = nullptr;      // [2]
    double* h_sums = nullptr;      // pinned [2], written by the step's last copy
    int* h_status = nullptr;       // pinned copy of the data agent's numeric status word
    float* d_meas = nullptr;       // msf_mace_set_counts: counts, y, Lambda (3 sinograms)
    int nblocks = 0;
    size_t N = 0;                  // voxels of one 4D volume
    // with the q-GGMRF prior the data agent and the prior agent run on two
    // streams forked from the caller's and joined before the consensus
    cudaStream_t s_prox = nullptr, s_prior = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_prox = nullptr, ev_prior = nullptr;
    // graph replay of one iteration
    cudaStream_t cap = nullptr;
    cudaGraphExec_t gexec = nullptr;
    msf_mace_params gprm;
    uint64_t gcnn = 0;
    uint64_t gtune = 0;            // projector launch shapes the graph was captured with
};

struct msf_mace_batch {
    std::vector<msf_mace*> items;
    std::vector<cudaStream_t> streams;
    std::vector<cudaEvent_t> done;
    cudaEvent_t fork = nullptr;
    cudaStream_t cap = nullptr;
    cudaGraphExec_t gexec = nullptr;
    std::vector<msf_mace_params> gprm;
    std::vector<uint64_t> gcnn, gtune;
    // every problem runs the three CNN agents with the same parameters: the
    // agents of all problems then run as multi-problem persistent launches
    bool shared = false;
    std::vector<uint64_t> shared_gen;   // CNN generations the flag was decided for
};

namespace msf {

struct MaceCoef {
    float mu[4];
    float two_rho;
    int K1;
};

// W_i += 2 rho (sum_j mu_j (2 X_j - W_j) - X_i) for every agent i, and the
// partial sums of sum_i mu_i (X_i - Xbar)^2 and Xbar^2 with Xbar = sum_i mu_i X_i.
// Each thread takes four consecutive voxels per step (float4 traffic; N a
// multiple of 4 and 16-byte aligned stacks, which the caller checks, else
// VEC = false); the per-voxel
// terms are FP32 and each step's sum of four is added to FP64 thread sums,
// so this HBM-bound pass does a few FP64 adds per four voxels.
template <int K1, bool VEC>
__global__ void __launch_bounds__(256) consensus_kernel(float* __restrict__ W, const float* __restrict__ X,
                                                         size_t N, MaceCoef c, double* __restrict__ partial) {
    double num = 0.0, den = 0.0;
    const size_t stride = (size_t)gridDim.x * blockDim.x;
    auto voxel = [&](const float (&x)[K1], float (&w)[K1], float& dev, float& xb2) {
        float zbar = 0.0f, xbar = 0.0f;
#pragma unroll
        for (int k = 0; k < K1; ++k) {
            zbar += c.mu[k] * (2.0f * x[k] - w[k]);
            xbar += c.mu[k] * x[k];
        }
        dev = 0.0f;
#pragma unroll
        for (int k = 0; k < K1; ++k) {
            w[k] = w[k] + c.two_rho * (zbar - x[k]);
            const float dxk = x[k] - xbar;
            dev = fmaf(c.mu[k] * dxk, dxk, dev);
        }
        xb2 = xbar * xbar;
    };
    if (VEC) {
        const size_t N4 = N / 4;
        const float4* X4 = reinterpret_cast<const float4*>(X);
        float4* W4 = reinterpret_cast<float4*>(W);
        for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < N4; i += stride) {
            float4 xv[K1], wv[K1];
#pragma unroll
            for (int k = 0; k < K1; ++k) {
                xv[k] = X4[(size_t)k * N4 + i];
                wv[k] = W4[(size_t)k * N4 + i];
            }
            float dsum = 0.0f, bsum = 0.0f;
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                float x[K1], w[K1], dev, xb2;
#pragma unroll
                for (int k = 0; k < K1; ++k) {
                    x[k] = reinterpret_cast<const float*>(&xv[k])[e];
                    w[k] = reinterpret_cast<const float*>(&wv[k])[e];
                }
                voxel(x, w, dev, xb2);
#pragma unroll
                for (int k = 0; k < K1; ++k) reinterpret_cast<float*>(&wv[k])[e] = w[k];
                dsum += dev;
                bsum += xb2;
            }
#pragma unroll
            for (int k = 0; k < K1; ++k) W4[(size_t)k * N4 + i] = wv[k];
            num += (double)dsum;
            den += (double)bsum;
        }
    } else {
        for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < N; i += stride) {
            float x[K1], w[K1], dev, xb2;
#pragma unroll
            for (int k = 0; k < K1; ++k) {
                x[k] = X[(size_t)k * N + i];
                w[k] = W[(size_t)k * N + i];
            }
            voxel(x, w, dev, xb2);
#pragma unroll
            for (int k = 0; k < K1; ++k) W[(size_t)k * N + i] = w[k];
            num += (double)dev;
            den += (double)xb2;
        }
    }
    const double sn = block_sum_f64(num);
    const double sd = block_sum_f64(den);
    if (threadIdx.x == 0) {
        partial[blockIdx.x] = sn;
        partial[gridDim.x + blockIdx.x] = sd;
    }
}

__global__ void sum2_kernel(const double* __restrict__ partial, int n, double* __restrict__ out) {
    double a = 0.0, b = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        a += partial[i];
        b += partial[n + i];
    }
    a = block_sum_f64(a);
    b = block_sum_f64(b);
    if (threadIdx.x == 0) {
        out[0] = a;
        out[1] = b;
    }
}

constexpr int CONSENSUS_BLOCKS = 152 * 8;
static_assert(MSF_CONSENSUS_SUMS == 2 * CONSENSUS_BLOCKS && MSF_CONSENSUS_WORK == MSF_CONSENSUS_SUMS + 2,
              "msf_mace_consensus workspace layout");

// The consensus pass over K1 stacked states of N voxels each, then the two
// FP64 sums (into sums[0..1]) of the per-block partials.
static msf_status launch_consensus(float* W, const float* X, int K1, size_t N, const MaceCoef& c, double* partial,
                                   double* sums, cudaStream_t st) {
    {
        MSF_PROF("mace_consensus", st);
        const bool vec = N % 4 == 0 && (uintptr_t)W % 16 == 0 && (uintptr_t)X % 16 == 0;
        if (K1 == 2 && vec)
            consensus_kernel<2, true><<<CONSENSUS_BLOCKS, 256, 0, st>>>(W, X, N, c, partial);
        else if (K1 == 2)
            consensus_kernel<2, false><<<CONSENSUS_BLOCKS, 256, 0, st>>>(W, X, N, c, partial);
        else if (vec)
            consensus_kernel<4, true><<<CONSENSUS_BLOCKS, 256, 0, st>>>(W, X, N, c, partial);
        else
            consensus_kernel<4, false><<<CONSENSUS_BLOCKS, 256, 0, st>>>(W, X, N, c, partial);
        MSF_LAUNCH_CHECK();
    }
    {
        MSF_PROF("mace_residual", st);
        sum2_kernel<<<1, 1024, 0, st>>>(partial, CONSENSUS_BLOCKS, sums);
        MSF_LAUNCH_CHECK();
    }
    return MSF_OK;
}

static msf_status check_params(const msf_mace* m, const msf_mace_params* prm) {
    MSF_REQUIRE(prm->rho > 0 && prm->rho < 1, "msf_mace_step: rho must lie in (0,1) (Eq. (12))");
    MSF_REQUIRE(prm->sigma > 0, "msf_mace_step: sigma must be positive");
    const int K1 = m->desc.K + 1;
    double musum = 0.0;
    for (int i = 0; i < K1; ++i) {
        MSF_REQUIRE(prm->mu[i] >= 0, "msf_mace_step: agent weights must be non-negative");
        musum += prm->mu[i];
    }
    MSF_REQUIRE(fabs(musum - 1.0) < 1e-9, "msf_mace_step: agent weights must sum to 1 (got %.17g)", musum);
    MSF_REQUIRE(prm->n_cg >= 0 && prm->n_sweeps >= 0 && prm->n_icd >= 0,
                "msf_mace_step: iteration counts must be >= 0");
    return MSF_OK;
}

static msf_status enqueue_data(msf_mace* m, const msf_mace_params* prm, void* sp) {
    const msf_mace_desc& d = m->desc;
    if (prm->n_icd > 0) return msf_prox_data_icd(m->dp, d.d_y, d.d_lambda, d.d_W, d.d_X, prm->sigma, prm->n_icd, sp);
    return msf_prox_data(m->dp, d.d_y, d.d_lambda, d.d_W, d.d_X, prm->sigma, prm->n_cg, sp);
}

static msf_status enqueue_consensus(msf_mace* m, const msf_mace_params* prm, cudaStream_t st) {
    const msf_mace_desc& d = m->desc;
    const int K1 = d.K + 1;
    MaceCoef c;
    for (int i = 0; i < 4; ++i) c.mu[i] = i < K1 ? (float)prm->mu[i] : 0.0f;
    c.two_rho = (float)(2.0 * prm->rho);
    c.K1 = K1;
    MSF_TRY(launch_consensus(d.d_W, d.d_X, K1, m->N, c, m->d_partial, m->d_sums, st));
    MSF_TRY_CUDA(cudaMemcpyAsync(m->h_sums, m->d_sums, 2 * sizeof(double), cudaMemcpyDeviceToHost, st));
    MSF_TRY_CUDA(cudaMemcpyAsync(m->h_status, dataprox_status(m->dp), sizeof(int), cudaMemcpyDeviceToHost, st));
    return MSF_OK;
}

// Enqueues one whole iteration on st, ending with the copy of the two FP64
// residual sums into the handle's pinned buffer.
static msf_status enqueue_step(msf_mace* m, const msf_mace_params* prm, cudaStream_t st) {
    const msf_mace_desc& d = m->desc;
    const size_t N = m->N;
    const int K1 = d.K + 1;
    const msf_vol* vol = projector_volume(d.proj);
    // The agents of F~ read disjoint blocks of W and write disjoint blocks of X.
    // With the q-GGMRF prior the data agent runs on a low-priority stream beside
    // the prior agent on a high-priority one, both joined before the consensus.
    // The CNN agents stay in stream order: beside the data agent's projector
    // kernels the persistent tcgen05 convs lose about a third of their speed
    // (they share the L1 / shared-memory pipe and HBM), a net loss.
    const bool fork = d.prior == MSF_PRIOR_QGGMRF;
    if (fork) {
        MSF_TRY_CUDA(cudaEventRecord(m->ev_fork, st));
        MSF_TRY_CUDA(cudaStreamWaitEvent(m->s_prox, m->ev_fork, 0));
        MSF_TRY_CUDA(cudaStreamWaitEvent(m->s_prior, m->ev_fork, 0));
    }
    void* sp = reinterpret_cast<void*>(fork ? m->s_prox : st);
    void* sa = reinterpret_cast<void*>(fork ? m->s_prior : st);
    // X_0 <- L~(W_0; X_0): n_cg CG iterations, or n_icd grouped-ICD sweeps
    MSF_TRY(enqueue_data(m, prm, sp));
    // X_k <- H_k(W_k)
    for (int k = 1; k < K1; ++k) {
        if (d.prior == MSF_PRIOR_QGGMRF) {
            MSF_TRY(msf_prox_qggmrf(vol, &d.mrf, d.d_W + k * N, d.d_X + k * N, prm->sigma, prm->n_sweeps, sa));
        } else {
            const msf_orient o = d.K == 1 ? d.orient : (msf_orient)(k - 1);
            MSF_TRY(msf_denoise(d.cnn, o, vol, d.d_W + k * N, d.d_X + k * N, sa));
        }
    }
    if (fork) {
        MSF_TRY_CUDA(cudaEventRecord(m->ev_prox, m->s_prox));
        MSF_TRY_CUDA(cudaEventRecord(m->ev_prior, m->s_prior));
        MSF_TRY_CUDA(cudaStreamWaitEvent(st, m->ev_prox, 0));
        MSF_TRY_CUDA(cudaStreamWaitEvent(st, m->ev_prior, 0));
    }
    // Z <- G(2X - W);  W <- W + 2 rho (Z - X)
    (void)N;
    return enqueue_consensus(m, prm, st);
}

static msf_status read_residual(const msf_mace* m, double* h_residual) {
    if (*m->h_status != 0)
        return fail(MSF_ERR_NUMERIC, "msf_mace_step: non-finite CG or ICD scalar in the data agent");
    const double num = m->h_sums[0], den = m->h_sums[1];
    if (!isfinite(num) || !isfinite(den)) return fail(MSF_ERR_NUMERIC, "msf_mace_step: non-finite consensus residual");
    *h_residual = den > 0 ? sqrt(num / den) : sqrt(num);
    return MSF_OK;
}

static bool same_params(const msf_mace_params& a, const msf_mace_params& b) {
    return a.rho == b.rho && a.sigma == b.sigma && memcmp(a.mu, b.mu, sizeof(a.mu)) == 0 && a.n_cg == b.n_cg &&
           a.n_sweeps == b.n_sweeps && a.n_icd == b.n_icd;
}

static void drop_graph(cudaGraphExec_t& g) {
    if (g) cudaGraphExecDestroy(g);
    g = nullptr;
}

// Captures `body` (enqueueing on the capture stream) into an executable graph.
template <typename F>
static msf_status capture(cudaStream_t cap, cudaGraphExec_t* out, F&& body) {
    MSF_TRY_CUDA(cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal));
    msf_status st = body();
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamEndCapture(cap, &g);
    if (st != MSF_OK) {
        if (g) cudaGraphDestroy(g);
        return st;
    }
    if (e != cudaSuccess) return fail(MSF_ERR_CUDA, "graph capture failed: %s", cudaGetErrorString(e));
    e = cudaGraphInstantiate(out, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return fail(MSF_ERR_CUDA, "graph instantiation failed: %s", cudaGetErrorString(e));
    return MSF_OK;
}

// Shared-CNN batch: the data agents on the problem streams (forked, joined),
// then each orientation's CNN agents of all problems as multi-problem
// persistent launches (msf_denoise_batch), then the consensus of every problem.
static msf_status enqueue_batch_shared(msf_mace_batch* b, const msf_mace_params* prm, cudaStream_t st) {
    const int n = (int)b->items.size();
    MSF_TRY_CUDA(cudaEventRecord(b->fork, st));
    for (int i = 0; i < n; ++i) {
        MSF_TRY_CUDA(cudaStreamWaitEvent(b->streams[i], b->fork, 0));
        MSF_TRY(enqueue_data(b->items[i], &prm[i], reinterpret_cast<void*>(b->streams[i])));
        MSF_TRY_CUDA(cudaEventRecord(b->done[i], b->streams[i]));
        MSF_TRY_CUDA(cudaStreamWaitEvent(st, b->done[i], 0));
    }
    std::vector<msf_cnn*> cnns(n);
    std::vector<msf_vol> vols(n);
    std::vector<const float*> in(n);
    std::vector<float*> out(n);
    for (int k = 1; k <= 3; ++k) {
        for (int i = 0; i < n; ++i) {
            msf_mace* m = b->items[i];
            cnns[i] = m->desc.cnn;
            vols[i] = *projector_volume(m->desc.proj);
            in[i] = m->desc.d_W + k * m->N;
            out[i] = m->desc.d_X + k * m->N;
        }
        MSF_TRY(msf_denoise_batch(cnns.data(), n, (msf_orient)(k - 1), vols.data(), in.data(), out.data(),
                                  reinterpret_cast<void*>(st)));
    }
    for (int i = 0; i < n; ++i) MSF_TRY(enqueue_consensus(b->items[i], &prm[i], st));
    return MSF_OK;
}

// Decides (outside any stream capture) whether the batch's CNN agents can share
// launches: every problem runs the three CNN agents and every handle holds the
// same parameters (compared on the host whenever a generation changed).
static msf_status decide_shared(msf_mace_batch* b) {
    const int n = (int)b->items.size();
    std::vector<uint64_t> gens(n);
    bool all_cnn = n <= 16;
    for (int i = 0; i < n; ++i) {
        const msf_mace_desc& d = b->items[i]->desc;
        all_cnn = all_cnn && d.prior == MSF_PRIOR_CNN && d.K == 3;
        gens[i] = cnn_generation(d.cnn);
    }
    if (!all_cnn) {
        b->shared = false;
        return MSF_OK;
    }
    if (gens == b->shared_gen) return MSF_OK;
    const size_t np = msf_cnn_param_count();
    std::vector<float> p0(np), pi(np);
    MSF_TRY(msf_cnn_get_params(b->items[0]->desc.cnn, p0.data(), np));
    bool same = true;
    for (int i = 1; i < n && same; ++i) {
        MSF_TRY(msf_cnn_get_params(b->items[i]->desc.cnn, pi.data(), np));
        same = memcmp(p0.data(), pi.data(), np * sizeof(float)) == 0;
    }
    b->shared = same;
    b->shared_gen = gens;
    return MSF_OK;
}

// Fork: every problem stream waits for `st`; each enqueues its iteration; join.
static msf_status enqueue_batch(msf_mace_batch* b, const msf_mace_params* prm, cudaStream_t st) {
    if (b->shared) return enqueue_batch_shared(b, prm, st);
    const int n = (int)b->items.size();
    MSF_TRY_CUDA(cudaEventRecord(b->fork, st));
    for (int i = 0; i < n; ++i) {
        MSF_TRY_CUDA(cudaStreamWaitEvent(b->streams[i], b->fork, 0));
        MSF_TRY(enqueue_step(b->items[i], &prm[i], b->streams[i]));
        MSF_TRY_CUDA(cudaEventRecord(b->done[i], b->streams[i]));
        MSF_TRY_CUDA(cudaStreamWaitEvent(st, b->done[i], 0));
    }
    return MSF_OK;
}

}  // namespace msf

using namespace msf;

// The two agent streams (the prior agent at the highest priority, the data
// agent at the lowest) and the fork/join events.
static bool make_agent_streams(msf_mace* m) {
    int least = 0, greatest = 0;
    if (cudaDeviceGetStreamPriorityRange(&least, &greatest) != cudaSuccess) return false;
    return cudaStreamCreateWithPriority(&m->s_prior, cudaStreamNonBlocking, greatest) == cudaSuccess &&
           cudaStreamCreateWithPriority(&m->s_prox, cudaStreamNonBlocking, least) == cudaSuccess &&
           cudaEventCreateWithFlags(&m->ev_fork, cudaEventDisableTiming) == cudaSuccess &&
           cudaEventCreateWithFlags(&m->ev_prox, cudaEventDisableTiming) == cudaSuccess &&
           cudaEventCreateWithFlags(&m->ev_prior, cudaEventDisableTiming) == cudaSuccess;
}

extern "C" msf_status msf_mace_create(const msf_mace_desc* desc, msf_mace** out) {
    MSF_REQUIRE(desc && out, "msf_mace_create: NULL argument");
    *out = nullptr;
    MSF_REQUIRE(desc->proj && desc->d_W && desc->d_X && desc->d_y && desc->d_lambda,
                "msf_mace_create: projector, W, X, y and lambda are required");
    if (desc->prior == MSF_PRIOR_CNN) {
        MSF_REQUIRE((desc->K == 3 || desc->K == 1) && desc->cnn,
                    "msf_mace_create: the CNN prior needs K = 3 (or K = 1) and a cnn handle");
        MSF_REQUIRE(desc->K == 3 || (desc->orient >= MSF_XY_T && desc->orient <= MSF_ZX_T),
                    "msf_mace_create: bad orientation %d for the single CNN agent", (int)desc->orient);
    } else if (desc->prior == MSF_PRIOR_QGGMRF) {
        MSF_REQUIRE(desc->K == 1, "msf_mace_create: the q-GGMRF prior uses K = 1");
        MSF_REQUIRE(desc->mrf.p == 2.0 && desc->mrf.q >= 1.0 && desc->mrf.q <= 2.0 && desc->mrf.T > 0 &&
                        desc->mrf.sigma_x > 0 && desc->mrf.b_temporal >= 0,
                    "msf_mace_create: invalid q-GGMRF parameters");
    } else {
        return fail(MSF_ERR_ARG, "msf_mace_create: unknown prior kind %d", (int)desc->prior);
    }
    msf_mace* m = new msf_mace();
    m->desc = *desc;
    msf_status st = msf_dataprox_create(desc->proj, &m->dp);
    if (st != MSF_OK) {
        delete m;
        return st;
    }
    // the projector's volume describes the problem
    const msf_vol* v = projector_volume(desc->proj);
    m->N = (size_t)v->nx * v->ny * v->nz * v->nt;
    m->nblocks = CONSENSUS_BLOCKS;
    if (cudaMalloc(&m->d_partial, 2 * m->nblocks * sizeof(double)) != cudaSuccess ||
        cudaMalloc(&m->d_sums, 2 * sizeof(double)) != cudaSuccess ||
        cudaMallocHost(&m->h_sums, 2 * sizeof(double)) != cudaSuccess ||
        cudaMallocHost(&m->h_status, sizeof(int)) != cudaSuccess ||
        cudaStreamCreateWithFlags(&m->cap, cudaStreamNonBlocking) != cudaSuccess ||
        !make_agent_streams(m)) {
        cudaGetLastError();
        msf_mace_destroy(m);
        return fail(MSF_ERR_NOMEM, "msf_mace_create: out of memory");
    }
    *out = m;
    return MSF_OK;
}

extern "C" void msf_mace_destroy(msf_mace* m) {
    if (!m) return;
    drop_graph(m->gexec);
    if (m->cap) cudaStreamDestroy(m->cap);
    if (m->s_prox) cudaStreamDestroy(m->s_prox);
    if (m->s_prior) cudaStreamDestroy(m->s_prior);
    if (m->ev_fork) cudaEventDestroy(m->ev_fork);
    if (m->ev_prox) cudaEventDestroy(m->ev_prox);
    if (m->ev_prior) cudaEventDestroy(m->ev_prior);
    msf_dataprox_destroy(m->dp);
    cudaFree(m->d_partial);
    cudaFree(m->d_sums);
    if (m->h_sums) cudaFreeHost(m->h_sums);
    if (m->h_status) cudaFreeHost(m->h_status);
    cudaFree(m->d_meas);
    delete m;
}

extern "C" msf_status msf_mace_step(msf_mace* m, const msf_mace_params* prm, double* h_residual, void* stream) {
    MSF_REQUIRE(m && prm, "msf_mace_step: NULL argument");
    MSF_TRY(check_params(m, prm));
    cudaStream_t st = as_stream(stream);
    if (prm->use_graph) {
        const uint64_t gen = cnn_generation(m->desc.cnn);
        const uint64_t tune = projector_tuning_gen(m->desc.proj);
        if (!m->gexec || !same_params(m->gprm, *prm) || m->gcnn != gen || m->gtune != tune) {
            drop_graph(m->gexec);
            // work outside stream order first: kernel attributes, weight folding
            MSF_TRY(cnn_prepare(m->desc.cnn, st));
            MSF_TRY_CUDA(cudaStreamSynchronize(st));
            MSF_TRY(capture(m->cap, &m->gexec, [&] { return enqueue_step(m, prm, m->cap); }));
            m->gprm = *prm;
            m->gcnn = gen;
            m->gtune = tune;
        }
        MSF_TRY_CUDA(cudaGraphLaunch(m->gexec, st));
    } else {
        MSF_TRY(enqueue_step(m, prm, st));
    }
    if (h_residual) {
        MSF_TRY_CUDA(cudaStreamSynchronize(st));
        MSF_TRY(read_residual(m, h_residual));
    }
    return MSF_OK;
}

extern "C" msf_status msf_mace_set_counts(msf_mace* m, const float* h_counts, double I0, double c, void* stream) {
    MSF_REQUIRE(m && h_counts, "msf_mace_set_counts: NULL argument");
    MSF_REQUIRE(I0 > 0 && c > 0 && isfinite(I0) && isfinite(c), "msf_mace_set_counts: I0 and c must be positive");
    const size_t M = projector_sino_size(m->desc.proj);
    cudaStream_t st = as_stream(stream);
    if (!m->d_meas) {
        if (cudaMalloc(&m->d_meas, 3 * M * sizeof(float)) != cudaSuccess) {
            cudaGetLastError();
            m->d_meas = nullptr;
            return fail(MSF_ERR_NOMEM, "msf_mace_set_counts: out of device memory");
        }
        m->desc.d_y = m->d_meas + M;
        m->desc.d_lambda = m->d_meas + 2 * M;
        drop_graph(m->gexec);   // a captured iteration read the caller's buffers
    }
    MSF_TRY_CUDA(cudaMemcpyAsync(m->d_meas, h_counts, M * sizeof(float), cudaMemcpyHostToDevice, st));
    return msf_weights(m->d_meas, m->d_meas + M, m->d_meas + 2 * M, M, I0, c, stream);
}

extern "C" msf_status msf_mace_batch_create(msf_mace** problems, int n, msf_mace_batch** out) {
    MSF_REQUIRE(problems && out && n > 0, "msf_mace_batch_create: need n > 0 problems");
    *out = nullptr;
    for (int i = 0; i < n; ++i) {
        MSF_REQUIRE(problems[i], "msf_mace_batch_create: problem %d is NULL", i);
        for (int j = 0; j < i; ++j) {
            MSF_REQUIRE(problems[j] != problems[i], "msf_mace_batch_create: problem %d listed twice", i);
            MSF_REQUIRE(!problems[i]->desc.cnn || problems[i]->desc.cnn != problems[j]->desc.cnn,
                        "msf_mace_batch_create: problems %d and %d share a CNN handle (its workspace)", j, i);
            MSF_REQUIRE(problems[i]->desc.proj != problems[j]->desc.proj,
                        "msf_mace_batch_create: problems %d and %d share a projector plan (its workspace)", j, i);
        }
    }
    msf_mace_batch* b = new msf_mace_batch();
    b->items.assign(problems, problems + n);
    b->streams.resize(n, nullptr);
    b->done.resize(n, nullptr);
    bool ok = cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming) == cudaSuccess &&
              cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking) == cudaSuccess;
    for (int i = 0; ok && i < n; ++i)
        ok = cudaStreamCreateWithFlags(&b->streams[i], cudaStreamNonBlocking) == cudaSuccess &&
             cudaEventCreateWithFlags(&b->done[i], cudaEventDisableTiming) == cudaSuccess;
    if (!ok) {
        msf_mace_batch_destroy(b);
        return fail(MSF_ERR_CUDA, "msf_mace_batch_create: cannot create streams");
    }
    *out = b;
    return MSF_OK;
}

extern "C" void msf_mace_batch_destroy(msf_mace_batch* b) {
    if (!b) return;
    drop_graph(b->gexec);
    for (cudaStream_t s : b->streams)
        if (s) cudaStreamDestroy(s);
    for (cudaEvent_t e : b->done)
        if (e) cudaEventDestroy(e);
    if (b->fork) cudaEventDestroy(b->fork);
    if (b->cap) cudaStreamDestroy(b->cap);
    delete b;
}

extern "C" msf_status msf_mace_batch_step(msf_mace_batch* b, const msf_mace_params* prm, double* h_residuals,
                                          void* stream) {
    MSF_REQUIRE(b && prm, "msf_mace_batch_step: NULL argument");
    const int n = (int)b->items.size();
    for (int i = 0; i < n; ++i) MSF_TRY(check_params(b->items[i], &prm[i]));
    cudaStream_t st = as_stream(stream);
    const bool was_shared = b->shared;
    MSF_TRY(decide_shared(b));
    bool graph = true;
    for (int i = 0; i < n; ++i) graph = graph && prm[i].use_graph;
    if (graph) {
        bool fresh = b->gexec != nullptr && (int)b->gprm.size() == n && was_shared == b->shared;
        for (int i = 0; fresh && i < n; ++i)
            fresh = same_params(b->gprm[i], prm[i]) && b->gcnn[i] == cnn_generation(b->items[i]->desc.cnn) &&
                    b->gtune[i] == projector_tuning_gen(b->items[i]->desc.proj);
        if (!fresh) {
            drop_graph(b->gexec);
            for (int i = 0; i < n; ++i) MSF_TRY(cnn_prepare(b->items[i]->desc.cnn, st));
            MSF_TRY_CUDA(cudaStreamSynchronize(st));
            MSF_TRY(capture(b->cap, &b->gexec, [&] { return enqueue_batch(b, prm, b->cap); }));
            b->gprm.assign(prm, prm + n);
            b->gcnn.resize(n);
            b->gtune.resize(n);
            for (int i = 0; i < n; ++i) {
                b->gcnn[i] = cnn_generation(b->items[i]->desc.cnn);
                b->gtune[i] = projector_tuning_gen(b->items[i]->desc.proj);
            }
        }
        MSF_TRY_CUDA(cudaGraphLaunch(b->gexec, st));
    } else {
        MSF_TRY(enqueue_batch(b, prm, st));
    }
    if (h_residuals) {
        MSF_TRY_CUDA(cudaStreamSynchronize(st));
        for (int i = 0; i < n; ++i) MSF_TRY(read_residual(b->items[i], &h_residuals[i]));
    }
    return MSF_OK;
}

extern "C" msf_status msf_mace_consensus(float* d_W, const float* d_X, int K1, size_t N, const double* mu, double rho,
                                         double* d_work, void* stream) {
    MSF_REQUIRE(d_W && d_X && mu && d_work, "msf_mace_consensus: NULL argument");
    MSF_REQUIRE(K1 == 2 || K1 == 4, "msf_mace_consensus: K + 1 must be 2 or 4, got %d", K1);
    MSF_REQUIRE(N > 0, "msf_mace_consensus: empty states");
    MSF_REQUIRE(rho > 0 && rho < 1, "msf_mace_consensus: rho must lie in (0,1) (Eq. (12))");
    double musum = 0.0;
    for (int i = 0; i < K1; ++i) {
        MSF_REQUIRE(mu[i] >= 0, "msf_mace_consensus: agent weights must be non-negative");
        musum += mu[i];
    }
    MSF_REQUIRE(fabs(musum - 1.0) < 1e-9, "msf_mace_consensus: agent weights must sum to 1 (got %.17g)", musum);
    MSF_TRY(check_device());
    MaceCoef c;
    for (int i = 0; i < 4; ++i) c.mu[i] = i < K1 ? (float)mu[i] : 0.0f;
    c.two_rho = (float)(2.0 * rho);
    c.K1 = K1;
    return launch_consensus(d_W, d_X, K1, N, c, d_work, d_work + 2 * CONSENSUS_BLOCKS, as_stream(stream));
}
