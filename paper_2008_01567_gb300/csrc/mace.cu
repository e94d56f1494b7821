// MACE consensus and the partial-update Mann iteration (Sec. III, Algorithm 1).
//
//   X <- F~(W; X)           (data agent L~ by warm-started CG, prior agents H_k)
//   Z <- G(2X - W)          (Eqs. (8)-(9): weighted average, replicated)
//   W <- W + 2 rho (Z - X)
//
// The consensus update is one pass over the K+1 stacked states that also forms
// the FP64 partial sums of the consensus spread of X.
#include <math.h>

#include "common.cuh"

struct msf_mace {
    msf_mace_desc desc;
    msf_dataprox* dp = nullptr;
    double* d_partial = nullptr;   // [2][nblocks]
    double* d_sums = nullptr;      // [2]
    double* h_sums = nullptr;      // pinned [2]
    int nblocks = 0;
    size_t N = 0;                  // voxels of one 4D volume
};

namespace msf {

struct MaceCoef {
    float mu[4];
    float two_rho;
    int K1;
};

// W_i += 2 rho (sum_j mu_j (2 X_j - W_j) - X_i) for every agent i, and the
// partial sums of sum_i mu_i (X_i - Xbar)^2 and Xbar^2 with Xbar = sum_i mu_i X_i.
template <int K1>
__global__ void __launch_bounds__(256) consensus_kernel(float* __restrict__ W, const float* __restrict__ X,
                                                         size_t N, MaceCoef c, double* __restrict__ partial) {
    double num = 0.0, den = 0.0;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < N; i += (size_t)gridDim.x * blockDim.x) {
        float x[K1], w[K1];
#pragma unroll
        for (int k = 0; k < K1; ++k) {
            x[k] = X[(size_t)k * N + i];
            w[k] = W[(size_t)k * N + i];
        }
        float zbar = 0.0f, xbar = 0.0f;
#pragma unroll
        for (int k = 0; k < K1; ++k) {
            zbar += c.mu[k] * (2.0f * x[k] - w[k]);
            xbar += c.mu[k] * x[k];
        }
        double dev = 0.0;
#pragma unroll
        for (int k = 0; k < K1; ++k) {
            W[(size_t)k * N + i] = w[k] + c.two_rho * (zbar - x[k]);
            const double dxk = (double)x[k] - (double)xbar;
            dev += (double)c.mu[k] * dxk * dxk;
        }
        num += dev;
        den += (double)xbar * (double)xbar;
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

}  // namespace msf

using namespace msf;

extern "C" msf_status msf_mace_create(const msf_mace_desc* desc, msf_mace** out) {
    MSF_REQUIRE(desc && out, "msf_mace_create: NULL argument");
    *out = nullptr;
    MSF_REQUIRE(desc->proj && desc->d_W && desc->d_X && desc->d_y && desc->d_lambda,
                "msf_mace_create: projector, W, X, y and lambda are required");
    if (desc->prior == MSF_PRIOR_CNN) {
        MSF_REQUIRE(desc->K == 3 && desc->cnn, "msf_mace_create: the CNN prior needs K = 3 and a cnn handle");
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
    m->nblocks = 152 * 8;
    if (cudaMalloc(&m->d_partial, 2 * m->nblocks * sizeof(double)) != cudaSuccess ||
        cudaMalloc(&m->d_sums, 2 * sizeof(double)) != cudaSuccess ||
        cudaMallocHost(&m->h_sums, 2 * sizeof(double)) != cudaSuccess) {
        cudaGetLastError();
        msf_mace_destroy(m);
        return fail(MSF_ERR_NOMEM, "msf_mace_create: out of memory");
    }
    *out = m;
    return MSF_OK;
}

extern "C" void msf_mace_destroy(msf_mace* m) {
    if (!m) return;
    msf_dataprox_destroy(m->dp);
    cudaFree(m->d_partial);
    cudaFree(m->d_sums);
    if (m->h_sums) cudaFreeHost(m->h_sums);
    delete m;
}

extern "C" msf_status msf_mace_step(msf_mace* m, const msf_mace_params* prm, double* h_residual, void* stream) {
    MSF_REQUIRE(m && prm, "msf_mace_step: NULL argument");
    MSF_REQUIRE(prm->rho > 0 && prm->rho < 1, "msf_mace_step: rho must lie in (0,1) (Eq. (12))");
    MSF_REQUIRE(prm->sigma > 0, "msf_mace_step: sigma must be positive");
    const int K1 = m->desc.K + 1;
    double musum = 0.0;
    for (int i = 0; i < K1; ++i) {
        MSF_REQUIRE(prm->mu[i] >= 0, "msf_mace_step: agent weights must be non-negative");
        musum += prm->mu[i];
    }
    MSF_REQUIRE(fabs(musum - 1.0) < 1e-9, "msf_mace_step: agent weights must sum to 1 (got %.17g)", musum);
    MSF_REQUIRE(prm->n_cg >= 0 && prm->n_sweeps >= 0, "msf_mace_step: iteration counts must be >= 0");
    cudaStream_t st = as_stream(stream);
    const msf_mace_desc& d = m->desc;
    const size_t N = m->N;
    const msf_vol* vol = projector_volume(d.proj);
    // X_0 <- L~(W_0; X_0)
    MSF_TRY(msf_prox_data(m->dp, d.d_y, d.d_lambda, d.d_W, d.d_X, prm->sigma, prm->n_cg, stream));
    // X_k <- H_k(W_k)
    for (int k = 1; k < K1; ++k) {
        if (d.prior == MSF_PRIOR_QGGMRF) {
            MSF_TRY(msf_prox_qggmrf(vol, &d.mrf, d.d_W + k * N, d.d_X + k * N, prm->sigma, prm->n_sweeps, stream));
        } else {
            MSF_TRY(msf_denoise(d.cnn, (msf_orient)(k - 1), vol, d.d_W + k * N, d.d_X + k * N, stream));
        }
    }
    // Z <- G(2X - W);  W <- W + 2 rho (Z - X)
    MaceCoef c;
    for (int i = 0; i < 4; ++i) c.mu[i] = i < K1 ? (float)prm->mu[i] : 0.0f;
    c.two_rho = (float)(2.0 * prm->rho);
    c.K1 = K1;
    MSF_PROF("mace_consensus", st);
    if (K1 == 2)
        consensus_kernel<2><<<m->nblocks, 256, 0, st>>>(d.d_W, d.d_X, N, c, m->d_partial);
    else
        consensus_kernel<4><<<m->nblocks, 256, 0, st>>>(d.d_W, d.d_X, N, c, m->d_partial);
    MSF_LAUNCH_CHECK();
    {
        MSF_PROF("mace_residual", st);
        sum2_kernel<<<1, 1024, 0, st>>>(m->d_partial, m->nblocks, m->d_sums);
        MSF_LAUNCH_CHECK();
    }
    if (h_residual) {
        MSF_TRY_CUDA(cudaMemcpyAsync(m->h_sums, m->d_sums, 2 * sizeof(double), cudaMemcpyDeviceToHost, st));
        MSF_TRY_CUDA(cudaStreamSynchronize(st));
        const double num = m->h_sums[0], den = m->h_sums[1];
        if (!isfinite(num) || !isfinite(den))
            return fail(MSF_ERR_NUMERIC, "msf_mace_step: non-finite consensus residual");
        *h_residual = den > 0 ? sqrt(num / den) : sqrt(num);
    }
    return MSF_OK;
}
