/*
 * msf.h -- C ABI of the GB300 multi-slice fusion library (libmsf.so).
 *
 * Method: "Multi-Slice Fusion for Sparse-View and Limited-Angle 4D CT
 * Reconstruction" (arXiv 2008.01567).  One Mann iteration of multi-agent
 * consensus equilibrium (MACE) on a 4D (x,y,z,t) volume: a per-frame data
 * proximal map L (Sec. III, Eq. (4)) built on a cone-beam projector A_n
 * (Sec. II, Eq. (2)), K prior agents H_k (Eq. (5)) -- three 2.5D CNN denoisers
 * (Sec. IV, Eq. (14)) or a 4D q-GGMRF MRF prior (Sec. VII) -- and the consensus
 * update of Algorithm 1.
 *
 * Conventions (every entry point):
 *  - Pointers named d_* are device pointers owned by the caller; h_* are host
 *    pointers.  The library never frees caller memory.  Handles own only their
 *    geometry tables, weights and workspaces, all allocated in *_create.
 *  - Work is enqueued asynchronously on `stream` (a cudaStream_t, NULL = legacy
 *    default stream).  Functions that return a host value (h_loss, h_residual)
 *    synchronise that stream before returning.
 *  - Return MSF_OK or an error code; nothing is thrown across the ABI.
 *    Argument errors are detected before any launch.  msf_last_error() gives a
 *    thread-local description of the last failure in the calling thread.
 *  - Layouts: a 3D frame is [nz][ny][nx] (x fastest); a 4D volume is
 *    [nt][nz][ny][nx]; a sinogram is [nt][views][nv][nu] (u fastest); a stack of
 *    K+1 agent states is [K+1][nt][nz][ny][nx].  All float data is FP32.
 *  - Geometry: voxel (ix,iy,iz) has centre ((ix-(nx-1)/2)*voxel, ...), the
 *    rotation axis is z, view angle th puts the source at
 *    (dso cos th, dso sin th, 0) and the detector centre at
 *    -(dsd-dso)(cos th, sin th, 0), with u axis (-sin th, cos th, 0) and v axis
 *    (0,0,1); pixel (iu,iv) sits at (iu-(nu-1)/2)*du, (iv-(nv-1)/2)*dv.
 */
#ifndef MSF_H
#define MSF_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    MSF_OK = 0,
    MSF_ERR_ARG = 1,        /* invalid argument; nothing was launched */
    MSF_ERR_CUDA = 2,       /* a CUDA runtime/driver call failed */
    MSF_ERR_NOMEM = 3,      /* device allocation failed in a *_create call */
    MSF_ERR_TIMEOUT = 4,    /* a bounded device-side wait gave up */
    MSF_ERR_NUMERIC = 5,    /* non-finite value detected in a reduction */
    MSF_ERR_UNSUPPORTED = 6 /* device is not sm_103 / feature not built */
} msf_status;

/* Thread-local message for the last non-OK status returned in this thread. */
const char* msf_last_error(void);
/* Library version string. */
const char* msf_version(void);

/* Per-kernel timing (diagnostics, off by default).  While enabled, every kernel
 * launch of the library is bracketed by a CUDA event pair recorded on the
 * launch's stream.  msf_profile_read synchronises the recorded events and
 * returns the number of distinct kernel names seen since the last reset; for
 * entry i < that number it fills *name (static string), *launches and
 * *total_ms (sum of the launches' event-measured durations).  Not for use
 * while a stream is being captured into a CUDA graph. */
void msf_profile_enable(int on);
void msf_profile_reset(void);
int msf_profile_read(int i, const char** name, int64_t* launches, double* total_ms);

/* Failure-detection self-test (no counterpart in the paper): launches a kernel
 * that waits, with the bounded wait every device-side wait of this library
 * uses, on an mbarrier that nothing completes.  Returns MSF_ERR_TIMEOUT once
 * the wait gives up after limit_ns (at most 2 s); the context stays usable.
 * Synchronises.  Any other status means the bounded wait is broken. */
msf_status msf_selftest_wait(uint64_t limit_ns, void* stream);

/* ------------------------------------------------------------ problem data */

/* One 4D volume: nt frames of nx*ny*nz isotropic voxels of edge `voxel`
 * (the x_n of Sec. II: N = nt * Ns, Ns = nx*ny*nz). */
typedef struct {
    int nx, ny, nz, nt;
    double voxel;
} msf_vol;

/* Circular-orbit flat-detector cone-beam scan (the measurement model of
 * Sec. II; the projection geometry is this library's reading, see msf.h head).
 * `views` views per time-point; angles[t*views + j] in radians (host memory,
 * copied at msf_projector_create). */
typedef struct {
    int nu, nv, views;
    double du, dv;
    double dso, dsd;
    const double* angles;
} msf_geom;

/* ------------------------------------------------------------ projector */

typedef struct msf_projector msf_projector;

/* Builds the projector plan for (geom, vol): a per-(view, detector column)
 * table of ray constants computed in FP64 on the device and stored in FP32.
 * Errors: MSF_ERR_ARG when sizes are non-positive, when the source or detector
 * would lie inside the volume's circumscribed cylinder (dso and dsd-dso must
 * exceed its radius), or when a ray could be steeper than 45 deg to the
 * rotation plane (the z-major case, which this projector does not model).
 * Allocates the table, two z-paired copies of a 4D volume (the forward's
 * inputs, 16*N bytes) and a step-weighted sinogram. */
msf_status msf_projector_create(const msf_geom* geom, const msf_vol* vol, msf_projector** out);
void msf_projector_destroy(msf_projector* p);
/* Device bytes held by the plan. */
size_t msf_projector_bytes(const msf_projector* p);

/* Autotuner: times the forward projector with ray blocks of 32x4, 64x2 and
 * 16x8 (columns x rows) and the gather adjoint with voxel runs of 8, 16 and 32
 * along z (and 64 when the gather grid of 64-voxel runs is still at least 24
 * waves of 8 blocks per SM deep) on this plan's geometry, and keeps the
 * fastest of each for the plan.
 * Results do not depend on the choice (same per-ray arithmetic and the same
 * per-voxel summation order).  Synchronises; allocates a temporary buffer.
 * h_choice (optional, 3 ints) receives {block columns, block rows, z-run}. */
msf_status msf_projector_autotune(msf_projector* p, void* stream, int* h_choice);

/* Sets the same two launch shapes directly (no paper counterpart: a launch
 * parameter, for callers that want a fixed configuration, e.g. to reproduce
 * a tuned run without timing it again).  fwd_cols x fwd_rows must be 32x4,
 * 64x2 or 16x8 and adj_zrun 8, 16, 32 or 64; anything else is MSF_ERR_ARG and
 * leaves the plan unchanged.  Results do not depend on the choice. */
msf_status msf_projector_set_tuning(msf_projector* p, int fwd_cols, int fwd_rows, int adj_zrun);

/* y = A x for every time-point: the system matrix A_n of Sec. II, Eq. (2),
 * modelled as a Joseph ray-driven projector.  For each ray (one per detector
 * pixel and view) the major axis is x when |d_x| >= |d_y| else y; on every
 * voxel-centre plane of that axis the frame is sampled bilinearly at the ray's
 * crossing point (taps outside the volume are zero) and weighted by
 * voxel*|d|/|d_major|.  d_x: [nt][nz][ny][nx]; d_y: [nt][views][nv][nu]
 * (overwritten).  FP32 arithmetic; per-ray constants from the FP64 plan. */
msf_status msf_project(msf_projector* p, const float* d_x, float* d_y, void* stream);

/* x = A^T y for every time-point: the matched adjoint of msf_project, computed
 * as a voxel-driven gather (no atomics) that re-derives, bit for bit, the
 * forward's interpolation weights for every ray touching the voxel.
 * d_y: sinogram; d_x: 4D volume (overwritten). */
msf_status msf_backproject(msf_projector* p, const float* d_y, float* d_x, void* stream);

/* The forward projection of msf_project for callers that cannot allocate
 * device memory.  The paper has no counterpart: this entry exists for host
 * applications that own the GPU's memory budget (their own pool or allocator,
 * or a fixed footprint decided before work starts) and so cannot let a library
 * call cudaMalloc, and for callers that must avoid cudaMalloc's implicit
 * device-wide synchronisation.  It needs no projector plan: the per-column ray
 * table is rebuilt on every call inside a fixed 8 MiB device array that the
 * library defines statically, which every GPU that loads the library holds
 * until the process exits.  The frame is read in its natural layout, so only
 * the caller's d_x and d_y are touched besides that array.
 * Limits: nt*views <= 8192 and nt*views*nu <= 250000; larger scans return
 * MSF_ERR_ARG before any work is enqueued (use msf_projector_create +
 * msf_project).  No cudaMalloc, cudaFree or other allocating call is made.
 * The first call on a device looks up the array's device address (with that
 * device current); make that first call before any stream capture.  All calls
 * share the one array and each call overwrites it, so calls that may overlap
 * on the GPU (different streams, different host threads) race and must be
 * serialised by the caller.  Same layouts as msf_project, and the same result
 * bit for bit (the same FP32 operations per crossing, in the same order).
 * Every (view, column) is checked on the host before any work is enqueued;
 * geometries that msf_projector_create rejects return MSF_ERR_ARG here too. */
msf_status msf_project_static(const msf_geom* geom, const msf_vol* vol, const float* d_x, float* d_y,
                              void* stream);

/* Measurement conditioning for M = nt*views*nv*nu rays:
 *   y = -ln(max(n,1)/I0)                (log-normalised counts)
 *   Lambda = c exp(-y)                   (Sec. II, the diagonal weight Lambda_n)
 * d_counts: photon counts; d_y, d_lambda: outputs (either may be NULL). */
msf_status msf_weights(const float* d_counts, float* d_y, float* d_lambda, size_t m,
                       double I0, double c, void* stream);

/* ------------------------------------------------------------ data agent */

typedef struct msf_dataprox msf_dataprox;

/* Workspace for the data proximal maps (CG and ICD) on the projector's problem
 * size: four 4D volumes, two sinograms and per-frame FP64 partial sums. */
msf_status msf_dataprox_create(msf_projector* p, msf_dataprox** out);
void msf_dataprox_destroy(msf_dataprox* d);

/* Partial-update data proximal map L~(v; x) of Sec. III, Eq. (13): n_cg
 * conjugate-gradient iterations on
 *     (A^T Lambda A + I/sigma^2) z = A^T Lambda y + v/sigma^2
 * (the minimiser of Eq. (4) with l from Eq. (2)), one independent solve per
 * time-point, warm-started from d_x and written back to d_x.  Vectors are FP32;
 * the dot products and the step scalars alpha, beta are FP64 per frame.
 * d_y, d_lambda: sinogram-shaped; d_v, d_x: 4D volumes.  sigma > 0, n_cg >= 0. */
msf_status msf_prox_data(msf_dataprox* d, const float* d_y, const float* d_lambda,
                         const float* d_v, float* d_x, double sigma, int n_cg, void* stream);

/* Partial-update data proximal map L~(v; x) of Sec. III, Eq. (13), by
 * iterative coordinate descent (the paper's own choice for L~, "a few ICD
 * iterations"), on the cost of Eq. (4) with l from Eq. (2):
 *     1/2 ||y - A z||^2_Lambda + ||z - v||^2 / (2 sigma^2),
 * one independent solve per time-point, warm-started from d_x and written back.
 * The voxel order is grouped so that a GPU can update many voxels at once: a
 * sweep visits the eight parity groups g = (pz*2 + py)*2 + px, (pz,py,px) =
 * (z,y,x) mod 2, in increasing order.  Inside a group every voxel s takes its
 * own coordinate Newton step against the same error sinogram e = y - A z,
 *     delta_s = -theta1_s / theta2_s,
 *     theta1_s = -(A^T Lambda e)_s + (z_s - v_s)/sigma^2,
 *     theta2_s = (A^T Lambda A)_ss + 1/sigma^2,
 * and the group moves by alpha_t * delta with alpha_t the exact minimiser of the
 * cost of frame t along delta; then e is updated.  (With one voxel per group
 * alpha = 1 and this is sequential ICD; with groups every step still lowers the
 * cost.)  n_sweeps sweeps; vectors FP32, the group sums and alpha FP64.
 * Same arguments and workspace as msf_prox_data; sigma > 0, n_sweeps >= 0. */
msf_status msf_prox_data_icd(msf_dataprox* d, const float* d_y, const float* d_lambda,
                             const float* d_v, float* d_x, double sigma, int n_sweeps, void* stream);

/* ------------------------------------------------------------ q-GGMRF agent */

/* 4D q-GGMRF MRF prior (Sec. VII, "MBIR+4D-MRF"): 26 spatial neighbours with
 * weights proportional to 1/distance normalised to sum 1, plus the two temporal
 * neighbours with weight b_temporal each; free boundaries.  Potential
 * rho(D) = |D|^p/(p sx^p) * u/(1+u), u = |D/(T sx)|^(q-p).  p must be 2 and
 * 1 <= q <= 2 (the symmetric-bound surrogate is then finite everywhere). */
typedef struct {
    double p, q, T, sigma_x, b_temporal;
} msf_mrf;

/* Prior proximal map H(v) of Sec. III, Eq. (5) for the q-GGMRF prior:
 * n_sweeps ICD sweeps in place on d_x (its content is the starting point).
 * A sweep visits the 16 parity colours ((pt*2+pz)*2+py)*2+px in increasing
 * order; each voxel takes the minimiser of the symmetric-bound surrogate
 *   z_s = (v_s/sigma^2 + 2 sum_r b_sr a(z_s-z_r) z_r) / (1/sigma^2 + 2 sum_r b_sr a(z_s-z_r)).
 * d_v, d_x: 4D volumes [nt][nz][ny][nx]. */
msf_status msf_prox_qggmrf(const msf_vol* vol, const msf_mrf* prm, const float* d_v, float* d_x,
                           double sigma, int n_sweeps, void* stream);

/* ------------------------------------------------------------ direct MAP (MBIR + 4D-MRF) */

/* The "MBIR + 4D-MRF" comparison of Sec. VI solved directly, without the MACE
 * split: the MAP estimate of Eq. (3),
 *     x* = argmin_x  l(x) + beta h(x),   l(x) = 1/2 sum_t ||y_t - A_t x_t||^2_Lambda,
 * with h the 4D q-GGMRF prior of msf_prox_qggmrf.  (With proximal agents and
 * weights mu = (mu_0, mu_1) the MACE equilibrium of Sec. III is this point with
 * beta = mu_1 / mu_0.)  The workspace holds four 4D volumes and a sinogram. */
typedef struct msf_map msf_map;
msf_status msf_map_create(msf_projector* p, msf_map** out);
void msf_map_destroy(msf_map* m);

/* Majorise-minimise: each of n_outer outer iterations replaces h by its
 * symmetric-bound quadratic surrogate built at the current x (equal to h there,
 * above it elsewhere: weights a(x_s - x_r) = rho'/(2 D) on every neighbour
 * pair) and takes n_cg conjugate-gradient steps, warm-started at x, on
 *     (A^T Lambda A + 2 beta L_a) x = A^T Lambda y,
 * (L_a x)_s = sum_r b_sr a_sr (x_s - x_r), over the whole 4D volume (the prior
 * couples the time-points, so the CG scalars are global; FP64).  Every outer
 * iteration lowers the cost.  d_x: warm start, overwritten.  beta > 0,
 * prm as msf_prox_qggmrf (p = 2, 1 <= q <= 2).  A non-finite CG scalar is
 * reported by the next msf_map_cost as MSF_ERR_NUMERIC. */
msf_status msf_map_solve(msf_map* m, const msf_mrf* prm, double beta, const float* d_y, const float* d_lambda,
                         float* d_x, int n_outer, int n_cg, void* stream);

/* h_cost[0] = l(x) + beta h(x) of Eq. (3) at d_x (FP64 sums; synchronises). */
msf_status msf_map_cost(msf_map* m, const msf_mrf* prm, double beta, const float* d_y, const float* d_lambda,
                        const float* d_x, double* h_cost, void* stream);

/* ------------------------------------------------------------ fixture correction (Appendix A) */

/* Blind correction of fixtures outside the field of view (Appendix A,
 * Algorithm 2): the shadow of out-of-view holders is smooth, so after removing
 * the projection of the masked reconstruction what remains, blurred, is mostly
 * that shadow, and a least-squares multiple of it is subtracted from y:
 *     x^m = x inside the cylinder |(x, y)| <= r_mask about the rotation axis
 *           (voxel centres; 0 outside),
 *     e   = y - A x^m                       (msf_project of the plan),
 *     p   = blur(e): every view blurred along u, then along v, by normalised
 *           Gaussian taps g_k ~ exp(-k^2/(2 blur_sigma^2)), |k| <= ceil(3 blur_sigma)
 *           (detector pixels; taps beyond the detector edge count as zero),
 *     c   = <e, p> / <p, p>  (FP64, one scalar for the whole scan; 0 if p = 0),
 *     y^corr = y - c p.
 * d_x is the reconstruction x = recon(y, A) of the algorithm's first line (the
 * caller's: e.g. X_0 of a MACE run); d_y, d_ycorr: sinograms (must differ);
 * 0 < blur_sigma <= 64/3 pixels.  h_c (optional, synchronises) receives c.
 * The workspace holds one 4D volume and two sinograms. */
typedef struct msf_fixcorr msf_fixcorr;
msf_status msf_fixcorr_create(msf_projector* p, msf_fixcorr** out);
void msf_fixcorr_destroy(msf_fixcorr* f);
msf_status msf_fixture_correct(msf_fixcorr* f, const float* d_y, const float* d_x, double r_mask, double blur_sigma,
                               float* d_ycorr, double* h_c, void* stream);

/* ------------------------------------------------------------ CNN agents */

/* Agent orientation (Sec. IV): convolution plane and slicing axis.
 * XY_T: slices z, image rows y, cols x.  YZ_T: slices x, rows z, cols y.
 * ZX_T: slices y, rows x, cols z.  Channels: time-points t-2..t+2 of the same
 * slice, clamped at the first and last time-point. */
typedef enum { MSF_XY_T = 0, MSF_YZ_T = 1, MSF_ZX_T = 2 } msf_orient;

typedef struct msf_cnn msf_cnn;

/* The 2.5D residual CNN of Sec. IV: layer 1 conv 5->64 + bias + ReLU; layers
 * 2..9 conv 64->64 + BatchNorm + ReLU; layer 10 conv 64->1 + bias; output
 * = centre frame - network output (residual through the centre channel).
 * 3x3 kernels, zero padding.  Inference runs BF16 tcgen05 implicit-GEMM
 * convolutions with FP32 accumulation and BatchNorm folded into the weights.
 * max_pixels bounds the images * H * W processed per internal chunk
 * (activation workspace = 2 * max_pixels * 128 bytes). */
msf_status msf_cnn_create(int64_t max_pixels, msf_cnn** out);
void msf_cnn_destroy(msf_cnn* c);

/* Number of FP32 parameters in the flat host layout used by set/get:
 * for l = 1..10: W_l [Cout][Cin][3][3] then b_l [Cout]; then for l = 2..9:
 * gamma_l[64], beta_l[64], running_mean_l[64], running_var_l[64]. */
size_t msf_cnn_param_count(void);
msf_status msf_cnn_set_params(msf_cnn* c, const float* h_params, size_t n);
msf_status msf_cnn_get_params(msf_cnn* c, float* h_params, size_t n);

/* Agent H_{orient,t}: d_in, d_out are 4D volumes described by vol.
 * Each output voxel = centre - CNN(5-frame window), computed slice by slice,
 * time-points in chunks (as many as max_pixels holds, at most 16, unless tuned).
 * The 64 -> 64 layers run as 32 x 8 row-pair tiles (two output rows share each
 * input slice through an N = 128 MMA) when the slice height is even, else as
 * 16 x 8 tiles, unless a tuning for this slice shape says otherwise. */
msf_status msf_denoise(msf_cnn* c, msf_orient orient, const msf_vol* vol,
                       const float* d_in, float* d_out, void* stream);

/* The agent H_{orient,t} of several problems at once (Sec. IV; the batch of
 * uneven problems): d_in[i], d_out[i] are problem i's 4D volumes vols[i], each
 * with its own handle cnns[i] (its activation workspace; handles must differ).
 * Every handle must hold the same parameters.  Problems whose time-points all
 * fit in one chunk of their handle and whose slices take row-pair tiles run
 * their 64 -> 64 layers together: one persistent launch per layer walks a work
 * list of (problem, tile) over all of them, with the first handle's weights;
 * their first layers and output stencils run per problem.  Other problems run
 * msf_denoise on their own.  Results equal msf_denoise's bit for bit.  At most
 * 16 problems. */
msf_status msf_denoise_batch(msf_cnn* const* cnns, int n, msf_orient orient, const msf_vol* vols,
                             const float* const* d_in, float* const* d_out, void* stream);

/* Conv launch tuning (no paper counterpart).  For the slices of `vol` in
 * orientation `orient`, msf_denoise uses the given 64 -> 64 tile shape and
 * `chunk` time-points per chunk (0: as many as fit, at most 16; never more
 * than max_pixels allows).  MSF_TILE_AUTO picks row pairs for even heights;
 * MSF_TILE_PAIR needs an even height.  The tile shape changes the order of the
 * FP32 accumulation inside the MMAs, so outputs may differ between shapes by
 * BF16 rounding of stored activations (both match the oracle within the
 * agent's tolerance); the chunk size does not change results. */
enum { MSF_TILE_AUTO = 0, MSF_TILE_16x8 = 1, MSF_TILE_PAIR = 2 };
msf_status msf_cnn_set_tuning(msf_cnn* c, msf_orient orient, const msf_vol* vol, int tile, int chunk);

/* Conv autotuner: for every orientation times msf_denoise on d_in (output to
 * d_out, which must differ) with each tile shape that fits (row pairs, 16 x 8)
 * and 16, 8 and 4 time-points per chunk (those below nt), and keeps the
 * fastest for vol's slice shapes.  Synchronises.  h_choice (optional, 6 ints)
 * receives {tile, chunk} per orientation. */
msf_status msf_cnn_autotune(msf_cnn* c, const msf_vol* vol, const float* d_in, float* d_out, void* stream,
                            int* h_choice);

/* One training step (Sec. V): forward with BatchNorm batch statistics, MSE loss
 * mean((out - clean)^2), backward, and Adam (beta1 0.9, beta2 0.999, eps 1e-8,
 * bias-corrected) on FP32 master weights; running BatchNorm statistics are
 * updated with momentum 0.1.  d_noisy: [B][5][H][W], d_clean: [B][H][W].
 * h_loss (optional) receives the loss of this step (synchronises). */
msf_status msf_train_step(msf_cnn* c, const float* d_noisy, const float* d_clean,
                          int B, int H, int W, float lr, float* h_loss, void* stream);

/* Reserves the training workspace for batches of up to max_train_pixels =
 * B*H*W pixels (about 3.7 KB per pixel: every layer's BF16 activations, FP32
 * pre-BatchNorm outputs, gradients and reduction buffers).  Must precede
 * msf_train_step; a larger reservation replaces a smaller one.
 * MSF_ERR_ARG unless 128 <= max_train_pixels <= 2^28. */
msf_status msf_cnn_train_reserve(msf_cnn* c, int64_t max_train_pixels);

/* Copies the gradients of the last msf_train_step (flat layout of
 * msf_cnn_get_params; the running-statistics entries are zero). */
msf_status msf_cnn_get_grads(msf_cnn* c, float* h_grads, size_t n);

/* Inspection of the last msf_train_step (no paper counterpart: test and debug
 * access to the intermediate tensors, so that every forward and backward
 * kernel can be checked on its own).  msf_cnn_train_trace(c, 1) (after
 * msf_cnn_train_reserve) makes every following step also keep the gradients
 * between layers, 18 BF16 tensors of the reserved pixel count (off: 0 frees
 * them).  msf_cnn_train_tensor copies one tensor of the last step to host
 * memory (synchronises the device); bytes must be its exact size, with
 * P = B*H*W of that step and pixels in [B][H][W] order:
 *   MSF_TT_ACT  layer 1..9: input of conv layer l (after ReLU), BF16 [P][64]
 *   MSF_TT_Z    layer 1..8: conv output before BatchNorm, FP32 [P][64]
 *   MSF_TT_DZ   layer 0..8: loss gradient w.r.t. conv l's output, BF16 [P][64]
 *               (needs the trace)
 *   MSF_TT_DA   layer 1..9: loss gradient w.r.t. conv l's input, BF16 [P][64]
 *               (needs the trace)
 *   MSF_TT_R    network output R (last conv), FP32 [P]; MSF_TT_DR its gradient
 *   MSF_TT_BN   layer 1..8: batch mean and 1/sqrt(var + eps), FP32 [2][64] */
enum { MSF_TT_ACT = 0, MSF_TT_Z = 1, MSF_TT_DZ = 2, MSF_TT_DA = 3, MSF_TT_R = 4, MSF_TT_DR = 5, MSF_TT_BN = 6 };
msf_status msf_cnn_train_trace(msf_cnn* c, int on);
msf_status msf_cnn_train_tensor(msf_cnn* c, int kind, int layer, void* h_dst, size_t bytes);

/* Training pairs (Sec. V: clean patches plus additive white Gaussian noise):
 * B patches of H x W with 5 channels cut from the clean volume stack d_vol
 * (vol->nt volumes of nx*ny*nz).  Each patch takes a random volume, a random
 * slicing axis whose 5 adjacent slices (clamped) stand in for the 5
 * time-points, a random slice and position, a random flip/transpose, and
 * noise sigma ~ U[sigma_lo, sigma_hi]; every channel gets independent
 * N(0, sigma^2) noise from a counter-based hash of (seed, element).
 * d_noisy: [B][5][H][W]; d_clean: [B][H][W] (the clean centre slice). */
msf_status msf_training_batch(const float* d_vol, const msf_vol* vol, int B, int H, int W, double sigma_lo,
                              double sigma_hi, uint64_t seed, float* d_noisy, float* d_clean, void* stream);

/* ------------------------------------------------------------ MACE */

typedef enum { MSF_PRIOR_QGGMRF = 0, MSF_PRIOR_CNN = 1 } msf_prior_kind;

typedef struct msf_mace msf_mace;

/* A MACE problem.  K prior agents: with MSF_PRIOR_CNN and K = 3 the agents
 * are H_xy,t, H_yz,t, H_zx,t sharing `cnn` (Eq. (14)); with MSF_PRIOR_CNN and
 * K = 1 the single agent is the CNN of orientation `orient` (the "MBIR + H" PnP
 * comparison of Sec. VI: one CNN prior beside the data agent); with
 * MSF_PRIOR_QGGMRF, K = 1 and the agent is the q-GGMRF prox with `mrf`.
 * `orient` is read only for the single-CNN case.  d_W and d_X hold the
 * K+1 stacked states [K+1][nt][nz][ny][nx] (caller-owned, initialised by the
 * caller; Algorithm 1 starts from W = X = [x0; ...; x0]).  d_y, d_lambda: the
 * measurements and weights.  The handle borrows proj and cnn. */
typedef struct {
    msf_projector* proj;
    msf_prior_kind prior;
    int K;
    msf_cnn* cnn;
    msf_mrf mrf;
    float* d_W;
    float* d_X;
    const float* d_y;
    const float* d_lambda;
    msf_orient orient;
} msf_mace_desc;

typedef struct {
    double rho;       /* Mann weight, 0 < rho < 1 (Eq. (12)) */
    double sigma;     /* proximal scale sigma > 0 (Eqs. (4)-(5)) */
    double mu[4];     /* agent weights of the average, Eq. (9); sum to 1 */
    int n_cg;         /* CG iterations of the partial update L~ (Eq. (13)) */
    int n_sweeps;     /* ICD sweeps of the q-GGMRF agent per iteration */
    int use_graph;    /* non-zero: run the iteration as a CUDA graph (see msf_mace_step) */
    int n_icd;        /* > 0: the data agent runs n_icd grouped-ICD sweeps
                         (msf_prox_data_icd) instead of n_cg CG iterations */
} msf_mace_params;

msf_status msf_mace_create(const msf_mace_desc* desc, msf_mace** out);
void msf_mace_destroy(msf_mace* m);

/* One pass of Algorithm 1:  X <- F~(W; X);  Z <- G(2X - W);  W <- W + 2 rho (Z - X).
 * X_0 <- L~(W_0; X_0) (warm-started CG), X_k <- H_k(W_k); the average of Eq. (9)
 * uses mu.  h_residual (optional, synchronises) receives the FP64 consensus
 * spread sqrt(sum_i mu_i ||X_i - Xbar||^2) / ||Xbar|| of the new X; a
 * non-finite CG or ICD scalar of the data agent in this or an earlier step is
 * reported there as MSF_ERR_NUMERIC.
 * With the q-GGMRF prior the data agent and the prior agent run concurrently
 * on two internal streams forked from `stream` and joined before the
 * consensus (the CNN agents run in stream order); the step as a whole is
 * ordered on `stream`.
 * With prm->use_graph the whole iteration (every kernel and the residual copy)
 * is captured once on an internal stream into a CUDA graph and replayed on
 * `stream`; the graph is re-captured when the parameters, the CNN's weights
 * or the projector's launch shapes (autotune, set_tuning) change.  Results
 * are identical to the eager path. */
msf_status msf_mace_step(msf_mace* m, const msf_mace_params* prm, double* h_residual, void* stream);

/* New measurements for a MACE problem from host memory: copies the photon
 * counts h_counts (host, [nt][views][nv][nu] FP32; pinned memory makes the
 * copy asynchronous) into the handle and forms y = -ln(max(n,1)/I0) and
 * Lambda = c exp(-y) there (msf_weights); from then on the handle's steps use
 * these instead of desc.d_y and desc.d_lambda.  The first call allocates three
 * sinograms in the handle (outside any stream capture) and drops a captured
 * iteration; later calls allocate nothing.  Ordered on `stream`. */
msf_status msf_mace_set_counts(msf_mace* m, const float* h_counts, double I0, double c, void* stream);

/* The consensus and Mann update of Algorithm 1 alone (Sec. III, Eqs. (8), (9),
 * (12)): W_i <- W_i + 2 rho (sum_j mu_j (2 X_j - W_j) - X_i) on caller-owned
 * stacks d_W, d_X of K1 = K + 1 states of N voxels each ([K1][N], FP32, K1 = 2
 * or 4), for callers that run the agents themselves -- e.g. one problem split
 * by time-point over ranks, each rank passing its own frames.  Also forms the
 * two FP64 sums of the consensus spread over these voxels,
 * d_work[MSF_CONSENSUS_SUMS] = sum_i mu_i ||X_i - Xbar||^2 and
 * d_work[MSF_CONSENSUS_SUMS + 1] = ||Xbar||^2 (device memory; the spread of
 * msf_mace_step is sqrt(first / second), with sums over all ranks when split).
 * d_work: device workspace of MSF_CONSENSUS_WORK doubles, owned by the caller.
 * Same kernels as msf_mace_step's consensus.  Errors: MSF_ERR_ARG for NULL
 * pointers, another K1, N = 0, rho outside (0,1), negative weights or weights
 * not summing to 1, before any launch. */
#define MSF_CONSENSUS_SUMS 2432
#define MSF_CONSENSUS_WORK 2434
msf_status msf_mace_consensus(float* d_W, const float* d_X, int K1, size_t N, const double* mu, double rho,
                              double* d_work, void* stream);

/* A queue of independent (uneven) MACE problems advanced together: each
 * problem runs on its own internal stream forked from the caller's stream and
 * joined back, so small problems share the GPU; with use_graph set for every
 * problem the whole batch iteration is one captured CUDA graph.  When every
 * problem runs the three CNN agents and all their handles hold the same
 * parameters (checked on the host whenever a handle's parameters change), the
 * data agents run forked as above and each orientation's CNN agents of all
 * problems run through msf_denoise_batch (multi-problem persistent launches).
 * Either way the results equal per-problem msf_mace_step bit for bit.
 * Problems must not share a projector plan or a CNN handle (their workspaces). */
typedef struct msf_mace_batch msf_mace_batch;
msf_status msf_mace_batch_create(msf_mace** problems, int n, msf_mace_batch** out);
void msf_mace_batch_destroy(msf_mace_batch* b);
/* prm: n parameter sets; h_residuals (optional, n values) synchronises. */
msf_status msf_mace_batch_step(msf_mace_batch* b, const msf_mace_params* prm, double* h_residuals, void* stream);

/* ------------------------------------------------------------ phantoms (test/bench data) */

/* Ellipsoid phantom records, 16 doubles each (host): centre(3), semi-axes(3),
 * rotation (9, row-major, row k = k-th axis), attenuation mu(1); overlaps add.
 * ell[t*n_ell + e] describes ellipsoid e at time-point t. */

/* Supersampled voxelisation: value = sum_e mu_e * fraction of the ss^3
 * sub-voxel sample points inside e.  d_x: 4D volume. */
msf_status msf_phantom_voxelize(const msf_vol* vol, const double* h_ell, int n_ell, int ss,
                                float* d_x, void* stream);
/* Exact line integrals of the phantom along every ray of the plan's scan. */
msf_status msf_phantom_project(msf_projector* p, const double* h_ell, int n_ell,
                               float* d_y, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* MSF_H */
