/*
 * gbfwi.h - C ABI of the GB300 (sm_103a) library for the data-parallel hot
 * path of preconditioned-BFGS elastic full-waveform inversion with low-rank
 * uncertainty quantification (Liu, Beller, Lei, Peter & Tromp 2020,
 * "Preconditioned BFGS-based uncertainty quantification in elastic full
 * waveform inversion").
 *
 * The path: forward and adjoint 2-D isotropic elastic spectral-element
 * simulations (Section 3.1, Appendix A, Eqs. A6-A18) giving the misfit of
 * Eq. A1 and its gradient; the diagonal Gauss-Newton / illumination maps
 * P1-P4 (Eqs. 4-8, A21-A22) smoothed, damped and inverted into B0; the
 * full-history BFGS inverse Hessian (Eqs. 3 and 9, Algorithms 1-2) applied in
 * compact form to blocks of vectors; and the single-pass randomized SVD of
 * Algorithm 3 giving the low-rank posterior covariance of Eqs. 10-14.
 *
 * Conventions (every entry point):
 *   - Return value: GBFWI_OK (0) or a negative GBFWI_E* code; output
 *     arguments are written only on success.  gbfwi_strerror() names a code.
 *   - Arrays: the caller owns every array argument.  Each array may be host
 *     or device memory; the library looks at the pointer (CUDA pointer
 *     attributes).  Device arrays must belong to the device that is current
 *     during the call (or be managed memory): another GPU's memory is
 *     rejected with GBFWI_EINVAL.  Host arrays are staged through
 *     library-owned device buffers and the call returns only after its host
 *     outputs are written;
 *     with device arrays the work is queued on `stream` (a cudaStream_t, or
 *     NULL for the legacy default stream) and the call returns once it is
 *     queued, except where an entry point says it synchronises.
 *   - Handles (gbfwi_mesh, gbfwi_bfgs) are opaque and library-owned; create
 *     and destroy them through this ABI.  A handle is not thread-safe: use
 *     one handle per host thread / stream.
 *   - Layout: node-grid fields are row-major [nz][nx] with nx = 4 nex + 1,
 *     nz = 4 nez + 1, row 0 at the surface and z = depth (GLL nodes of a
 *     structured mesh of square elements, NGLL = 5).  Parameter vectors are
 *     [3][nz][nx] in the order rho, vp, vs (n = 3 nx nz).  Seismograms are
 *     [nshot][nrec][2][nt] (x then z displacement component), sample n-1
 *     holding time step n (t = n dt), n = 1..nt.
 *   - Precision: wavefields, models, kernels and BFGS vectors are FP32;
 *     misfits and the small BFGS / randomized-SVD matrices are FP64.
 */
#ifndef GBFWI_H
#define GBFWI_H

#ifdef __cplusplus
extern "C" {
#endif

enum {
    GBFWI_OK = 0,
    GBFWI_EINVAL = -1,      /* bad argument (size, pointer, range, order of calls) */
    GBFWI_ENOMEM = -2,      /* device or host allocation failed */
    GBFWI_ECUDA = -3,       /* a CUDA runtime call or kernel launch failed */
    GBFWI_ECFL = -4,        /* dt * vp_max / (min GLL node spacing) > 0.5 */
    GBFWI_ECURV = -5,       /* BFGS pair rejected: y^T s <= 1e-12 |s| |y| */
    GBFWI_ENONFINITE = -6,  /* a NaN or Inf reached the seismograms or the model */
    GBFWI_ETIMEOUT = -7,    /* a time-step kernel's bounded wait for its staged inputs gave up: the
                               simulation results are invalid.  Reported by the next call on the
                               mesh that waits for the device (forward into device memory does not) */
    GBFWI_ENOMODEL = -8,    /* simulation requested before gbfwi_set_model */
    GBFWI_ESCRATCH = -9     /* request larger than the fixed scratch of a no-allocation entry point */
};

/* Largest number of shots gbfwi_misfit_noalloc accepts. */
#define GBFWI_NOALLOC_MAX_SHOTS 256

typedef struct gbfwi_mesh gbfwi_mesh;
typedef struct gbfwi_bfgs gbfwi_bfgs;

/* Structured quad mesh and time axis (Section 3.1: spectral elements,
 * absorbing boundaries; the paper's runs use SPECFEM2D).  Edges other than
 * the top are first-order Stacey absorbing boundaries. */
typedef struct {
    int nex, nez;           /* elements along x and along depth (>= 1) */
    double h;               /* element side in metres (> 0) */
    int ngll;               /* GLL points per direction: must be 5 */
    int free_surface_top;   /* 1: traction-free top edge, 0: Stacey on top too */
    double dt;              /* time step in seconds (> 0) */
    int nt;                 /* time steps; records at n = 1..nt (>= 2) */
    int precision;          /* 0 = FP32 wavefields (the only value accepted) */
} gbfwi_mesh_desc;

/* Ricker point source, r(t) = amp (1 - 2 pi^2 f0^2 (t-t0)^2) exp(-pi^2 f0^2 (t-t0)^2)
 * (Section 3.1 uses a Ricker wavelet).  type 0: explosive moment tensor
 * amp * I (nodal force amp * grad psi(x_s)); type 1 / 2: point force along
 * x / z (nodal force amp * psi(x_s)).  A point on a shared element edge
 * belongs to the element of smaller index. */
typedef struct {
    double x, z;            /* position in metres, z = depth */
    int type;               /* 0 explosive, 1 force x, 2 force z */
    double f0, t0, amp;     /* peak frequency (Hz), delay (s), amplitude */
} gbfwi_source;

/* Launch schedule (chosen by the autotuner or the caller). */
typedef struct {
    int shots_per_launch;   /* shots advanced together in one launch (>= 1) */
    int tile;               /* element-tile variant, 0..gbfwi_num_tiles()-1 */
    int use_graph;          /* 1: replay the time loop as CUDA graphs */
    int ckpt_every;         /* 0: keep the whole forward history on the device;
                               k > 0: keep a snapshot every k steps and
                               recompute each segment during the adjoint */
    int streams;            /* shot batches simulated concurrently on separate
                               library streams by gbfwi_adjoint_gradient (1..8);
                               each keeps its own history */
} gbfwi_schedule;

/* ---------------------------------------------------------------- mesh -- */

/* Build the mesh, GLL tables, source and receiver interpolation tables.
 * src[nsrc] (host), rec_xz[nrec][2] (host, x then depth).  Every point must
 * lie inside the mesh.  -> EINVAL, ENOMEM, ECUDA.  *out receives the handle. */
int gbfwi_mesh_create(const gbfwi_mesh_desc *desc, const gbfwi_source *src, int nsrc,
                      const double *rec_xz, int nrec, gbfwi_mesh **out);

/* Free the mesh and every device buffer it owns.  NULL is accepted. */
int gbfwi_mesh_destroy(gbfwi_mesh *mesh);

/* Node-grid size: *nx = 4 nex + 1, *nz = 4 nez + 1. */
int gbfwi_mesh_dims(const gbfwi_mesh *mesh, int *nx, int *nz);

/* Node coordinates in metres, host arrays [nz][nx]. */
int gbfwi_node_coords(const gbfwi_mesh *mesh, double *x, double *z);

/* Number of element-tile variants the library was built with, and their
 * shapes (tile elements along x, along z). */
int gbfwi_num_tiles(void);
int gbfwi_tile_shape(int tile, int *tx, int *tz);

/* Read / replace the launch schedule. */
int gbfwi_get_schedule(const gbfwi_mesh *mesh, gbfwi_schedule *sch);
int gbfwi_set_schedule(gbfwi_mesh *mesh, const gbfwi_schedule *sch);

/* Model on the node grid, each [nz][nx] FP32 (Eq. A7 parametrisation
 * alpha = vp, beta = vs, rho): lambda = rho (vp^2 - 2 vs^2), mu = rho vs^2.
 * Checks rho > 0, vp > vs > 0, finite values, and the stability bound
 * dt vp_max / dx_min <= 0.5 (dx_min = smallest GLL node spacing) -> ECFL.
 * Synchronises the stream (the check reads the model on the host). */
int gbfwi_set_model(gbfwi_mesh *mesh, const float *rho, const float *vp, const float *vs,
                    void *stream);

/* ------------------------------------------------------------ simulate -- */

/* Forward simulations (Eqs. A6-A7, Newmark beta = 0, gamma = 1/2 with
 * implicit Stacey damping) from rest for the sources shot_ids[nshot] (host
 * ints indexing the mesh's sources).  seis: [nshot][nrec][2][nt] receiver
 * displacements s_n = P u_n.  -> EINVAL, ENOMODEL, ECUDA, ENOMEM. */
int gbfwi_forward(gbfwi_mesh *mesh, const int *shot_ids, int nshot, float *seis, void *stream);

/* Misfit only, f = 1/2 dt sum |s - d|^2 (Eq. A1) summed over the shots: the
 * forward simulations of gbfwi_forward and the residual reduction, without
 * the adjoint (line searches; the forward half of an autograd wrapper).
 * d_obs: [nshot][nrec][2][nt] in shot_ids order.  *misfit: host double.
 * Synchronises the stream.  -> EINVAL, ENOMODEL, ENONFINITE, ECUDA, ENOMEM. */
int gbfwi_misfit(gbfwi_mesh *mesh, const int *shot_ids, int nshot, const float *d_obs, double *misfit,
                 void *stream);

/* Misfit f = 1/2 dt sum |s - d|^2 (Eq. A1) and its exact discrete gradient
 * with respect to the nodal (rho, vp, vs) (the discrete form of Eqs.
 * A16-A18: the adjoint of the time stepping, run backwards and correlated
 * with the forward field), summed over the shots.  d_obs: [nshot][nrec][2][nt]
 * observed data in shot_ids order.  *misfit: host double.  grad: [3][nz][nx].
 * ckpt_every < 0 keeps the mesh schedule; >= 0 overrides its ckpt_every.
 * Synchronises the stream (the misfit is returned on the host).
 * -> EINVAL, ENOMODEL, ENONFINITE, ECUDA, ENOMEM. */
int gbfwi_adjoint_gradient(gbfwi_mesh *mesh, const int *shot_ids, int nshot,
                           const float *d_obs, double *misfit, float *grad,
                           int ckpt_every, void *stream);

/* Diagonal Hessian preconditioner of kind 1..4 (Eqs. 4-8, A21-A22), summed
 * over the shots: P1 source illumination int a.a dt, P2 |int a.abar dt|,
 * P3 Gauss-Newton H_alpha_alpha / H_beta_beta of the source wavefield,
 * P4 the same with the receiver wavefield (driven by the synthetic data,
 * after Eq. A22) and term-wise absolute values.  Each map carries the
 * quadrature measure of its node (like the gradient).  The rho entry is
 * H_rho_rho (Eq. A21/A22, third line) for every kind; P1/P2 give the same
 * map for rho, vp and vs.
 * H:  [3][nz][nx] raw map (may be NULL).
 * B0: [3][nz][nx] = 1 / (S(H) + damp_factor * median(S(H))) per parameter,
 *     S = Gaussian smoothing of standard deviation smooth_sigma_m metres
 *     (quadrature-weighted average in physical space, truncated at 5 sigma).
 * Synchronises the stream.  -> EINVAL, ENOMODEL, ECUDA, ENOMEM. */
int gbfwi_precond_diag(gbfwi_mesh *mesh, const int *shot_ids, int nshot, int kind,
                       double smooth_sigma_m, double damp_factor, float *H, float *B0,
                       void *stream);

/* ---------------------------------------------------------------- BFGS -- */

/* Full-history BFGS store for n unknowns and up to kmax pairs (Section 3.1:
 * every s_i, y_i is kept; the paper memory-maps them), with the diagonal
 * initial inverse Hessian B0[n] (Eq. 4; device or host, copied).  The
 * store (2 kmax n FP32) lives on the current device.  -> EINVAL, ENOMEM. */
int gbfwi_bfgs_create(long long n, int kmax, const float *B0, gbfwi_bfgs **out);

/* Append the pair s = m_{k+1} - m_k, y = g_{k+1} - g_k (Eq. 2) and extend
 * the small matrices S^T Y and Y^T B0 Y of the compact form.  A pair with
 * y^T s <= 1e-12 |s| |y| is not stored -> ECURV; a full store -> EINVAL.
 * Synchronises the stream (the curvature test is read on the host). */
int gbfwi_bfgs_update(gbfwi_bfgs *b, const float *s, const float *y, void *stream);

/* Pairs currently stored (>= 0), or a negative code. */
int gbfwi_bfgs_count(const gbfwi_bfgs *b);

/* Z = (H - minus_B0 * gamma B0) X for a block X[p][n] (rows are vectors),
 * H the BFGS inverse Hessian of Eq. 3 started from gamma * B0 after all
 * stored pairs (Eq. 9), applied in the compact form of Byrd, Nocedal &
 * Schnabel (1994), which equals the two-loop recursions of Algorithms 1
 * (gamma = gamma_k) and 2 (gamma = 1, minus_B0 = 1).  Z: [p][n].
 * 1 <= p <= 256.  -> EINVAL, ECUDA, ENOMEM. */
int gbfwi_bfgs_apply(gbfwi_bfgs *b, const float *X, int p, float *Z, double gamma,
                     int minus_B0, void *stream);

/* Low-rank inverse Hessian and posterior standard deviation (Algorithm 3
 * on B_{n+1} - B0, Eqs. 10-14 with C_m = eps_prior I):
 *   E = (B_{n+1} - B0) X, QR = E, Omega (Q^T X) = Q^T E (Omega symmetrised),
 *   U Lambda U^T = Omega, V = Q U, eigenpairs ordered by |lambda| descending;
 *   std_i = sqrt(eps_prior * max(0, sum_k V_ki^2 lambda_k + B0_i)).
 * X: [p][n] probing block, or NULL to draw standard normals on the device
 * from Philox4x32-10 with `seed` (counter = element index / 4).  V: [rank][n]
 * (may be NULL), lambda: [rank] FP64 (may be NULL), std: [n] (may be NULL).
 * Q is rank-revealing: pivoted Cholesky of the FP64 Gram matrix E E^T (QR
 * with column pivoting on E) keeps the probe rows whose residual norm is at
 * least 1e-4 of the largest (the FP32 data resolve nothing finer), so
 * r = dim Q <= p; Omega (r x r) is then the least-squares solution, equal to
 * the solve above when r = p, and eigenpairs beyond r are returned as
 * lambda = 0 with zero rows of V.  E, Q and the projections are formed in
 * the coordinates of W = [S, B0 Y] (E = C W with C = (M W^T X)^T, the store
 * keeps W^T W), so the n-long work is W^T X and V only.
 * 1 <= rank <= p <= 256.  Synchronises the stream.
 * -> EINVAL, ECUDA, ENOMEM, ENONFINITE (E = 0 or non-finite, a singular
 *    Q^T X). */
int gbfwi_lowrank_invhess(gbfwi_bfgs *b, const float *X, int p, int rank,
                          unsigned long long seed, double eps_prior, float *V,
                          double *lambda, float *std, void *stream);

/* Two-pass variant of gbfwi_lowrank_invhess (Algorithm 3 with the
 * Rayleigh-Ritz second pass of Halko, Martinsson & Tropp 2011, Alg. 5.3):
 * the same probes, E = (B_{n+1} - B0) X and rank-revealing basis Q, then
 * a second application of the compact form to the basis,
 * C = Q (B_{n+1} - B0) Q^T (r x r, symmetrised), U Lambda U^T = C,
 * V = U^T Q.  It avoids the (Q^T X)^-1 of the single pass, whose error
 * grows with cond(Q^T X); in the coordinates of W the second application
 * is a product of small matrices, (G T^T)^T M (G T^T), with G = W^T W.
 * Arguments, outputs and errors as gbfwi_lowrank_invhess.  Synchronises
 * the stream. */
int gbfwi_lowrank_twopass(gbfwi_bfgs *b, const float *X, int p, int rank,
                          unsigned long long seed, double eps_prior, float *V,
                          double *lambda, float *std, void *stream);

/* Exact low-rank part of the retrieved inverse Hessian (Eqs. 9-14 without
 * random probes).  In compact form B_{n+1} - B0 = W M W^T with W = [S, B0 Y]
 * (n x 2k) and M = [[R^-T (D + Y^T B0 Y) R^-1, -R^-T], [-R^-1, 0]], so its
 * rank is at most 2k: Q (orthonormal rows spanning the rows of W^T) from
 * pivoted Cholesky of the column-scaled FP64 Gram matrix W^T W kept by the
 * store (QR with column pivoting; directions below 1e-4 of the largest
 * dropped) and one CholeskyQR pass, both on coordinates (Q = T W^T), then
 * U Lambda U^T = (Q W) M (Q W)^T and V = U^T Q (the one n-long pass).
 * Eigenpairs ordered by |lambda| descending; std as in
 * gbfwi_lowrank_invhess.  V: [rank][n] (may be NULL), lambda: [rank] FP64
 * (may be NULL), std: [n] (may be NULL).  1 <= k <= 128 stored pairs,
 * 1 <= rank <= 2k.  Synchronises the stream.
 * -> EINVAL, ECUDA, ENOMEM, ENONFINITE. */
int gbfwi_lowrank_exact(gbfwi_bfgs *b, int rank, double eps_prior, float *V, double *lambda,
                        float *std, void *stream);

/* Free the store.  NULL is accepted. */
int gbfwi_bfgs_destroy(gbfwi_bfgs *b);

/* ------------------------------------------- learned preconditioner -- */

/* A U-Net that predicts the logarithm of the raw diagonal pseudo-Hessian H
 * (the P-maps of Eqs. 5-8 as returned by gbfwi_precond_diag) from five input
 * channels on an image grid: vp / 4700, vs / 2700, rho / 2500 and the
 * source-illumination and receiver-coverage masks (gbfwi_unet_features).
 * The paper has no learned component: the network is the standard U-Net of
 * Ronneberger, Fischer & Brox (2015) with `levels` levels of base * 2^l
 * channels: per level two 3x3 convolutions with ReLU, 2x2 average pooling
 * down, nearest 2x upsampling up with the skip connection concatenated after
 * the upsampled features, and a 1x1 output convolution.  Weights and stored
 * activations are bfloat16 (round to nearest even), every sum is FP32; the
 * convolutions run as BF16 tensor-core GEMMs.  Its use: B0 of the BFGS from
 * the predicted H through gbfwi_precond_from_hessian, with the computed map
 * as the fallback (the decision is the caller's). */
typedef struct gbfwi_unet gbfwi_unet;

typedef struct {
    int levels;     /* 1 .. 6 */
    int base;       /* channels of level 0, a multiple of 8 */
    int cin, cout;  /* input / output channels (5 and 3 for the preconditioner) */
    int height;     /* image rows, a multiple of 2^(levels-1) */
    int width;      /* image columns, a multiple of 8 * 2^(levels-1) */
} gbfwi_unet_desc;

/* Create a network with all parameters zero (set them with
 * gbfwi_unet_set_params) and its activation buffers for one image.
 * -> EINVAL, ENOMEM, ECUDA. */
int gbfwi_unet_create(const gbfwi_unet_desc *desc, gbfwi_unet **out);

/* Free the network.  NULL is accepted. */
int gbfwi_unet_destroy(gbfwi_unet *net);

/* Length of the flat FP32 parameter vector (padded layout below), or a
 * negative code. */
long long gbfwi_unet_num_params(const gbfwi_unet *net);

/* Layer `layer` (parameter order: encoder levels 0..L-1 with two 3x3
 * convolutions each, decoder levels L-2..0 with two each, the first on
 * [upsampled, skip] channels, then the 1x1 output convolution):
 * info[7] = {cout, cin, k, cout_pad, kc_pad, w_offset, b_offset}.  Its
 * weights are the [cout_pad][kc_pad] block at w_offset of the flat vector,
 * entry (o, c*k*k + ky*k + kx) for W[o][c][ky][kx], zero beyond cout and
 * cin*k*k; its biases the cout_pad entries at b_offset.  layer < 0 returns
 * the number of layers.  -> EINVAL. */
int gbfwi_unet_layer_info(const gbfwi_unet *net, int layer, int *info);

/* Copy the flat parameter vector in (resetting the Adam state) or out.
 * Synchronise the stream.  -> EINVAL, ECUDA. */
int gbfwi_unet_set_params(gbfwi_unet *net, const float *params, void *stream);
int gbfwi_unet_get_params(const gbfwi_unet *net, float *params, void *stream);

/* y [cout][height][width] (FP32) = U-Net(x [cin][height][width]).
 * Synchronises the stream.  -> EINVAL, ENONFINITE, ECUDA. */
int gbfwi_unet_forward(gbfwi_unet *net, const float *x, float *y, void *stream);

/* Gradient of sum(dy * U-Net(x)) with respect to the flat parameter vector
 * (padded entries are zero), for an output gradient dy [cout][height][width];
 * grad: [num_params] FP32.  Synchronises the stream.  -> EINVAL, ECUDA. */
int gbfwi_unet_gradient(gbfwi_unet *net, const float *x, const float *dy, float *grad, void *stream);

/* One Adam step (Kingma & Ba 2015; beta1 0.9, beta2 0.999, eps 1e-8, bias
 * corrected) on the mean over `batch` samples of the mean squared error
 * between U-Net(x_b) and target_b.  x: [batch][cin][height][width], target:
 * [batch][cout][height][width]; *loss (host, may be NULL) = the batch mean
 * of the losses before the step.  batch <= 1024.  Synchronises the stream.
 * -> EINVAL, ENONFINITE, ECUDA. */
int gbfwi_unet_train_step(gbfwi_unet *net, const float *x, const float *target, int batch, double lr,
                          double *loss, void *stream);

/* The five U-Net input channels [5][height][width] for the model (rho, vp,
 * vs: [nz][nx]) on this mesh: vp / 4700, vs / 2700, rho / 2500 and the
 * masks sum_s exp(-|x - x_s|^2 / 2 sigma^2) over the mesh's sources and over
 * its receivers, each divided by its maximum, all bilinearly resampled from
 * the node grid with corner nodes on corner pixels.  Synchronises the
 * stream.  -> EINVAL, ENOMEM, ECUDA. */
int gbfwi_unet_features(gbfwi_mesh *mesh, const float *rho, const float *vp, const float *vs, double sigma_m,
                        int height, int width, float *x, void *stream);

/* Bilinear resampling of device arrays [channels][sh][sw] onto
 * [channels][dh][dw], corner samples aligned; op 1: interpolate log(max(v,
 * 1e-30)); op 2: exponentiate the interpolated value.  -> EINVAL, ECUDA. */
int gbfwi_resample(const float *src, int channels, int sh, int sw, float *dst, int dh, int dw, int op,
                   void *stream);

/* B0 [3][nz][nx] = 1 / (S(H) + damp_factor * median(S(H))) from a given
 * raw map H [3][nz][nx] (for example a predicted one): the smoothing,
 * damping and inversion of gbfwi_precond_diag.  Synchronises the stream.
 * -> EINVAL, ECUDA, ENOMEM. */
int gbfwi_precond_from_hessian(gbfwi_mesh *mesh, const float *H, double smooth_sigma_m, double damp_factor,
                               float *B0, void *stream);

/* -------------------------------------------------- without allocation -- */

/* Per-shot misfit f_s = 1/2 dt sum |s - d|^2 of synthetics against observed
 * data, for callers that must not allocate device memory during the call
 * (for example an application whose own pool or arena owns the GPU memory
 * and forbids further cudaMalloc, or a time-critical loop that cannot afford
 * an allocation failure or the synchronisation of a cudaFree).  The paper
 * has no counterpart: this is the misfit reduction of
 * gbfwi_adjoint_gradient with its scratch in a fixed device array.
 *   syn, obs: device arrays [nshot][samples_per_shot] FP32 (e.g. the
 *             [nshot][nrec][2][nt] seismograms of gbfwi_forward);
 *   misfit:   host array [nshot] FP64, written only on success.
 * nshot <= GBFWI_NOALLOC_MAX_SHOTS, else GBFWI_ESCRATCH.  The call allocates
 * nothing, copies its results to host memory and synchronises the stream, so
 * it cannot be called on a stream that is being captured into a CUDA graph
 * (-> EINVAL).  The first call on a device looks up the scratch array's
 * device address; under CUDA's default lazy module loading that first call
 * is also where the library's device code and the array (about 130 KB) are
 * loaded onto that device, so make it before the memory is handed to the
 * caller's own pool (or load modules eagerly, CUDA_MODULE_LOADING=EAGER).
 * All calls share one scratch array per device and it keeps the last call's
 * partial sums: calls that overlap on the GPU race.
 * -> EINVAL, ESCRATCH, ENONFINITE, ECUDA. */
int gbfwi_misfit_noalloc(const float *syn, const float *obs, int nshot, long long samples_per_shot,
                         double dt, double *misfit, void *stream);

/* ------------------------------------------------------------ counters -- */

/* Kernel launches issued through this library by the calling process since
 * it was loaded (every entry point, every handle).  Host-only. */
long long gbfwi_launch_count(void);

/* Enable (1) or disable (0) per-phase timing of gbfwi_adjoint_gradient on
 * this mesh: CUDA events recorded on the caller's stream around the forward
 * passes and around the adjoint passes of every shot batch. */
int gbfwi_enable_timing(gbfwi_mesh *mesh, int on);

/* Device time (ms) of the forward passes and of the adjoint passes of the
 * most recent timed gbfwi_adjoint_gradient on this mesh, and the number of
 * time-step kernel launches in each (the adjoint passes include the segment
 * recomputation when checkpointing).  -> EINVAL when nothing was timed. */
int gbfwi_last_phase_times(const gbfwi_mesh *mesh, double *fwd_ms, double *adj_ms,
                           long long *fwd_launches, long long *adj_launches);

/* Static description of an error code. */
const char *gbfwi_strerror(int code);

#ifdef __cplusplus
}
#endif
#endif /* GBFWI_H */
