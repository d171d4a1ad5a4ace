/*
 * kcs.h -- C ABI of the Kinetic Compressive Sensing hot path on one B300 GPU.
 *
 * The library implements the Iterated Conditional Modes loop of Scipioni et
 * al., "Kinetic Compressive Sensing" (Sec. II-D): (a) the OS-MAP-OSL update of
 * every frame's activity image with the kinetics-derived prior (Eq. 2-3) and
 * (b) the voxel-parallel MAP Levenberg-Marquardt fit of the FDG two-tissue
 * irreversible model under a Huber prior on the kinetic maps (Eq. 4-6).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - Every function returns an int status (KCS_OK = 0).  On failure the
 *    thread-local text of kcs_last_error() says why; nothing has been
 *    launched when the status is KCS_ERR_INVALID_ARG.
 *  - Array arguments are DEVICE pointers owned by the caller, float32,
 *    C-contiguous in the layouts stated below, 16-byte aligned; the library
 *    never frees them and never keeps them beyond the call, except inside a
 *    kcs_study_t, which stores the pointers its descriptor names (the caller
 *    keeps them alive until kcs_destroy_study).
 *  - Compute calls take a cudaStream_t (passed as void*, NULL = legacy default
 *    stream), are asynchronous on that stream and allocate nothing; scratch
 *    memory is passed in as a workspace whose size the *_workspace_size
 *    functions report.  Only the create_* functions allocate (small tables).
 *  - Layouts (Z planes, ny rows, nx columns, A angles, B bins, M frames):
 *      image x, model TAC F       [Z][ny][nx][M]   (frames innermost)
 *      sinogram (counts, randoms) [Z][A][B][M]     (angles in natural order)
 *      subset sinogram            [Z][A_k][B][M]   (A_k angles of subset k)
 *      kinetic maps               [4][Z][ny][nx]   (K1, k2, k3, Vb planes)
 *      per-voxel scalars          [Z][ny][nx]
 *    n_frames must be a multiple of 4 and at most 32.
 *  - Time is in minutes; frame_dt are frame durations.
 */
#ifndef KCS_H
#define KCS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct kcs_geometry kcs_geometry_t;
typedef struct kcs_kinetics kcs_kinetics_t;
typedef struct kcs_study kcs_study_t;

enum kcs_status {
  KCS_OK = 0,
  KCS_ERR_INVALID_ARG = 1,
  KCS_ERR_CUDA = 2,
  KCS_ERR_OOM = 3,
  KCS_ERR_TIMEOUT = 4,
  KCS_ERR_UNIMPLEMENTED = 5,
  KCS_ERR_RANGE = 6
};

/* Layout of the randoms argument of the OSL calls. */
enum kcs_randoms_layout {
  KCS_RANDOMS_NONE = 0,      /* no randoms (pointer ignored)            */
  KCS_RANDOMS_PER_FRAME = 1, /* float [M]: the same r_m in every bin     */
  KCS_RANDOMS_FULL = 2       /* float [Z][A][B][M]                       */
};

/* Storage type of an image / ratio sinogram (KCS_F32, KCS_BF16, KCS_F16) or of
 * the counts (KCS_F32, KCS_U16) in the *_ex entry points (the precision form).
 * Arithmetic is float32 whatever the storage; a stored image holds x / scale_m
 * with a caller-chosen per-frame scale [M] (device; NULL = 1); a 16-bit image
 * or ratio array must be 8-byte aligned.  Half-precision stores saturate at
 * 65504 instead of overflowing. */
enum kcs_storage {
  KCS_F32 = 0,
  KCS_BF16 = 1,
  KCS_F16 = 2,
  KCS_U16 = 3
};

/* Thread-local description of the last failure on this thread ("" if none). */
const char* kcs_last_error(void);
/* ABI version, incremented on any incompatible change. */
int kcs_version(void);

/* ---------------------------------------------------------------- geometry
 * Parallel-beam stacked-2D geometry with a ray-driven Joseph projector; the
 * system matrix p_vd of Eq. 2 (the paper leaves the projector unnamed).
 * Voxel (i, j) has centre ((i-(nx-1)/2) h, (j-(ny-1)/2) h), h = vox_mm.
 * Angle a has theta = a*pi/A; bin b has offset u = (b-(B-1)/2) bin_mm and
 * the ray {p : p.(cos theta, sin theta) = u}.  Angles with A <= 4a <= 3A are
 * sampled at every column (rows interpolated linearly), the others at every
 * row; step weight h / max(|cos|,|sin|).  Ordered subset k holds the angles
 * a = k, k+S, k+2S, ... (the "OS" of OS-MAP-OSL, Sec. I).
 * Allocates a small per-angle table on the current device. */
int kcs_create_geometry(kcs_geometry_t** out, int nx, int ny, int nz, float vox_mm,
                        int n_bins, int n_angles, float bin_mm, int n_subsets);
/* The same, with the per-angle table uploaded asynchronously on stream: the
 * geometry is ready for work issued later on that stream (or after the stream
 * has been synchronised); kcs_create_geometry waits for the upload. */
int kcs_create_geometry_ex(kcs_geometry_t** out, int nx, int ny, int nz, float vox_mm,
                           int n_bins, int n_angles, float bin_mm, int n_subsets, void* stream);
int kcs_destroy_geometry(kcs_geometry_t* g);
/* Host copy of the angle indices of subset k (subset = -1: all angles).
 * angles_out may be NULL to query the count only. */
int kcs_geometry_subset_angles(const kcs_geometry_t* g, int subset, int* angles_out,
                               int* n_out);

/* y = P_k x: forward projection of every frame onto the rays of subset k
 * (subset = -1: all angles).  x [Z][ny][nx][M] -> y [Z][A_k][B][M]
 * (overwritten).  The weights are the geometric p_vd (no frame duration). */
int kcs_forward_project(const kcs_geometry_t* g, int subset, int n_frames,
                        const float* x, float* y, void* stream);
/* x = P_k^T y: the exact transpose of kcs_forward_project (same (v, d, w)
 * triples, gathered per voxel, no atomics).  y [Z][A_k][B][M] ->
 * x [Z][ny][nx][M] (overwritten). */
int kcs_back_project(const kcs_geometry_t* g, int subset, int n_frames,
                     const float* y, float* x, void* stream);
/* Precision form of the two calls above (Eq. 2's sums over stored data):
 * kcs_forward_project_ex projects an image stored as x_type (KCS_F32,
 * KCS_BF16, KCS_F16) holding x / x_scale[m] (x_scale [M] device, NULL = 1),
 * accumulating in float32: y = P_k (x_scale * x) as float32.
 * kcs_back_project_ex back-projects a sinogram stored as y_type holding
 * y / y_scale[m]: x = P_k^T (y_scale * y) as float32, the exact transpose of
 * kcs_forward_project_ex.  16-bit arrays must be 8-byte aligned.  With KCS_F32
 * and NULL scales both equal the plain calls bit for bit. */
int kcs_forward_project_ex(const kcs_geometry_t* g, int subset, int n_frames, const void* x,
                           int x_type, const float* x_scale, float* y, void* stream);
int kcs_back_project_ex(const kcs_geometry_t* g, int subset, int n_frames, const void* y,
                        int y_type, const float* y_scale, float* x, void* stream);
/* sens = sum_{d in S_k} n_d p_vd per voxel [Z][ny][nx] (bin_factor NULL: n_d = 1). */
int kcs_sensitivity(const kcs_geometry_t* g, int subset, const float* bin_factor,
                    float* sens, void* stream);

/* -------------------------------------------------------- OS-MAP-OSL (a)
 * One OS-MAP-OSL-KP update of every frame on subset k (Eq. 2 with the
 * kinetics-derived prior of Eq. 3), in place on x:
 *   ybar = kappa dt_m n_d (P x)_dm + r_dm,   rho = s / ybar (0 if ybar <= 0)
 *   x <- x * kappa dt_m (P_k^T n rho)_vm
 *          / max(kappa dt_m sens_v + (beta/S)(x - F)/sigma2, 1e-3 kappa dt_m sens_v)
 * with sens_v = sum_{d in S_k} n_d p_vd; voxels with sens_v = 0 keep x.
 * frame_dt [M] (device); counts and randoms in natural angle order (the
 * subset's rows are read in place); bin_factor [Z][A][B] or NULL (n_d = 1);
 * F_model [Z][ny][nx][M] or NULL (prior off; beta ignored).
 * workspace >= kcs_osl_workspace_size bytes (holds rho of one subset). */
size_t kcs_osl_workspace_size(const kcs_geometry_t* g, int n_frames);
int kcs_osl_update(const kcs_geometry_t* g, int subset, int n_frames, const float* frame_dt,
                   float kappa, const float* counts, const float* randoms, int randoms_layout,
                   const float* bin_factor, const float* F_model, float beta_kp, float sigma2,
                   float* x, void* workspace, size_t ws_bytes, void* stream);
/* The two halves of kcs_osl_update, for callers that time or reuse them:
 * kcs_osl_ratio writes rho = s / (kappa dt_m n_d (P_k x)_dm + r_dm) (0 where the
 * denominator is <= 0) to rho [Z][A_k][B][M]; kcs_osl_backproject applies
 * the multiplicative OSL update of x from that rho (Eq. 2-3). */
int kcs_osl_ratio(const kcs_geometry_t* g, int subset, int n_frames, const float* frame_dt,
                  float kappa, const float* counts, const float* randoms, int randoms_layout,
                  const float* bin_factor, const float* x, float* rho, void* stream);
int kcs_osl_backproject(const kcs_geometry_t* g, int subset, int n_frames, const float* frame_dt,
                        float kappa, const float* bin_factor, const float* rho,
                        const float* F_model, float beta_kp, float sigma2, float* x,
                        void* stream);
/* Precision form of the three calls above: counts stored as counts_type, the
 * image x as x_type with per-frame scale x_scale, and the ratio rho (or the
 * workspace holding it) stored as x_type; projections and updates are float32.
 * The split calls also take the row pitch of rho: rho is [Z][A_k][B][rho_frames]
 * with frames 0..n_frames-1 of each row used, rho_frames a multiple of 4 in
 * [n_frames, 256] (n_frames: dense rows, as in the plain calls). */
int kcs_osl_ratio_ex(const kcs_geometry_t* g, int subset, int n_frames, const float* frame_dt,
                     float kappa, const void* counts, int counts_type, const float* randoms,
                     int randoms_layout, const float* bin_factor, const void* x, int x_type,
                     const float* x_scale, void* rho, int rho_frames, void* stream);
int kcs_osl_backproject_ex(const kcs_geometry_t* g, int subset, int n_frames,
                           const float* frame_dt, float kappa, const float* bin_factor,
                           const void* rho, int rho_frames, const float* F_model, float beta_kp,
                           float sigma2, void* x, int x_type, const float* x_scale,
                           void* stream);
/* The row pitch (frames) of the ratio kcs_osl_update keeps in its workspace,
 * and the fastest for the split calls: for KCS_F32 an odd number of 4-frame
 * quads (n_frames + 4 when n_frames / 4 is even), so that the back-projection's
 * 16-byte shared-memory reads of up to 8 consecutive bins hit distinct bank
 * groups; n_frames for 16-bit storage.  Pure function, no GPU work. */
int kcs_osl_rho_frames(int n_frames, int x_type);
int kcs_osl_update_ex(const kcs_geometry_t* g, int subset, int n_frames, const float* frame_dt,
                      float kappa, const void* counts, int counts_type, const float* randoms,
                      int randoms_layout, const float* bin_factor, const float* F_model,
                      float beta_kp, float sigma2, void* x, int x_type, const float* x_scale,
                      void* workspace, size_t ws_bytes, void* stream);
/* Uniform start image per frame: c_m = max(sum(s - r), 0) / (kappa dt_m sum(n P 1)),
 * at least 1e-6, written to every voxel of x [Z][ny][nx][M].
 * workspace >= kcs_osl_workspace_size bytes. */
int kcs_init_image(const kcs_geometry_t* g, int n_frames, const float* frame_dt, float kappa,
                   const float* counts, const float* randoms, int randoms_layout,
                   const float* bin_factor, float* x, void* workspace, size_t ws_bytes,
                   void* stream);
/* Poisson log-likelihood of image x against the counts over all angles, bins
 * and frames (Eq. 1's data term; log s! dropped):
 *   L = sum_{d,m} s_dm log ybar_dm - ybar_dm,  ybar = kappa dt_m n_d (P x) + r
 * (s log ybar taken as 0 where ybar <= 0), accumulated in float64 into *out
 * (device double).  A monitoring metric: one full forward projection.  Storage
 * types as in the precision form; workspace >= 8 KB (e.g. the OSL workspace).
 * The float64 partial sums are added atomically, so the last bits may differ
 * between runs. */
int kcs_loglik(const kcs_geometry_t* g, int n_frames, const float* frame_dt, float kappa,
               const void* counts, int counts_type, const float* randoms, int randoms_layout,
               const float* bin_factor, const void* x, int x_type, const float* x_scale,
               double* out, void* workspace, size_t ws_bytes, void* stream);
/* The per-frame levels c_m of that start image into level [M] (device float),
 * without writing an image: the natural per-frame scale of the precision form
 * (the start image is then stored as exactly 1). */
int kcs_init_level(const kcs_geometry_t* g, int n_frames, const float* frame_dt, float kappa,
                   const void* counts, int counts_type, const float* randoms, int randoms_layout,
                   const float* bin_factor, float* level, void* workspace, size_t ws_bytes,
                   void* stream);
/* Precision form: counts as counts_type; x written as x_type holding c_m / x_scale[m]. */
int kcs_init_image_ex(const kcs_geometry_t* g, int n_frames, const float* frame_dt, float kappa,
                      const void* counts, int counts_type, const float* randoms,
                      int randoms_layout, const float* bin_factor, void* x, int x_type,
                      const float* x_scale, void* workspace, size_t ws_bytes, void* stream);

/* ---------------------------------------------------------- kinetics
 * FDG two-tissue irreversible model with blood fraction (Sec. III-A, IV-A),
 * parameters (K1, k2, k3, Vb), a = k2 + k3, driven by the Feng plasma input
 *   Cp(t) = (A1 t - A2 - A3) e^{-l1 t} + A2 e^{-l2 t} + A3 e^{-l3 t},
 *   F_m = (1/dt_m) int_{frame m} [(1 - Vb) C_T + Vb Cp] dt,
 * evaluated analytically (Sec. II-C).  With a fixed the model is linear in
 * K1, k3, Vb: F_m = (1 - Vb) K1 (A_m(a) + k3 B_m(a)) + Vb cp_m.  This call
 * tabulates A_m, B_m and their a-derivatives once, in float64 on the device,
 * at the nodes of a grid of a (spacing 1/512 per minute), from the exact
 * interval-by-interval convolution (per interval e^{-aD} times a power series
 * in a with non-negative input-moment coefficients), and keeps per grid cell
 * the coefficients of the cubic Hermite interpolants; evaluations read one
 * cell per frame (values within ~2e-7 of each frame's range, slopes within
 * ~5e-6 of the largest slope).
 * t_start, t_end: host arrays of n_frames frame limits (ordered, no overlap;
 * gaps allowed); feng: host {A1, A2, A3, l1, l2, l3}.  Valid for
 * 0 <= k2 + k3 <= 3.75 per minute (the LM box reaches 3).  Synchronous. */
int kcs_create_kinetics(kcs_kinetics_t** out, int n_frames, const double* t_start,
                        const double* t_end, const double* feng, void* stream);
int kcs_destroy_kinetics(kcs_kinetics_t* k);

/* F = model TACs of n_vox voxels: params [4][n_vox] -> F [n_vox][M];
 * J [n_vox][M][4] (d/dK1, d/dk2, d/dk3, d/dVb) when not NULL.  n_vox = 0 is a
 * no-op (the pointers may then be NULL); so for kcs_tac_vjp and kcs_ki. */
int kcs_tac_eval(const kcs_kinetics_t* k, int64_t n_vox, const float* params, float* F,
                 float* J, void* stream);
/* Reverse mode of kcs_tac_eval: gparams[q][v] = sum_m dF_vm/dxi_q * gF[v][m]
 * (the analytic kinetic Jacobian of Sec. II-C transposed), for differentiating
 * y = P F(params) by composing with kcs_back_project.  params [4][n_vox],
 * gF [n_vox][M] -> gparams [4][n_vox] (overwritten). */
int kcs_tac_vjp(const kcs_kinetics_t* k, int64_t n_vox, const float* params, const float* gF,
                float* gparams, void* stream);
/* Ki = K1 k3 / (k2 + k3) (0 where k2 + k3 = 0), Sec. IV-B: [4][n_vox] -> [n_vox]. */
int kcs_ki(int64_t n_vox, const float* params, float* ki, void* stream);

/* ------------------------------------------------------------ MAP-LM (b)
 * Huber gradient dH/dxi_p = sum_{k in N8(v)} clamp(xi_p - xi_{k,p}, -delta, delta)
 * over the in-plane 3x3 clique (Eq. 6, Sec. II-C), per map: [4][Z][ny][nx]. */
int kcs_huber_grad(int nx, int ny, int nz, const float* params, float delta, float* grad,
                   void* stream);
/* The same with a choice of neighbourhood: 8 (the in-plane 3x3 clique above)
 * or 26 (the 3x3x3 cube: a 3D variant the paper does not use; it couples
 * adjacent planes, so plane sharding then needs a one-plane halo). */
int kcs_huber_grad_nb(int nx, int ny, int nz, const float* params, float delta,
                      int neighbourhood, float* grad, void* stream);
/* n_steps synchronous MAP-LM steps (Eq. 4) of every voxel's TAC x [Z][ny][nx][M]:
 *   (J^T J + lambda I) step = J^T (x - F) - beta_h dH/dxi  (float-float Cholesky)
 *   trial = clamp(xi + step, 0, (2, 2, 1, 1)); accept iff the voxel objective
 *   Phi = 1/2 |x - F|^2 + beta_h sum_p sum_{N8} huber(xi_p - xi_{k,p}) falls by
 *   more than tau Phi, with the neighbours frozen at their start-of-step values;
 *   lambda /= 10 (>= 1e-7) on accept, *= 10 (<= 1e7) on reject.
 * The paper gives no acceptance rule: tau = 0 accepts any decrease (equal
 * objectives reject); kcs_map_lm_fit and kcs_map_lm_fit_ex use the sufficient-
 * decrease threshold tau = KCS_LM_TAU_DEFAULT, kcs_map_lm_fit_nb takes tau.
 * params [4][Z][ny][nx] in/out; lambda [Z][ny][nx] in/out, or NULL to start
 * every voxel at 1e-2; F_out [Z][ny][nx][M] receives F(final params) when not
 * NULL.  workspace >= kcs_lm_workspace_size(nx, ny, nz) bytes. */
#define KCS_LM_TAU_DEFAULT 1e-5f
size_t kcs_lm_workspace_size(int nx, int ny, int nz);
int kcs_map_lm_fit(const kcs_kinetics_t* k, int nx, int ny, int nz, const float* x,
                   float* params, float* lambda, int n_steps, float beta_h, float delta,
                   float* F_out, void* workspace, size_t ws_bytes, void* stream);
/* Precision form: the image TACs x stored as x_type (KCS_F32/BF16/F16) with
 * per-frame scale x_scale [M] (NULL = 1); the fit itself is unchanged (float32
 * model, float-float 4x4 solve). */
int kcs_map_lm_fit_ex(const kcs_kinetics_t* k, int nx, int ny, int nz, const void* x,
                      int x_type, const float* x_scale, float* params, float* lambda,
                      int n_steps, float beta_h, float delta, float* F_out, void* workspace,
                      size_t ws_bytes, void* stream);
/* kcs_map_lm_fit_ex with the Huber neighbourhood as in kcs_huber_grad_nb
 * (8 or 26) and the acceptance threshold tau in [0, 1) (KCS_ERR_INVALID_ARG
 * otherwise). */
int kcs_map_lm_fit_nb(const kcs_kinetics_t* k, int nx, int ny, int nz, const void* x,
                      int x_type, const float* x_scale, float* params, float* lambda,
                      int n_steps, float beta_h, float delta, int neighbourhood, float tau,
                      float* F_out, void* workspace, size_t ws_bytes, void* stream);

/* ------------------------------------------------- MAP-LM without allocation
 * The paper has no counterpart to this entry point; it exists for callers that
 * cannot allocate device memory: an application that owns all device memory
 * through its own pool and forbids raw allocations by plug-ins, or a service
 * that must not allocate after start-up.  It is kcs_map_lm_fit with the
 * workspace replaced by a fixed array inside the library (about 10 MB, held on
 * every GPU that loads the library until the process exits), so it takes no
 * workspace argument and never allocates.
 *  - At most KCS_LM_STATIC_MAX_VOXELS voxels (nx*ny*nz); larger problems are
 *    rejected with KCS_ERR_INVALID_ARG and a message (use kcs_map_lm_fit).
 *  - The first call on a device looks up the array's device address with that
 *    device current; make that first call before any stream capture.
 *  - The stream (if not NULL) must belong to the current device: the array's
 *    address differs per device, so a stream of another device is rejected
 *    with KCS_ERR_INVALID_ARG.
 *  - Every call on a device shares the one array: calls whose work overlaps on
 *    the GPU (different streams, or host threads without ordering) race and
 *    corrupt each other; serialise them.  Nothing in the array needs to start at
 *    zero (each step writes what it later reads).
 * Arguments as for kcs_map_lm_fit. */
#define KCS_LM_STATIC_MAX_VOXELS 65536
int kcs_map_lm_fit_static(const kcs_kinetics_t* k, int nx, int ny, int nz, const float* x,
                          float* params, float* lambda, int n_steps, float beta_h, float delta,
                          float* F_out, void* stream);

/* ------------------------------------------------------- measurement
 * Arithmetic peak probe (not part of the method): launches blocks x 256
 * threads that each advance 16 independent multiply-add chains iters times in
 * float32 (precision = 32, FFMA) or float64 (precision = 64, DFMA), on stream;
 * *flops receives the number of floating-point operations the launch performs
 * (a multiply-add counts 2).  The caller times the launch with CUDA events:
 * flops / time is the measured FFMA or DFMA rate of the GPU, the denominator of
 * a kernel's fraction of arithmetic peak.  sink: device buffer of at least
 * 8 x blocks bytes (never written for the chains' values).  Asynchronous. */
int kcs_fma_peak_launch(int precision, int blocks, int iters, double* flops, void* sink,
                        void* stream);

/* Device-side failure detection: the number of bounded waits inside the
 * library's kernels (bulk-copy completion barriers) that ran out instead of
 * completing, summed over the process on the current device.  A timed-out
 * kernel skips the rest of its work rather than hanging.  Synchronous (reads a
 * device counter); returns KCS_ERR_TIMEOUT if the count is non-zero. */
int kcs_device_status(unsigned int* wait_timeouts);
/* Reset that counter to zero (synchronous). */
int kcs_device_status_reset(void);
/* Self-test of the failure path: one kernel waits, with at most spin_limit
 * polls (1 .. 2^20), on a barrier that nothing completes, so the wait runs
 * out and the counter read by kcs_device_status rises by one.  No fault, no
 * hang; the context stays usable. */
int kcs_selftest_wait_timeout(int spin_limit, void* stream);

/* --------------------------------------------------------------- ICM
 * A study binds a geometry, a kinetics table and the caller's device buffers;
 * kcs_icm_iterate runs Sec. II-D's alternation on it, all on one stream:
 *   for each iteration: one OSL pass over subsets 0..S-1 (prior built from
 *   F = F(params) when an earlier iteration ran or params_given is set),
 *   then n_lm MAP-LM steps warm-started from params (lambda reset to 1e-2),
 *   then F <- F(params).
 * x must hold a start image (e.g. from kcs_init_image); params must hold the
 * start maps. */
typedef struct kcs_study_desc {
  const kcs_geometry_t* geom;
  const kcs_kinetics_t* kin;
  int n_frames;
  float kappa;             /* count calibration: counts per (activity . mm . min) */
  const float* frame_dt;   /* [M] device                                      */
  const void* counts;      /* [Z][A][B][M], counts_type                       */
  const float* randoms;    /* see randoms_layout                              */
  int randoms_layout;
  const float* bin_factor; /* [Z][A][B] or NULL                               */
  void* x;                 /* [Z][ny][nx][M] in/out, x_type                   */
  float* params;           /* [4][Z][ny][nx] in/out                           */
  float* F;                /* [Z][ny][nx][M] out (model TACs of params)       */
  int params_given;        /* nonzero: prior on from the first iteration      */
  int n_lm;                /* MAP-LM steps per iteration                      */
  float beta_kp, sigma2;   /* kinetics-derived prior (Eq. 3)                  */
  float beta_h, delta;     /* Huber prior (Eq. 4-6)                           */
  void* workspace;         /* >= kcs_study_workspace_size bytes               */
  size_t ws_bytes;
  /* precision form (zero-initialised = float32 everywhere): counts stored as
   * counts_type (KCS_F32 / KCS_U16), x and the ratio as x_type (KCS_F32 /
   * KCS_BF16 / KCS_F16) with per-frame scale x_scale [M] (device, NULL = 1). */
  int counts_type;
  int x_type;
  const float* x_scale;
  /* reconstruction method (Sec. IV-A; zero-initialised = KCS):
   *   KCS_METHOD_KCS      the ICM above (kinetics prior + Huber MAP-LM),
   *   KCS_METHOD_DIRECT   the same without the spatial prior (beta_h taken as 0),
   *   KCS_METHOD_INDIRECT each iteration is an OSEM pass (no prior, no fit);
   *                       the kinetic fit runs once, after the reconstruction,
   *                       in kcs_study_fit (post-reconstruction fitting). */
  int method;
  /* Huber neighbourhood of the fit: 0 or 8 = in-plane 3x3 (Sec. II-C), 26 = 3x3x3 */
  int neighbourhood;
  /* MAP-LM acceptance threshold (see kcs_map_lm_fit_nb): lm_tau when
   * lm_tau_given is nonzero, else KCS_LM_TAU_DEFAULT. */
  float lm_tau;
  int lm_tau_given;
} kcs_study_desc_t;

enum { KCS_METHOD_KCS = 0, KCS_METHOD_DIRECT = 1, KCS_METHOD_INDIRECT = 2 };

size_t kcs_study_workspace_size(const kcs_geometry_t* g, int n_frames);
int kcs_create_study(kcs_study_t** out, const kcs_study_desc_t* desc);
int kcs_destroy_study(kcs_study_t* st);
/* Run n_iter ICM iterations (asynchronous on stream). */
int kcs_icm_iterate(kcs_study_t* st, int n_iter, void* stream);
/* kcs_icm_iterate with host I/O for streaming a study through the GPU:
 * before each iteration the counts are copied from counts_host (pinned host
 * memory holding the study's counts in their layout and type; NULL: no
 * copy) into the study's counts buffer, and after each iteration the maps are
 * copied to params_host + k * params_host_stride floats (pinned host memory,
 * [4][Z][ny][nx] per iteration; stride 0 overwrites one block, otherwise the
 * stride is >= 4 x voxels; NULL: no copy).  The copies run on a private
 * stream and overlap the compute: iteration k+1's counts arrive during
 * iteration k's MAP-LM steps (which do not read the counts), iteration k's
 * maps leave during iteration k+1's OSL pass (which does not touch them).
 * When the rows of a subset are every S-th sinogram row of the volume (the
 * angle count a multiple of S, or a single plane), the first iteration's
 * counts come in by one strided copy per subset and its OSL pass waits only
 * for each subset's own rows.  Results equal kcs_icm_iterate's bit for bit.  Asynchronous: the caller's
 * stream completes after the last copy; the host buffers must stay valid
 * until then.  Host-issued (no graph replay). */
int kcs_icm_iterate_host(kcs_study_t* st, int n_iter, const void* counts_host,
                         float* params_host, size_t params_host_stride, void* stream);
/* Replay the steady-state ICM iteration (prior on) from a CUDA graph recorded
 * at its first use (enable = 1), or issue every launch from the host (enable =
 * 0, the default; also releases a recorded graph).  Results are identical;
 * the graph removes per-launch host cost (Sec. II-D loop, small studies).  The
 * graph is recorded on a private stream and launched on the caller's stream. */
int kcs_study_set_graph(kcs_study_t* st, int enable);
/* n_steps MAP-LM steps on the study's current image from its current maps
 * (lambda reset to 1e-2), then F <- F(params): the post-reconstruction fit of
 * KCS_METHOD_INDIRECT (beta_h taken as 0 for INDIRECT and DIRECT).
 * Asynchronous on stream. */
int kcs_study_fit(kcs_study_t* st, int n_steps, void* stream);
/* Number of ICM iterations issued so far on this study. */
int kcs_study_iterations(const kcs_study_t* st);
/* Set that number, e.g. when resuming from a checkpoint of x, params and F:
 * the next iteration then builds its prior from F as the interrupted run
 * would have. */
int kcs_study_set_iterations(kcs_study_t* st, int iterations);

#ifdef __cplusplus
}
#endif
#endif /* KCS_H */
