/*
 * mslice.h -- C ABI of libmslice: the reflection-geometry multislice forward
 * model of Coherent Surface Scattering Imaging (arxiv 2212.01253) and its
 * gradient, on one NVIDIA GB300 (sm_103a).
 *
 * Physics (paper notation):
 *   Eq. 1 (Sec. 1)  one slice of thickness Delta:
 *       phi(Z0+Delta) = F^-1{ exp(-i Delta (kX^2+kY^2)/2k) F{ exp((k/2i) int (1-n^2) dZ) phi(Z0) } }
 *     implemented with n = 1 - delta + i beta, the linearised 1-n^2 ~ 2(delta - i beta),
 *     one voxel per slice, so the transmission is t = exp(-i k Delta (delta - i beta)),
 *     and without the global phase exp(i k Delta).
 *   Fig. 1a: the exit wave of the last slice is Fourier transformed and squared:
 *     I = |Psi|^2, Psi = F_unitary(t_Ns * phi_{Ns-1}) (the last propagation and the
 *     free propagation to the detector are pure Fourier phases and are skipped).
 *   Eq. 4 (Sec. 4.1): the loss is the squared error of amplitudes; this library
 *     sums it (no 1/N): L = sum (sqrt(s I) - m)^2, m = sqrt(I_meas).
 *   Sec. 2, Eq. 2-3: the incidence angle alpha_i and the in-plane angle psi of
 *     each wavefield (view) are applied by tilting its probe, phi_0(y, z) =
 *     exp(-i k (sin(alpha_i) z + sin(psi) y)) (toward the substrate for
 *     alpha_i > 0), instead of rotating the volume (paraxially equivalent).
 *
 * Axes and layouts (all arrays row-major, last index fastest):
 *   x  = slice index along the beam, ns slices of thickness slice_nm (Delta);
 *   z  = surface normal, nz pixels of dz_nm, z index 0 = bottom (substrate side);
 *   y  = in-plane transverse axis, ny pixels of dy_nm.
 *   A complex value is two floats (re, im).  The volume holds delta + i*beta.
 *   Frequencies: k_y = 2 pi fftfreq(ny, dy), k_z = 2 pi fftfreq(nz, dz); forward DFT
 *   kernel exp(-i ...); detector images are in natural (unshifted) FFT order.
 *
 * Memory and streams:
 *   Every pointer argument except `p` is a DEVICE pointer owned by the caller.
 *   The library allocates no device memory: scratch lives in the caller's
 *   workspace `ws` (size from mslice_workspace_size(), 256-byte aligned; its
 *   contents need no initialisation and are clobbered).  All work is enqueued on
 *   `stream` (a cudaStream_t, NULL = legacy default stream) and is asynchronous;
 *   outputs are valid once the stream reaches them.  Outputs must not alias
 *   inputs or the workspace.  Calls sharing one workspace must not overlap.
 *   The one exception is mslice_forward_static(), whose workspace is a fixed
 *   device array owned by the library itself (declared below).
 *
 * Errors: functions return MSLICE_OK (0) or a negative MSLICE_E* code; they never
 * abort or trap.  Device-side waits are bounded: a wait that runs out marks the
 * workspace's status word; mslice_status() reports it as MSLICE_ETIMEDOUT.
 */
#ifndef MSLICE_H
#define MSLICE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define MSLICE_MAX_ANGLES 64
#define MSLICE_MAX_N 1024

/* return codes */
#define MSLICE_OK 0
#define MSLICE_EINVAL (-1)        /* bad size, pointer, alignment or parameter */
#define MSLICE_EUNSUPPORTED (-2)  /* valid request outside what is built */
#define MSLICE_ELAUNCH (-3)       /* a CUDA launch or runtime call failed */
#define MSLICE_ETIMEDOUT (-4)     /* a bounded device-side wait ran out */
#define MSLICE_EWORKSPACE (-5)    /* workspace smaller than mslice_workspace_size() */

/* ops for mslice_workspace_size */
#define MSLICE_OP_FORWARD 0
#define MSLICE_OP_ADJOINT 1
#define MSLICE_OP_LOSS_GRAD 2

/* flags */
#define MSLICE_EXIT_WAVE 1u  /* forward: field_out = phi_Ns (after the full last
                                propagation) and intensity = |phi_Ns|^2 instead of
                                the far field; used for near-field checks */
#define MSLICE_PER_STRUCTURE 2u  /* wavefield w propagates through its own volume:
                                    vol and grad_vol are [nw][ns][nz][ny] (nw
                                    independent structures of one grid shape,
                                    each with its own incidence angle) */
#define MSLICE_EXACT_TRANSMISSION 4u  /* Eq. 1 with the exact 1 - n^2 = 2w - w^2,
                                         w = delta - i beta: t = exp(-i k Delta
                                         (w - w^2/2)) instead of the linearised
                                         exp(-i k Delta w); the gradient follows
                                         (d log t / dw = -i k Delta (1 - w)) */
#define MSLICE_ANGULAR 16u  /* angular-spectrum propagator instead of the
                               paraxial Fresnel one of Eq. 1:
                               exp(i Delta (sqrt(k^2 - k_y^2 - k_z^2) - k)), and
                               exp(-Delta sqrt(k_perp^2 - k^2)) exp(-i Delta k)
                               for evanescent k_perp > k.  Not separable: the
                               field is kept in (k_y, z) space between a row
                               and a column pass per slice (two grid barriers
                               per slice).  Combines with MSLICE_EXIT_WAVE and
                               MSLICE_STRANG (half steps over Delta/2 of the
                               same propagator). */
#define MSLICE_STRANG 8u  /* symmetric splitting of Eq. 1's slice step: half a
                             step of free propagation (Delta/2) before the first
                             slice; with MSLICE_EXIT_WAVE the last propagation is
                             a half step too.  The far field omits that final half
                             step (a unit-modulus phase on the detector), so I,
                             the loss and the gradient are those of the default
                             transmission-first loop started from
                             F^-1 P(Delta/2) F phi_0.  Second order in Delta
                             over slices of uniform content; the default is
                             first order.  Costs one extra slice-loop launch. */

typedef struct mslice_params {
    double wavelength_nm;      /* lambda; k = 2 pi / lambda is formed in FP64 */
    double slice_nm;           /* Delta: slice thickness along the beam */
    double dy_nm;              /* pixel size along y */
    double dz_nm;              /* pixel size along z (surface normal) */
    int32_t ny, nz;            /* powers of two in [1, MSLICE_MAX_N] */
    int32_t ns;                /* number of slices, >= 1 */
    int32_t nw;                /* number of wavefields (incidence angles), 1..MSLICE_MAX_ANGLES */
    double alpha_i_rad[MSLICE_MAX_ANGLES]; /* incidence angle of each wavefield */
    double psi_rad[MSLICE_MAX_ANGLES]; /* in-plane (yaw) angle of each wavefield's beam, |psi| < 0.1
                                  rad: the default probe of wavefield w carries the phase
                                  exp(-i k sin(psi_w) y) (user probes are used as given) */
    int32_t checkpoint_every;  /* adjoint segment length in slices; <= 0 means 32 */
    uint32_t flags;            /* MSLICE_EXIT_WAVE, MSLICE_PER_STRUCTURE, MSLICE_EXACT_TRANSMISSION,
                                  MSLICE_STRANG, MSLICE_ANGULAR */
    int32_t grid_blocks;       /* launch shape: blocks of the persistent kernels, 0 = automatic
                                  (capped at the co-resident maximum) */
    int32_t col_width;         /* launch shape: columns per column-pass group (4, 8 or 16),
                                  0 = automatic; see mslice_autotune in the Python package */
    int32_t schedule;          /* schedule of the angular-spectrum slice loop (MSLICE_ANGULAR, two
                                  passes per slice): 0 = automatic (= 1), 1 = one grid barrier
                                  after each pass, 2 = the wavefields in two groups whose passes
                                  alternate with split-phase barriers (nw >= 2; results are
                                  bitwise identical to 1).  The paraxial slice loop runs one
                                  pass per slice, alternating between rows and columns, with one
                                  grid barrier per slice, and ignores this field. */
} mslice_params;

/* Bytes of workspace needed by `op` (MSLICE_OP_*) for these parameters;
 * 0 if the parameters are invalid. */
size_t mslice_workspace_size(const mslice_params *p, int op);

/* Forward model (Eq. 1 slice loop, then the far field of Fig. 1a).
 *   vol        [ns][nz][ny] complex: delta + i beta of each voxel (read only, 16-byte aligned)
 *   probe      NULL for the tilted unit plane wave exp(-i k sin(alpha_w) z_l),
 *              or [nw][nz][ny] complex user probe phi_0 (Sec. 5: any probe shape)
 *   intensity  [nw][nz][ny] float: I = |Psi|^2 (may be NULL)
 *   field_out  NULL or [nw][nz][ny] complex: Psi (or phi_Ns with MSLICE_EXIT_WAVE) */
int mslice_forward(const mslice_params *p, const float *vol, const float *probe,
                   float *intensity, float *field_out, void *ws, size_t ws_bytes,
                   void *stream);

/* mslice_forward without a caller workspace and without any allocation.  The
 * paper has no counterpart: this entry point is for callers that cannot
 * allocate device memory -- code running while a foreign framework captures a
 * CUDA graph (where a cudaMalloc would break the capture), or real-time and
 * plugin hosts whose device allocator is off limits to them.  The workspace is
 * a fixed 32 MiB device array inside the library (every GPU that loads the
 * library holds it until the process exits); parameters whose forward
 * workspace (mslice_workspace_size(p, MSLICE_OP_FORWARD)) exceeds 32 MiB are
 * rejected with MSLICE_EWORKSPACE (32 MiB covers e.g. 512x512 x 14 slices or
 * 256x256 x 60 slices).  The first call on a device looks up the array's
 * device address (cudaGetSymbolAddress, with that device current); make that
 * first call before any stream capture.  The looked-up address is kept for
 * the life of the process: after a cudaDeviceReset of that device, or an
 * unload and reload of the library, it is stale, and the library must be
 * reloaded.  Device indices of 64 and above get MSLICE_EUNSUPPORTED.  Every
 * call shares the one array and leaves its last contents there (the control
 * words are cleared at the start of each call): calls that overlap on the
 * GPU -- on different streams, or from different host threads -- race and
 * must not be issued.  Other arguments and errors as for mslice_forward. */
int mslice_forward_static(const mslice_params *p, const float *vol, const float *probe,
                          float *intensity, float *field_out, void *stream);

/* mslice_status() for the library-owned workspace of mslice_forward_static on
 * the current device: waits for `stream`, then returns MSLICE_OK, or
 * MSLICE_ETIMEDOUT if a bounded device-side wait of the last static call ran
 * out (its intensities are then not valid).  Allocates nothing. */
int mslice_forward_static_status(void *stream);

/* Gradient of a real loss through the forward model, for a given detector
 * gradient (replaces the autograd backward of Sec. 3-4).
 *   g_psi      [nw][nz][ny] complex: dL/dRe(Psi) + i dL/dIm(Psi)
 *   grad_vol   [ns][nz][ny] complex out: dL/ddelta + i dL/dbeta, summed over
 *              wavefields.  Slice checkpoints every checkpoint_every slices are
 *              kept in the workspace and segments are recomputed. */
int mslice_adjoint(const mslice_params *p, const float *vol, const float *probe,
                   const float *g_psi, float *grad_vol, void *ws, size_t ws_bytes,
                   void *stream);

/* Amplitude loss of Eq. 4 (summed) and its gradient on delta/beta.
 *   meas_amp   [nw][nz][ny] float: m = sqrt(I_meas)
 *   scale      s > 0: model intensity scale (photon flux)
 *   loss_out   device double[1]: L = sum_w sum_px (sqrt(s I) - m)^2 (FP64 sum)
 *   grad_vol   [ns][nz][ny] complex out, as for mslice_adjoint
 *   intensity  NULL or [nw][nz][ny] float out: I of the model */
int mslice_loss_grad(const mslice_params *p, const float *vol, const float *probe,
                     const float *meas_amp, float scale, double *loss_out, float *grad_vol,
                     float *intensity, void *ws, size_t ws_bytes, void *stream);

/* Loss and gradient of nw independent structures of one grid shape, advanced
 * together (flag MSLICE_PER_STRUCTURE is implied):
 *   vols       [nw][ns][nz][ny] complex, one volume per structure
 *   meas_amp   [nw][nz][ny] float, scales: host float[nw] (s of each structure)
 *   loss_out   device double[1]: sum over the structures
 *   grad_vol   [nw][ns][nz][ny] complex out, one gradient per structure
 * Workspace: mslice_workspace_size(p with the flag set, MSLICE_OP_LOSS_GRAD). */
int mslice_loss_grad_multi(const mslice_params *p, const float *vols, const float *probe,
                           const float *meas_amp, const float *scales, double *loss_out,
                           float *grad_vol, float *intensity, void *ws, size_t ws_bytes,
                           void *stream);

/* ------------------------------------------------------------------------
 * Batched runs of many independent structures of uneven grid shape (the
 * paper's forward model of Eq. 1 and the loss of Eq. 4, for many samples at
 * once; the batching itself has no counterpart in the paper).  Jobs of one
 * grid shape (ny, nz, ns) advance together as the wavefields of one
 * per-structure run (up to MSLICE_MAX_ANGLES per run); the runs ("groups") are
 * spread over `lanes` library-owned streams, forked from and joined back into
 * `stream`: longest first (work = voxels x slices x structures, or for slice
 * loops of little work the number of slices) onto the least loaded lane, each
 * group on the blocks its row and column tasks fill (one task per warp), at
 * most half the SMs.  With lanes == 1 every group runs on the default grid,
 * one after the other.  Lanes beyond the process's hardware work queues
 * (CUDA_DEVICE_MAX_CONNECTIONS, 8 unless set before the CUDA context is
 * created) share queues and partly serialise.
 * Every job's results are bitwise those of a single-structure call with the
 * same launch shape.
 * ------------------------------------------------------------------------ */
typedef struct mslice_job {
    int32_t ny, nz, ns;        /* grid of this structure: powers of two in [1, MSLICE_MAX_N], ns >= 1 */
    int32_t col_width;         /* launch shape of this job's group (the group takes its first job's):
                                  columns per column-pass group, 0 = automatic */
    double alpha_i_rad;        /* incidence angle */
    double psi_rad;            /* in-plane angle (|psi| < 0.1 rad), as psi_rad of mslice_params */
    float scale;               /* s > 0: model intensity scale of the loss (loss + gradient only) */
    float reserved;            /* 0 */
    const float *vol;          /* [ns][nz][ny] complex delta + i beta, device, 16-byte aligned */
    const float *meas_amp;     /* [nz][ny] float sqrt(I_meas), device (loss + gradient only) */
    float *grad_vol;           /* [ns][nz][ny] complex out: dL/ddelta + i dL/dbeta (loss + gradient) */
    float *intensity;          /* [nz][ny] float out: I (required by the forward; may be NULL otherwise) */
    double *loss_out;          /* device double[1] out: this job's loss, or NULL (loss + gradient) */
} mslice_job;

/* Bytes of workspace of a batched call (op MSLICE_OP_FORWARD or
 * MSLICE_OP_LOSS_GRAD) for these jobs and lanes; 0 if the request is invalid.
 * `common` gives the wavelength, slice thickness, pixel sizes, checkpoint
 * interval, flags (MSLICE_EXACT_TRANSMISSION, MSLICE_STRANG;
 * MSLICE_EXIT_WAVE for the forward) and grid_blocks (used when lanes == 1);
 * its ny, nz, ns, nw, alpha_i_rad and psi_rad are ignored (every job has its
 * own grid and angles). */
size_t mslice_batched_workspace_size(const mslice_params *common, const mslice_job *jobs, int njobs, int op,
                                     int lanes);

/* Loss and gradient of every job: jobs[i].grad_vol, jobs[i].loss_out (if
 * given) and jobs[i].intensity (if given); loss_total: NULL or device
 * double[1], the sum of the jobs' losses (FP64, summed per group in job order
 * and over the groups in order).  1 <= lanes <= 16.  The lane streams and
 * events are created on the first call with lanes > 1 on a device: make that
 * call before any stream capture.  Calls that share the workspace, or that
 * run with lanes > 1 at the same time on one device, must not overlap.
 * Errors: MSLICE_EINVAL (a bad job, pointer, alignment or lane count),
 * MSLICE_EUNSUPPORTED (MSLICE_ANGULAR, or MSLICE_EXIT_WAVE), MSLICE_EWORKSPACE,
 * MSLICE_ELAUNCH. */
int mslice_loss_grad_batched(const mslice_params *common, const mslice_job *jobs, int njobs, int lanes,
                             double *loss_total, void *ws, size_t ws_bytes, void *stream);

/* The plan of a batched call, on the host (no device work): *ngroups, and
 * for every job its group (group_of_job[njobs], may be NULL), for every group
 * its lane (lane_of_group[ngroups], may be NULL; at most njobs groups) and the
 * blocks of its persistent grid (blocks_of_group[ngroups], may be NULL; 0 =
 * the default grid, lanes == 1).  The SM count is the current device's (152
 * when no device can be queried).
 * Groups are numbered in order of their first job; a group holds the jobs of
 * one grid shape (ny, nz, ns), at most MSLICE_MAX_ANGLES, in job order. */
int mslice_batched_plan(const mslice_params *common, const mslice_job *jobs, int njobs, int op, int lanes,
                        int *group_of_job, int *lane_of_group, int *blocks_of_group, int *ngroups);

/* mslice_status() of every group of a batched call (same jobs, op and lanes):
 * waits for `stream`, then MSLICE_OK, or MSLICE_ETIMEDOUT if a bounded
 * device-side wait of any group ran out. */
int mslice_batched_status(const mslice_params *common, const mslice_job *jobs, int njobs, int op, int lanes,
                          const void *ws, void *stream);

/* Far-field intensity of every job into jobs[i].intensity (the exit wave's
 * with MSLICE_EXIT_WAVE).  Arguments and errors as for
 * mslice_loss_grad_batched. */
int mslice_forward_batched(const mslice_params *common, const mslice_job *jobs, int njobs, int lanes, void *ws,
                           size_t ws_bytes, void *stream);

/* The FP64-built constant arrays ("C" of Fig. 1), rounded to float:
 *   py [ny] complex: exp(-i Delta k_y^2 / 2k);  pz [nz] complex: exp(-i Delta k_z^2 / 2k)
 *   probe_z [nw][nz] complex: exp(-i k sin(alpha_w) z_l) (default probe, one value per row)
 * Any output may be NULL.  Uses the workspace of MSLICE_OP_FORWARD. */
int mslice_plan_tables(const mslice_params *p, float *py, float *pz, float *probe_z,
                       void *ws, size_t ws_bytes, void *stream);

/* Transmission of every voxel (Eq. 1 first factor): t = exp(-i k Delta (delta - i beta)),
 * phase arguments k*Delta*delta and k*Delta*beta formed in FP64.
 *   vol [ns][nz][ny] complex in;  t_out [ns][nz][ny] complex out.  No workspace. */
int mslice_transmission(const mslice_params *p, const float *vol, float *t_out, void *stream);

/* Vector-Jacobian product of the detector intensity I = |Psi|^2 (Fig. 1a):
 * g_psi[i] = 2 dI[i] Psi[i], the detector gradient (dL/dRe + i dL/dIm) that
 * mslice_adjoint() takes when the loss is a function of I.  n complex
 * elements; psi, g_psi complex, dI float; no workspace. */
int mslice_intensity_vjp(const float *psi, const float *dI, float *g_psi, size_t n, void *stream);

/* Waits for `stream`, then reads the workspace status word: MSLICE_OK, or
 * MSLICE_ETIMEDOUT if a device-side wait of an earlier call ran out. */
int mslice_status(const void *ws, void *stream);

/* Test hook for the bounded grid wait: launches `nblocks` cooperating blocks
 * that wait for nblocks + withhold arrivals with a limit of timeout_ns.  With
 * withhold > 0 nobody ever completes the wait, every block gives up after the
 * limit and the status word records MSLICE_ETIMEDOUT.  ws >= 4096 bytes. */
int mslice_debug_wait(int nblocks, int withhold, long long timeout_ns, void *ws,
                      size_t ws_bytes, void *stream);

/* ------------------------------------------------------------------------
 * Reconstruction helpers (Sec. 4: coarse reconstruction voxels mapped onto the
 * finer multislice grid, optimised with ADAM).
 * ------------------------------------------------------------------------ */

/* Coarse parameter grid: theta[cx][cz][cy] (real delta of each coarse voxel)
 * maps onto the block of the fine volume starting at slice x0, row z0,
 * column y0, each coarse voxel covering bx slices x bz rows x by columns.
 * The fine voxel gets delta = theta and beta = beta_ratio * theta (one
 * material with a fixed beta/delta ratio); voxels outside the block are not
 * touched.  Sec. 4.1 and 4.2 use coarse voxels elongated along the beam. */
typedef struct mslice_coarse {
    int32_t cx, cz, cy;      /* coarse grid */
    int32_t bx, bz, by;      /* block size in fine voxels */
    int32_t x0, z0, y0;      /* fine-grid offset of the block */
    float beta_ratio;        /* d beta / d theta: the material's beta / delta (or the
                                ratio of the differences for two materials) */
    float base_delta;        /* delta + i beta of the block at theta = 0: 0 for voxels */
    float base_beta;         /*   that are vacuum or material, the host material's index for
                                inclusions buried in it (Sec. 4.1, Au in Si) */
} mslice_coarse;

/* vol[x0 + bx*a + i][z0 + bz*b + k][y0 + by*c + l]
 *     = (base_delta + theta[a][b][c]) + i (base_beta + beta_ratio theta[a][b][c]).
 * theta float [cx][cz][cy]; vol complex [ns][nz][ny] (p gives ns, nz, ny). */
int mslice_coarse_to_fine(const mslice_params *p, const mslice_coarse *c, const float *theta,
                          float *vol, void *stream);

/* Adjoint of mslice_coarse_to_fine on a gradient grad_vol = dL/ddelta + i dL/dbeta:
 * g_theta[a][b][c] = sum over the block of (dL/ddelta + beta_ratio dL/dbeta).
 * Each coarse voxel is summed by one thread in a fixed order (deterministic). */
int mslice_fine_to_coarse(const mslice_params *p, const mslice_coarse *c, const float *grad_vol,
                          float *g_theta, void *stream);

/* Material snapping of the coarse parameters (Sec. 4.1: after every 20 epochs
 * each voxel is replaced by the nearest of the refractive indexes of interest):
 * theta[i] = the level nearest to theta[i] (the lower one on a tie), for
 * 1 <= nlevels <= 8 levels given in host memory; n parameters, in place. */
int mslice_snap(float *theta, size_t n, const float *levels, int nlevels, void *stream);

/* Shrink-wrap support update (Sec. 4.2, after Marchesini et al. 2003: every
 * twenty epochs, also a nearest-neighbour filter between material and air)
 * on a coarse parameter grid theta[cx][cz][cy], device memory, in place:
 *   blur    = theta convolved with a normalised Gaussian of width sigma coarse
 *             voxels, separably along y, then z, then x; taps t = -r..r,
 *             r = floor(3 sigma + 0.5) <= 16 (else MSLICE_EUNSUPPORTED); zero
 *             outside the grid;
 *   support = blur >= threshold * max(blur), 0 <= threshold <= 1;
 *   theta   = 0 outside the support (air, or the host of a buried pattern).
 * The blur takes its taps in order with FP32 products and sums rounded one by
 * one (no fused multiply-add), so the support is reproducible bit for bit.
 * kept: NULL or a device int that receives the support's size.  ws: device
 * workspace, 16-byte aligned, of mslice_shrinkwrap_workspace(cx*cz*cy) bytes,
 * owned by the caller.  Returns MSLICE_EINVAL for a null theta or ws, a
 * non-positive grid size or sigma, a threshold outside [0, 1] or a short or
 * misaligned workspace; MSLICE_ELAUNCH when a launch fails. */
size_t mslice_shrinkwrap_workspace(size_t n);
int mslice_shrinkwrap(float *theta, int cx, int cz, int cy, float sigma, float threshold, int *kept, void *ws,
                      size_t ws_bytes, void *stream);

/* One ADAM step (Kingma & Ba, cited in Sec. 4.1) on n parameters, in place:
 *   m = b1 m + (1-b1) g;  v = b2 v + (1-b2) g^2;
 *   theta -= lr * (m / (1-b1^t)) / (sqrt(v / (1-b2^t)) + eps);  theta = clamp(theta, lo, hi)
 * t >= 1 is the step number; m and v start at 0. */
int mslice_adam_step(float *theta, float *m, float *v, const float *grad, size_t n, float lr,
                     float b1, float b2, float eps, int t, float lo, float hi, void *stream);

/* ------------------------------------------------------------------------
 * Frame rotation (Eq. 2-3): the paper simulates in the lab frame, rotating
 * the index volume by a pitch of alpha_i after a yaw of psi so that a straight
 * beam meets it.  The slice loops above work in the sample frame with a
 * tilted probe instead (the paraxially equivalent form); these calls build
 * the lab-frame volume for the paper's formulation and map lab-frame
 * gradients back.
 *
 * Axes (x, z, y) with x = j slice_nm, z = l dz_nm, y = m dy_nm; both volumes
 * are [ns][nz][ny] complex64 on that lattice (ns, nz, ny and the spacings
 * come from p; its other fields are ignored, and ny, nz need not be powers
 * of two here).  With M = R_pitch(alpha) R_yaw(psi),
 *   R_pitch: x' = cos(a) x - sin(a) z,  z' = sin(a) x + cos(a) z
 *   R_yaw:   x' = cos(p) x - sin(p) y,  y' = sin(p) x + cos(p) y
 * the lab voxel at r takes the sample volume at s = c + M^T (r - c), c the
 * rotation centre center_nm[3] = (x, z, y) in host memory: the surface rises
 * by tan(alpha) along +x and a feature drifts toward +y by tan(psi).
 * Trilinear interpolation in index units, each index clamped to [0, n-1]
 * (the volume extends past its faces by its edge values).
 * ------------------------------------------------------------------------ */

/* vol_lab = R vol_sample.  Device buffers owned by the caller, 8-byte
 * aligned, not aliased; asynchronous on stream.  Returns MSLICE_EINVAL for a
 * null or misaligned pointer, vol_sample == vol_lab, a non-positive spacing,
 * a size outside [1, MSLICE_MAX_N] across the beam or ns < 1, or a non-finite
 * angle or centre; MSLICE_EUNSUPPORTED when ns * nz >= 2^31 or a sample
 * index would leave +-2^30; MSLICE_ELAUNCH when the launch fails. */
int mslice_rotate(const mslice_params *p, double alpha_rad, double psi_rad, const double *center_nm,
                  const float *vol_sample, float *vol_lab, void *stream);

/* g_sample = R^T g_lab (overwritten): the lab-frame gradient gathered back
 * with the interpolation weights.  Every sample voxel sums the lab voxels
 * whose stencils touch it in a fixed order, each stencil computed as
 * mslice_rotate computes it, so the result is bitwise reproducible (no
 * atomics).  Buffers and errors as for mslice_rotate. */
int mslice_rotate_adjoint(const mslice_params *p, double alpha_rad, double psi_rad, const double *center_nm,
                          const float *g_lab, float *g_sample, void *stream);

/* ------------------------------------------------------------------------
 * Learned initialiser kernels: a small network maps the log-scaled detector
 * image to a coarse delta volume that starts the gradient reconstruction.
 * (The paper has no network; its reconstructions start from a guess, Sec. 4.)
 * ------------------------------------------------------------------------ */

/* Dense layer on the tensor cores: C[m][n] = beta*C[m][n] + sum_k A(m,k) B(n,k)
 * (+ bias[n]) (ReLU if relu), A(m,k) = A[m*sam + k*sak], B(n,k) = B[n*sbn + k*sbk]
 * (strides give transposes; sam = sak = 0 makes A a constant).  FP32 arrays,
 * operands rounded to BF16 (nearest even), FP32 accumulation.  bias may be
 * NULL; beta = 0 overwrites C.  Long-K shapes split K over CTAs: the partial
 * sums go to ws (caller-owned device memory, 16-byte aligned, at least
 * mslice_nn_gemm_workspace(M, N, K) bytes; 0 means none is needed) and are
 * summed in a fixed order, so results are deterministic.  C must not alias A,
 * B or ws. */
size_t mslice_nn_gemm_workspace(int M, int N, int K);
int mslice_nn_gemm(int M, int N, int K, const float *A, long long sam, long long sak, const float *B,
                   long long sbn, long long sbk, float *C, long long ldc, const float *bias, int relu,
                   float beta, void *ws, size_t ws_bytes, void *stream);

/* Dense layer on the 5th-generation tensor cores (tcgen05.mma into tensor
 * memory, operands by TMA): C[m][n] = beta*C[m][n] + sum_k A[m][k] B[n][k]
 * (+ bias[n]) (ReLU if relu), FP32 accumulation.
 *   A  [M][lda] BF16, row-major (k contiguous), 16-byte aligned, lda >= K and
 *      a multiple of 8;  B [N][ldb] BF16, the same;  C [M][ldc] float32,
 *      ldc >= N;  bias: NULL or float32[N].  All device memory owned by the
 *      caller; C must not alias A, B or bias.
 * One CTA per 128 x 256 tile of C; asynchronous on stream.  Errors:
 * MSLICE_EINVAL (sizes, null or misaligned pointers, strides),
 * MSLICE_EUNSUPPORTED (M > 65535 * 128, or no tensor-map encoder in the
 * driver), MSLICE_ELAUNCH.  Every device-side wait is bounded (about 1 s);
 * mslice_nn_gemm_bf16_status reports one that ran out. */
int mslice_nn_gemm_bf16(int M, int N, int K, const void *A, long long lda, const void *B, long long ldb, float *C,
                        long long ldc, const float *bias, int relu, float beta, void *stream);

/* Waits for stream; MSLICE_ETIMEDOUT (and clears it) if a bounded wait of a
 * tensor-core GEMM ran out since the last call, else MSLICE_OK. */
int mslice_nn_gemm_bf16_status(void *stream);

/* Operand packing for mslice_nn_gemm_bf16: dst[r][k] = BF16(src[r*s_row +
 * k*s_k]) rounded to nearest even for k < K, and 0 for K <= k < ld (the
 * strides give transposes).  dst: [rows][ld] 2-byte elements, device,
 * 2-byte aligned.  MSLICE_EINVAL for null pointers, rows or K < 1, ld < K. */
int mslice_nn_pack_bf16(const float *src, long long s_row, long long s_k, int rows, int K, void *dst, long long ld,
                        void *stream);
/* Patch permutation between NHWC [B][H][W][C] and [B][H/p][W/p][p][p][C]
 * (inverse = 0: NHWC -> patches; 1: back).  A convolution with kernel = stride
 * = p is a GEMM on the patch layout; its transpose is a GEMM followed by the
 * inverse permutation.  H and W must be multiples of p; in and out must not alias. */
int mslice_nn_space_to_depth(const float *in, float *out, int B, int H, int W, int C, int p, int inverse,
                             void *stream);
/* ReLU backward: dz = dy where y > 0, else 0 (y = ReLU output), n elements. */
int mslice_nn_relu_backward(const float *y, const float *dy, float *dz, size_t n, void *stream);
/* Output layer: y = hi * sigmoid(z) [rows][cols]; with a target t, the mean
 * squared error per row into row_loss[rows] (FP64, divided by rows*cols) and
 * dz = dL/dz of L = mean((y - t)^2); target, dz, row_loss may be NULL. */
int mslice_nn_sigmoid_mse(const float *z, const float *target, float *y, float *dz, double *row_loss,
                          int rows, int cols, float hi, void *stream);
/* Network input from detector images [nimg][nz][ny] (natural FFT order):
 * counts > 0: intensities, a = sqrt(s I) with s = counts / sum(I) per image;
 * counts == 0: intensities already in photon counts, a = sqrt(I);
 * counts < 0: the input is the amplitude a itself (e.g. sqrt of measured counts).
 * Then a += 0.5 noise[i] when noise (a standard normal array of the same shape)
 * is given, clamped at 0 (the spread of a Poisson amplitude), and
 * x = gain * log(1 + a^2), written centred (fftshift) to x [nimg][nz][ny]. */
int mslice_nn_detector_features(const float *intensity, const float *noise, float *x, int nimg, int nz,
                                int ny, float counts, float gain, void *stream);
/* Training volumes: out[s][i0][i1][i2] = value inside any of the
 * boxes_per_sample boxes of sample s, else 0; boxes int32
 * [nsamples][boxes_per_sample][6] = (lo0, hi0, lo1, hi1, lo2, hi2), half-open. */
int mslice_nn_rasterize_boxes(const int *boxes, int boxes_per_sample, int nsamples, int d0, int d1, int d2,
                              float value, float *out, void *stream);

/* Per-kernel timing (tracing).  While enabled, every kernel launch of the
 * library is bracketed by a CUDA event pair recorded on the launching stream;
 * mslice_profile_read() waits for the recorded events and returns, per kernel
 * name, the launch count, the summed device time and the summed work units
 * (one unit = one grid point of one wavefield advanced through one slice).
 * Enabling resets the counters.  Not thread-safe; host-side bookkeeping only. */
typedef struct mslice_kernel_time {
    char name[32];
    int32_t launches;
    double total_ms;
    double units;
} mslice_kernel_time;

int mslice_profile_enable(int on);
/* Fills up to max_entries records; returns the number filled or a negative code. */
int mslice_profile_read(mslice_kernel_time *out, int max_entries);

/* Text of the last failing CUDA runtime call of this thread ("" if none);
 * explains an MSLICE_ELAUNCH. */
const char *mslice_last_cuda_error(void);

/* Static text for a return code. */
const char *mslice_strerror(int code);

#ifdef __cplusplus
}
#endif
#endif /* MSLICE_H */
