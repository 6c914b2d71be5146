/*
 * ddflb.h - C ABI of the GB300 (sm_103a) double-distribution-function lattice
 * Boltzmann library with local vorticity recovery.
 *
 * Method: Hajabdollahi & Premnath, "Local vorticity computation in double
 * distribution functions based lattice Boltzmann methods for flow and scalar
 * transport", arXiv 1908.06742.  Two D2Q9 lattices advance together: the flow
 * populations f with the MRT collision of Sec. 2 (Eq. MRT-LBEfluidmotion_transformed,
 * optional body force) and the passive-scalar populations g with the MRT collision
 * of Sec. 3 (Eq. MRT-LBECDE), whose third-order off-diagonal equilibria carry
 * the anisotropy beta1 != beta2 (Eq. eqmrawmoment_CDE).  The strain rate S_ij
 * and the vorticity omega_z are recovered node by node from the second-order
 * non-equilibrium moments of both lattices (Sec. 4, Eqs. crossderivativeRHS1 to
 * vorticityexpression), with no finite differences.
 *
 * Conventions for every entry point:
 *  - Units are lattice units, dx = dt = 1 (Sec. 5).  Node (i, j) is at x = i,
 *    y = j; fields are row-major [ny][nx] float arrays, x fastest.
 *  - Pointers named dev_* or documented as device pointers must be CUDA device
 *    memory of the current device.  The library never allocates device memory:
 *    the caller owns the workspace and every field buffer, and must keep them
 *    alive until ddflb_destroy / ddflb_batch_destroy.
 *  - Calls are asynchronous on the stream given at creation, except the *_stats
 *    calls, which synchronise that stream.
 *  - Errors are returned as ddflb_status, never thrown; a message describing
 *    the last error of the calling thread is available from ddflb_last_error().
 *  - Time: the state after n calls-worth of steps is the PRE-collision state
 *    f(x, t = n), g(x, t = n); ddflb_fields reports the fields of that state.
 */
#ifndef DDFLB_H
#define DDFLB_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  DDFLB_OK = 0,
  DDFLB_EINVAL = 1,         /* invalid argument or parameter */
  DDFLB_ENOMEM = 2,         /* workspace smaller than *_workspace_bytes() */
  DDFLB_ECUDA = 3,          /* a CUDA runtime call failed (message has the CUDA error) */
  DDFLB_EDIVERGED = 4,      /* a reduction found a non-finite mass or scalar sum */
  DDFLB_ENOTCONVERGED = 5,  /* a run-to-tolerance call stopped at its step limit */
  DDFLB_ETIMEOUT = 6        /* a device-side wait gave up after its spin limit */
} ddflb_status;

/* Boundary kinds (Sec. 5).  Walls are half-way bounce-back for f (Sec. 5.1,
 * 5.4); the moving wall adds the momentum term 2 w_a rho0 (e_a . u_w) / c_s^2;
 * the scalar takes a fixed value on walls by anti-bounce-back
 * g_a = -g*_abar + 2 w_a phi_w (the paper fixes the value, not the scheme). */
typedef enum {
  DDFLB_BC_PERIODIC = 0, /* periodic in x and y (Sec. 5.2)                          */
  DDFLB_BC_CAVITY = 1,   /* walls on all sides; top wall (above row ny-1) moves with
                            (u_lid, 0) and holds phi_lid, others hold phi_wall (5.4) */
  DDFLB_BC_CHANNEL = 2   /* periodic in x; static bottom wall with phi_wall, top wall
                            moving with (u_lid, 0) holding phi_lid (Sec. 5.1, 5.3)   */
} ddflb_bc;

/* Storage precision of the populations.  Populations are stored as deviations
 * from the rest equilibrium, (f_a - w_a rho0) * scale_f and (g_a - w_a phi0) *
 * scale_g; collision arithmetic is always FP32. */
typedef enum { DDFLB_FP32 = 0, DDFLB_FP16 = 1, DDFLB_BF16 = 2 } ddflb_storage;

/* Collision model of the scalar lattice.  MRT: Sec. 3 (raw moments, rates
 * omega_g).  SRT: App. B, g~ = g - (g - g^eq)/tau_phi with 1/tau_phi =
 * omega_g[1] (entries 2..8 are ignored; run as the MRT with all rates equal,
 * which is the same collision).  CASCADED: App. C, central moments relaxed at
 * the rates omega_g through the cascade of moment changes h_1..h_8 in the
 * orthogonal basis K (K6, K7 read as 2|e_y> - 3|e_x^2 e_y>, 2|e_x> - 3|e_x e_y^2>,
 * the orthogonal forms the paper's inner products require).  CENTRAL: App. D,
 * central moments relaxed directly (raw -> central -> relax -> raw).  For the
 * two central-moment models the equilibria are Eq. (eqmcentralmoment_CDE) and
 * omega is recovered from the central xy non-equilibrium moment with
 * (beta - 1) in the scalar-gradient correction (the Chapman-Enskog expansion
 * of a central-moment collision; the paper does not write it out).  The
 * batched entry points accept MRT and SRT only. */
typedef enum {
  DDFLB_SCALAR_MRT = 0,
  DDFLB_SCALAR_SRT = 1,
  DDFLB_SCALAR_CASCADED = 2,
  DDFLB_SCALAR_CENTRAL = 3
} ddflb_scalar_model;

/* ddflb_params.flags */
#define DDFLB_FLAG_HOST_IO 1 /* reserve a staging area so ddflb_init_host /
                                ddflb_fields_host can take host buffers */

typedef struct {
  int32_t nx, ny;       /* grid size, each >= 2 (channel: nx >= 1)                */
  int32_t bc;           /* ddflb_bc                                               */
  int32_t storage;      /* ddflb_storage                                          */
  /* Relaxation diagonals in the non-orthogonal basis of Eq. (basisvectors):
   * omega_f = diag(0,0,0,w3,w4,w5,w6,w7,w8) of Eq. (relaxationtimematrix_fluidmotion),
   * nu = cs2 (1/w4 - 1/2) with w4 = w5; omega_g = diag(0,w1^phi..w8^phi) of
   * Eq. (relaxationtimematrix_CDE), D_phi = cs2_phi (1/w1^phi - 1/2).  Entries
   * 0..2 of omega_f and entry 0 of omega_g must be 0 (conserved moments). Every
   * rate must lie in [0, 2]. */
  double omega_f[9];
  double omega_g[9];
  double beta1, beta2;  /* scalar-flux anisotropy, |beta1 - beta2| > 1e-6 (Sec. 4) */
  double cs2, cs2_phi;  /* c_s^2 and c_sphi^2: must be 1/3 (as in all of Sec. 5)    */
  double rho0, phi0;    /* rest state: storage offsets; rho0 also in the lid term   */
  double u_lid;         /* x velocity of the moving wall (cavity, channel)          */
  double phi_lid;       /* scalar value held by the moving wall                     */
  double phi_wall;      /* scalar value held by the other walls                     */
  double phi_min;       /* where |phi| < phi_min the cross derivatives and omega
                           are written as NaN (Sec. 4 requires phi != 0)            */
  double scale_f, scale_g; /* storage scale (power of two; <= 0 means 1)           */
  int32_t check_every;  /* steps between reductions in ddflb_step (0 = none)        */
  int32_t flags;        /* DDFLB_FLAG_*                                             */
  /* Body force F in the momentum equation (Sec. 2), acting at node x at time t:
   *   F(x, t) = (fx + field_x(x), fy + field_y(x)) cos(force_omega t)
   * (force_omega = 0: steady; field from ddflb_set_force_field, zero without).
   * With a force the flow populations held are f-bar = f - S/2, S the source of
   * Eq. (MRT-LBEfluidmotion_transformed) whose moments are the sigma' listed
   * after Eq. (eqmrawmoment); u = (sum_a f-bar_a e_a + F/2) / rho (Eq.
   * hydrodynamic_fields); ddflb_populations returns f-bar.  The batched entry
   * points and ddflb_reduce_noalloc accept only fx = fy = force_omega = 0. */
  double fx, fy;
  double force_omega;
  /* Scalar collision model (ddflb_scalar_model).  The local kinematics of
   * Sec. 4 are evaluated to match it. */
  int32_t scalar_model;
  int32_t reserved;     /* must be 0 */
} ddflb_params;

typedef struct ddflb_ctx ddflb_ctx;

/* Bytes of device workspace ddflb_create needs for these parameters (0 if the
 * parameters are invalid; see ddflb_last_error). */
size_t ddflb_workspace_bytes(const ddflb_params* p);

/* Validate *p, carve the population buffers, reduction scratch and status
 * block out of dev_workspace (device memory of at least
 * ddflb_workspace_bytes(p) bytes, 256-byte aligned), and bind cuda_stream
 * (a cudaStream_t; NULL = legacy default stream).  Host memory for the handle
 * is the only allocation.  Errors: EINVAL (parameters, alignment, NULL),
 * ENOMEM (bytes too small). */
ddflb_status ddflb_create(const ddflb_params* p, void* dev_workspace, size_t bytes,
                          void* cuda_stream, ddflb_ctx** out);

/* Set the state at t = 0 from macroscopic device fields rho, ux, uy, phi
 * ([ny][nx] floats each) and optional gradients grads (6 planes [6][ny][nx]:
 * d_x u_x, d_y u_x, d_x u_y, d_y u_y, d_x phi, d_y phi; NULL = equilibrium).
 * The populations are the equilibria of Eqs. (eqmrawmoment), (eqmrawmoment_CDE)
 * plus the Chapman-Enskog non-equilibrium parts of Eqs. (strainratexxpyy) to
 * (strainratexy) and (1stnoneqmmomentx_CDE), (1stnoneqmmomenty_CDE),
 * (offdiagonal2ndnoneqmmoment_CDE).  Resets the step counter and status. */
ddflb_status ddflb_init(ddflb_ctx* c, const float* rho, const float* ux, const float* uy,
                        const float* phi, const float* grads);

/* ddflb_init with HOST input buffers (same layout); the copies run through
 * the input staging area, on the context stream or, after ddflb_set_io_streams,
 * on the upload stream.  The call does not wait for them: the host buffers must
 * stay valid and unchanged until they are done (ddflb_io_wait, or a
 * synchronisation of the stream that ran them); pinned memory lets the copies
 * overlap with compute.  Requires DDFLB_FLAG_HOST_IO at creation (else EINVAL). */
ddflb_status ddflb_init_host(ddflb_ctx* c, const float* rho, const float* ux, const float* uy,
                             const float* phi, const float* grads);

/* Advance n >= 0 time steps: one fused pass per step streams f and g (pull),
 * applies the wall rules, collides both lattices in moment space and stores the
 * post-collision deviations.  At every multiple K of check_every a reduction
 * records the mass, scalar and the velocity residual
 * r = |u(t) - u(t-K)|_2 / (K |u(t)|_2) (FP64 sums; the mean relative change
 * per step over the interval, which stays above the FP32 rounding jitter of a
 * one-step difference) in the device status block; once a sum is non-finite
 * further steps are skipped and the next ddflb_stats returns EDIVERGED. */
ddflb_status ddflb_step(ddflb_ctx* c, int64_t n);

/* Local kinematics of the current state (Sec. 4): density, velocity, scalar,
 * S_xx = d_x u_x, S_xy = (d_x u_y + d_y u_x)/2, S_yy = d_y u_y and
 * omega_z = d_x u_y - d_y u_x, each into a [ny][nx] device float buffer.  Any
 * pointer may be NULL to skip that field. */
ddflb_status ddflb_fields(ddflb_ctx* c, float* rho, float* ux, float* uy, float* phi,
                          float* sxx, float* sxy, float* syy, float* omega);

/* Further local fields of the current state in one pass, each into a [ny][nx]
 * device float buffer (any pointer may be NULL):
 *  - the full velocity gradient d_x u_x, d_y u_x, d_x u_y, d_y u_y: diagonal
 *    parts from Eqs. (diagvelderivativeresult1), (diagvelderivativeresult2),
 *    the cross derivatives from Eqs. (offdiagvelderivativeresult1),
 *    (offdiagvelderivativeresult2);
 *  - the scalar gradient d_x phi, d_y phi from the first-order scalar
 *    non-equilibrium moments (Eqs. 1stnoneqmmomentx_CDE, 1stnoneqmmomenty_CDE);
 *  - the velocity-gradient invariants and the Lamb vector named in Sec. 1,
 *    Q = -S_ij S_ij / 2 + omega_k omega_k / 4,
 *    R = (S_ij S_jk S_ki + 3/4 omega_i omega_j S_ij) / 3 and L = omega x u,
 *    for the planar flow (omega along z, so R = S_ij S_jk S_ki / 3 and
 *    L = (-omega u_y, omega u_x)).
 * Quantities that need omega are NaN where |phi| < phi_min. */
ddflb_status ddflb_derived(ddflb_ctx* c, float* dxux, float* dyux, float* dxuy, float* dyuy,
                           float* dxphi, float* dyphi, float* q, float* r, float* lamb_x,
                           float* lamb_y);

/* ddflb_fields into HOST buffers (staged; requires DDFLB_FLAG_HOST_IO).  The
 * call waits until the host buffers hold the result (ddflb_fields_host_async
 * followed by ddflb_io_wait). */
ddflb_status ddflb_fields_host(ddflb_ctx* c, float* rho, float* ux, float* uy, float* phi,
                               float* sxx, float* sxy, float* syy, float* omega);

/* ddflb_fields into HOST buffers without waiting: the fields kernel writes the
 * output staging area on the context stream and the copies to the host run on
 * the I/O stream (or the context stream); the host buffers hold the result
 * after ddflb_io_wait.  The next ddflb_fields_host_async waits on the device
 * for these copies before it reuses the staging area. */
ddflb_status ddflb_fields_host_async(ddflb_ctx* c, float* rho, float* ux, float* uy, float* phi,
                                     float* sxx, float* sxy, float* syy, float* omega);

/* Run the uploads of ddflb_init_host on upload_stream and the downloads of
 * ddflb_fields_host_async on download_stream (two distinct cudaStream_t of
 * the context's device; both NULL: back to the context stream), so that they
 * overlap with the time steps and with each other: the upload of step k+1 and
 * the download of step k run while step k+1 computes.  Ordering against the
 * compute stream is kept with events: an upload waits until the previous
 * ddflb_init has consumed the input staging area, ddflb_init waits for its
 * upload, a download waits for its fields kernel, and the next fields kernel
 * waits for the previous download.  Host-side pipelining only (no paper
 * counterpart).  Requires DDFLB_FLAG_HOST_IO. */
ddflb_status ddflb_set_io_streams(ddflb_ctx* c, void* upload_stream, void* download_stream);

/* Wait until every host copy queued by this context has completed. */
ddflb_status ddflb_io_wait(ddflb_ctx* c);

/* The pre-collision populations of the current state as full values (not
 * deviations), f and g each [9][ny][nx] device floats (either may be NULL). */
ddflb_status ddflb_populations(ddflb_ctx* c, float* f, float* g);

/* Reduce the current state now and return (synchronising the stream): total
 * mass sum rho, total scalar sum phi, the residual of the last check (NaN if
 * none yet) and the number of steps taken.  Any output pointer may be NULL.
 * Returns EDIVERGED once a non-finite sum has been seen. */
ddflb_status ddflb_stats(ddflb_ctx* c, double* mass, double* scalar, double* residual,
                         int64_t* step);
/* Advance until steady state (Sec. 5.4 reports the cavity flows at steady
 * state): steps up to each residual check (the context's check_every K must be
 * > 0) and reads r = |u(t) - u(t-K)| / (K |u(t)|) from the check, as
 * ddflb_stats reports it.  Returns OK as soon as r < tol; EDIVERGED once a
 * non-finite sum is seen; ENOTCONVERGED after max_steps steps, or when
 * stall_checks > 0 consecutive checks have not lowered r below its best value
 * so far (the residual has reached its precision floor above tol).  Steps
 * taken by this call go to *steps_taken (may be NULL).  Synchronises the
 * context stream at every check.  Errors: EINVAL (check_every <= 0, tol <= 0,
 * negative counts). */
ddflb_status ddflb_run_to_tolerance(ddflb_ctx* c, double tol, int64_t max_steps,
                                    int32_t stall_checks, int64_t* steps_taken);

/* Checkpoint: size in bytes of the raw state, and copies of it to/from a
 * caller device buffer (device-to-device, asynchronous).  Resuming from a saved
 * state reproduces the run bit for bit. */
size_t ddflb_state_bytes(const ddflb_ctx* c);
ddflb_status ddflb_get_state(ddflb_ctx* c, void* dev_dst, size_t bytes, int64_t* step);
ddflb_status ddflb_set_state(ddflb_ctx* c, const void* dev_src, size_t bytes, int64_t step);

/* ddflb_reduce_noalloc - the paper has no counterpart; this exists for
 * callers that cannot allocate device memory where they need the reductions
 * (loops where cudaMalloc is forbidden, plug-ins handed only existing
 * buffers).  It runs the same reduction as ddflb_stats / the residual checks
 * of ddflb_step on a raw state buffer (the layout ddflb_get_state writes for
 * parameters *p) and allocates nothing: its scratch (block partial sums, a
 * status block and a velocity snapshot) is a file-scope device array of the
 * library, sized for at most DDFLB_NOALLOC_MAX_NODES nodes (about 8.4 MB,
 * held by every GPU that loads the library until the process exits).
 *   mode bit 1: also compute the residual |u - u_snap|_2 / |u|_2 against the
 *               snapshot stored by an earlier call (EINVAL if none of this
 *               nx x ny grid was stored on this device);
 *   mode bit 2: store this state's velocity as the new snapshot.
 * dev_out: 4 device doubles (mass, scalar, sum |u|^2, residual or NaN).
 * Asynchronous on cuda_stream.  The first call on a device, with that device
 * current, looks up the scratch address (not capturable): make it before any
 * stream capture.  All calls on a device share the scratch and it keeps the
 * last call's snapshot; calls that overlap on the GPU (other streams, other
 * threads) race on it.  Errors: EINVAL (parameters, sizes beyond the maximum,
 * NULL pointers, missing snapshot), ECUDA. */
#define DDFLB_NOALLOC_MAX_NODES (1 << 20)
ddflb_status ddflb_reduce_noalloc(const ddflb_params* p, const void* dev_state,
                                  size_t state_bytes, int32_t mode, double* dev_out,
                                  void* cuda_stream);

/* Autotuner for the step kernel: times each thread-block shape (128x1, 256x1,
 * 64x2, 32x4, 64x4, 32x8, 64x1) with each kernel variant (path 1: one node per
 * thread; path 2, 16-bit storage with even nx only: two adjacent nodes per
 * thread with aligned 4-byte pair accesses), and path 3 (four nodes per
 * thread, its own 128x1 block) once where it applies, over trial_steps with
 * CUDA events, and keeps the fastest.  Runs on zeroed populations, so it OVERWRITES the state and
 * resets the step counter: call it before ddflb_init.  Synchronises. */
ddflb_status ddflb_autotune(ddflb_ctx* c, int32_t trial_steps, int32_t* block_x,
                            int32_t* block_y, int32_t* path, double* ms_per_step);
/* Set the step kernel's block shape directly (e.g. from a cached tuning):
 * block_x a multiple of 32, 32..256 threads in all. */
ddflb_status ddflb_set_block(ddflb_ctx* c, int32_t block_x, int32_t block_y);
/* Step kernel variant: 1 one node per thread; 2 paired nodes, two adjacent
 * nodes per thread with aligned 4-byte pair accesses (16-bit storage, even nx,
 * unforced, MRT or SRT scalar; otherwise falls back to one node per thread);
 * 3 four adjacent nodes per thread with aligned 8-byte accesses (as 2, with
 * nx a multiple of 4; nodes next to a wall one by one; otherwise falls back to
 * 2, then 1);
 * 0 (default) = 3 for 16-bit storage (else 2 on a periodic lattice, else 1),
 * 1 for FP32.  All give bit-identical
 * results; which is faster depends on the shape, so the autotuner times them. */
ddflb_status ddflb_set_path(ddflb_ctx* c, int32_t path);

/* Spatially varying part of the body force (Sec. 2; e.g. the four-rolls mill
 * of Sec. 5.2): dev_field is a device array [2][ny][nx] of floats (F_x plane,
 * then F_y), added to (fx, fy) of the parameters and modulated with them by
 * cos(force_omega t).  The caller owns the array and keeps it alive and
 * unchanged while the context steps; NULL removes the field.  Takes effect for
 * the next ddflb_init, ddflb_step, ddflb_fields and ddflb_stats.  A forced
 * context always runs the one-node-per-thread step kernel. */
ddflb_status ddflb_set_force_field(ddflb_ctx* c, const float* dev_field);

/* Release the handle (host memory only; the workspace stays the caller's). */
ddflb_status ddflb_destroy(ddflb_ctx* c);

/* ---------------------------------------------------------------------------
 * One lattice divided into y-slabs.  The collide-and-stream update of Secs. 2
 * and 3 is local: a node pulls the post-collision populations of its eight
 * neighbours only, so a slab of rows can advance on its own if, before each
 * step, the populations that cross its faces are copied in from the slabs
 * beside it.  Per face and step that is 3 populations (those with e_y = +1
 * going up, e_y = -1 going down) x 2 lattices x nx values.  Divided runs are
 * bit-identical to the undivided lattice.
 *
 * A slab context is a ddflb_ctx for rows [y0, y0 + rows) of the lattice *p
 * (p->ny is the whole lattice's height).  Its population buffers carry one
 * ghost row on each face shared with another slab: both faces of a slab of a
 * periodic lattice (unless rows = p->ny), the inner faces of a cavity or
 * channel, whose walls stay with the bottom and top slabs.  Every ddflb_*
 * call on a whole lattice applies to it, for its own rows: ddflb_init and
 * ddflb_fields take and give [rows][nx] arrays, ddflb_set_force_field a
 * [2][rows][nx] array, ddflb_stats and ddflb_sums sum its own nodes.  While
 * it has a ghost row: check_every must be 0 (combine ddflb_sums over slabs
 * instead), force_omega must be 0, and ddflb_step takes n <= 1.  The protocol
 * is init, then per step: ddflb_step(slab, 1) on every slab, then refresh the
 * ghost rows (ddflb_halo_exchange_local for slabs on one device, or
 * ddflb_halo_pack -> send/receive -> ddflb_halo_unpack between processes).
 * The init writes the first step's ghost values itself: no exchange before
 * the first step.  Fields, populations and sums read the ghost rows, so they
 * too follow an exchange.  16-bit storage steps node by node in a slab (bit-
 * identical to the grouped kernels of a whole lattice).  Errors: EINVAL (rows
 * outside the lattice, check_every != 0 or force_omega != 0 with a ghost
 * row), ENOMEM, as ddflb_create. */
size_t ddflb_slab_workspace_bytes(const ddflb_params* p, int32_t y0, int32_t rows);
ddflb_status ddflb_slab_create(const ddflb_params* p, int32_t y0, int32_t rows, void* dev_workspace,
                               size_t bytes, void* cuda_stream, ddflb_ctx** out);
/* Elements of the storage type (4 bytes at FP32, 2 at 16 bit) in one face
 * message: [6][nx] = flow then scalar, 3 populations each. */
size_t ddflb_halo_elems(const ddflb_ctx* c);
/* Copy the outgoing populations of the current state into device buffers of
 * ddflb_halo_elems elements: dev_down gets directions 4, 7, 8 of the bottom
 * row (for the slab below), dev_up directions 2, 5, 6 of the top row (for the
 * slab above).  Either may be NULL; EINVAL for a face without a neighbour. */
ddflb_status ddflb_halo_pack(ddflb_ctx* c, void* dev_down, void* dev_up);
/* Write what the slab below sent up (dev_from_below) and what the slab above
 * sent down (dev_from_above) into the ghost rows.  Either may be NULL. */
ddflb_status ddflb_halo_unpack(ddflb_ctx* c, const void* dev_from_below,
                               const void* dev_from_above);
/* Every face of `parts` slabs of one lattice held on one device, given bottom
 * to top (covering all rows, same stream, same step): one kernel copies each
 * slab's outgoing rows straight into its neighbours' ghost rows (wrapping for
 * a periodic lattice).  At most 64 slabs.  parts = 1 with a whole-lattice
 * context is a no-op. */
ddflb_status ddflb_halo_exchange_local(ddflb_ctx* const* slabs, int32_t parts);
/* Reduce the current state now (FP64 sums over the context's own nodes) and
 * synchronise: out[0] = sum (rho - rho0), out[1] = sum (phi - phi0),
 * out[2] = sum |u|^2, out[3] = sum |u - u_snap|^2 (mode bit 1; NaN without).
 * mode bit 2 stores this state's velocity as the new snapshot.  Summed over
 * the slabs of a lattice these give its mass, scalar and the residual
 * sqrt(sum out[3] / sum out[2]) / K for snapshots K steps apart (the same r as
 * ddflb_step's checks).  Errors: EINVAL (mode bit 1 without a snapshot),
 * EDIVERGED. */
ddflb_status ddflb_sums(ddflb_ctx* c, int32_t mode, double* out);

/* ---------------------------------------------------------------------------
 * Batched lattices: n independent lattice pairs (each its own ddflb_params:
 * size, boundary kind, rates, lid) advanced together.  Each chunk of steps is
 * one persistent cooperative launch that walks a flattened tile list of all
 * instances, with a device-wide barrier between time steps whose waits are
 * bounded in time (a wait that runs out ends the launch; *_stats then returns
 * ETIMEOUT).  A chunk launch is captured once as a CUDA graph and replayed.
 * All instances share storage precision and check_every.  Every check_every
 * steps each instance's residual r = |u(t)-u(t-K)|/(K |u(t)|) is reduced in a
 * fixed order; an instance whose r falls below the tolerance (converged) or
 * whose sums are not finite (diverged) is frozen from then on. */
#define DDFLB_INST_CONVERGED 1
#define DDFLB_INST_DIVERGED 2
#define DDFLB_INST_CAPPED 4  /* frozen at its own step limit without converging */
typedef struct ddflb_batch ddflb_batch;

/* Workspace bytes for n instances with parameters p[0..n-1] (0 if invalid). */
size_t ddflb_batch_workspace_bytes(int32_t n, const ddflb_params* p);
/* Carve the batch out of dev_workspace (256-byte aligned, caller-owned) and
 * upload its tile list (synchronises the stream once).  Default tiles 128 x 1,
 * as many co-resident CTAs per SM as fit.  Errors: EINVAL, ENOMEM, ECUDA. */
ddflb_status ddflb_batch_create(int32_t n, const ddflb_params* p, void* dev_workspace,
                                size_t bytes, void* cuda_stream, ddflb_batch** out);
/* Tolerance for the convergence freeze (0 = never freeze on convergence),
 * steps per persistent launch, the barrier wait limit in seconds, and whether
 * the freeze also waits for the scalar residual |phi(t)-phi(t-K)|/(K |phi(t)|)
 * to fall below tol (the vorticity of Sec. 4 depends on the scalar lattice). */
ddflb_status ddflb_batch_set_run(ddflb_batch* b, double tol, int32_t steps_per_launch,
                                 double barrier_timeout_s, int32_t scalar_residual);
/* Run settings of instance i, overriding the batch's: its own tolerance (tol
 * >= 0; a negative tol returns to the batch's) and a step limit max_steps (> 0:
 * at the first check at least max_steps steps after its last init, an
 * instance that has not converged is frozen with DDFLB_INST_CAPPED; 0: no
 * limit).  Kept across ddflb_batch_init; takes effect at the next check.
 * E.g. one launch holds cold runs to 1e-8 next to long reference runs to
 * 1e-10 capped at four times the cold steps.  Synchronises the stream. */
ddflb_status ddflb_batch_set_instance_run(ddflb_batch* b, int32_t i, double tol,
                                          int64_t max_steps);
/* How a chunk of steps is launched.  0 (default): one persistent cooperative
 * launch, every CTA walking its range of tiles step after step with a bounded
 * device-wide barrier between steps (suits many small lattices, where a
 * launch per step would cost more than the step).  1: one ordinary launch per
 * step with one CTA per tile, then a check kernel (one CTA per instance, idle
 * except at multiples of check_every) and at the end of the chunk a state-time
 * update, all captured in one graph per chunk; no barrier, more resident warps
 * (suits large batches).  Same results bit for bit.  The autotuner tries both. */
ddflb_status ddflb_batch_set_schedule(ddflb_batch* b, int32_t schedule);
ddflb_status ddflb_batch_get_schedule(const ddflb_batch* b, int32_t* schedule);
/* Tile shape (32x4, 64x2, 128x1, 32x8, 64x4, 128x2, 256x1) and CTAs per SM
 * (0 = as many as fit); rebuilds the tile list.  Used by the autotuner. */
ddflb_status ddflb_batch_set_tiles(ddflb_batch* b, int32_t tile_x, int32_t tile_y,
                                   int32_t blocks_per_sm);
ddflb_status ddflb_batch_get_tiles(const ddflb_batch* b, int32_t* tile_x, int32_t* tile_y,
                                   int32_t* blocks_per_sm);
/* Initialise instance i at the batch's current time from device fields, as
 * ddflb_init (clears its converged/diverged flags). */
ddflb_status ddflb_batch_init(ddflb_batch* b, int32_t i, const float* rho, const float* ux,
                              const float* uy, const float* phi, const float* grads);
/* Advance all active instances n steps (asynchronous). */
ddflb_status ddflb_batch_step(ddflb_batch* b, int64_t n);
/* Local kinematics of instance i's current state, as ddflb_fields. */
ddflb_status ddflb_batch_fields(ddflb_batch* b, int32_t i, float* rho, float* ux, float* uy,
                                float* phi, float* sxx, float* sxy, float* syy, float* omega);
/* Per-instance host arrays (any may be NULL): last residual, flags, the steps
 * from the instance's last ddflb_batch_init to the check at which the residual
 * first fell below tol (-1: not yet), the state time of its current state and
 * the state time of its last init (so state_time - init_time steps have been
 * run on it).  Synchronises; ETIMEOUT if a barrier wait ran out. */
ddflb_status ddflb_batch_stats(ddflb_batch* b, double* residual, int32_t* flags,
                               int64_t* steps_to_tol, int64_t* state_time, int64_t* init_time);
/* Autotuner: times every supported tile shape with the persistent launch at
 * full and half residency and with one launch per step (trial_steps per timed
 * chunk, CUDA events) and keeps the fastest (ddflb_batch_get_schedule tells
 * which schedule); returns the tile shape, CTAs per SM and time per step.  Runs on zeroed populations, so it
 * OVERWRITES every instance's state and resets the time to 0: call it before
 * ddflb_batch_init.  Synchronises the stream. */
ddflb_status ddflb_batch_autotune(ddflb_batch* b, int32_t trial_steps, int32_t* tile_x,
                                  int32_t* tile_y, int32_t* blocks_per_sm, double* ms_per_step);
/* Test hook: CTA `block` of the next launch skips its first barrier so that the
 * others' bounded waits run out (-1 disables).  Never faults or hangs. */
ddflb_status ddflb_batch_debug_skip_barrier(ddflb_batch* b, int32_t block);
ddflb_status ddflb_batch_destroy(ddflb_batch* b);

/* ---------------------------------------------------------------------------
 * Warm-start surrogate network kernels.  The paper has no network; these
 * serve the learned warm start (a small U-Net that predicts steady cavity
 * fields from the flow parameters; its output only initialises the
 * populations, the method then runs to the residual tolerance as usual).
 * Tensors: BF16 (__nv_bfloat16 bits) or FP32 device arrays, activations NHWC
 * with a channel stride cs (so a concatenation is two writers of one buffer).
 * All calls are asynchronous on `stream`; errors: EINVAL (shapes, alignment),
 * ECUDA (launch). */

/* C = act(A . B^T + bias) on tensor cores, FP32 accumulation.  A [M][K]
 * (row stride lda), B [N][K] (ldb): BF16, K-contiguous, 16-byte aligned, K,
 * lda, ldb multiples of 8.  Outputs: Cf FP32 [M][ldc] and/or Cb BF16
 * [M][ldcb] (either may be NULL); bias FP32 [N] or NULL; act 0 = none,
 * 1 = leaky ReLU (slope 0.02); accumulate: Cf += result.  splits > 1 splits
 * the K range over that many CTA slices writing to `partial` (FP32, at least
 * splits*M*N, caller-owned), summed in a fixed order afterwards (Cf only). */
ddflb_status ddflb_nn_gemm(const void* A, const void* B, int32_t M, int32_t N, int32_t K,
                           int32_t lda, int32_t ldb, float* Cf, int32_t ldc, void* Cb,
                           int32_t ldcb, const float* bias, int32_t act, int32_t accumulate,
                           int32_t splits, float* partial, void* stream);
/* GEMM kernel for all later ddflb_nn_gemm calls of the process:
 *  0 (default) = tcgen05, persistent when there are more 128 x {32, 64, 128}
 *    tiles than SMs (one CTA per SM walks the tiles; a TMA warp fills a ring of
 *    128-byte-swizzled shared-memory slots, one thread issues the MMAs into two
 *    alternating FP32 accumulators in tensor memory, four warps run the
 *    epilogue of the previous tile meanwhile), otherwise as path 2;
 *  1 = mma.sync m16n8k16 (register accumulators);
 *  2 = tcgen05 with one tile per CTA.
 * Same results up to the order of FP32 additions. */
ddflb_status ddflb_nn_set_gemm_path(int32_t path);
/* Copy to *error and clear the tcgen05 GEMM's device error word (1 = a bounded
 * wait ran out and a tile was skipped; 0 = none).  Synchronises `stream`. */
ddflb_status ddflb_nn_take_error(int32_t* error, void* stream);
/* 3x3 convolution with zero padding as an implicit GEMM on the tensor cores:
 * Y[p][n] = act(sum over taps t and channels c of X[p + s(t)][c] Wt[n][t][c]
 * + bias[n]), with s(t) = (t / 3 - 1, t % 3 - 1) in (y, x), X BF16 NHWC
 * [B][H][W] with channel stride cs (C channels read, C a multiple of 64),
 * Wt BF16 [N][9 C] (tap-major then channel, the im2col order), outputs as
 * ddflb_nn_gemm (Cf FP32 [B H W][ldc] and/or Cb BF16 [B H W][ldcb]).  No
 * patch matrix is formed: the TMA producer reads each tap's 128-pixel box of
 * the activation (a 4-D tensor map over c, w, h, image; zeros outside the
 * image) straight into the swizzled operand tile, in the same K order as
 * im2col + ddflb_nn_gemm, whose results it reproduces bit for bit.  Needs W
 * a divisor or a multiple of 128, the tile boxes whole (H divisible by
 * 128 / W where W < 128; B by 128 / (H W) where H W < 128), B H W a multiple
 * of 128, X and Wt 16-byte aligned; else EINVAL (use im2col).  Asynchronous
 * on stream; always the tcgen05 kernel (ddflb_nn_set_gemm_path does not
 * apply). */
ddflb_status ddflb_nn_conv3x3(const void* X, int32_t B, int32_t H, int32_t W, int32_t C,
                              int32_t cs, const void* Wt, int32_t N, float* Cf, int32_t ldc,
                              void* Cb, int32_t ldcb, const float* bias, int32_t act,
                              int32_t accumulate, void* stream);
/* How ddflb_nn_conv3x3 reads the activation, for all later calls of the
 * process: 0 (default) = where W is a multiple of 128 (tiles are row
 * segments) and C >= 128, one band of 130 pixels (the segment and a halo
 * pixel each side) per input row and 64-channel chunk, read by the row's three
 * taps at shifted descriptor addresses (3 loads instead of 9 per tile and
 * chunk), elsewhere one box per tap; 1 = one box per tap everywhere.  Same results bit for bit
 * (the K order is the im2col order in both). */
ddflb_status ddflb_nn_set_conv_path(int32_t path);
/* Weights of the adjoint convolution: Wf[ci][t][co] = Wt[co][8 - t][ci]
 * (BF16, Wt [Co][9][Ci] -> Wf [Ci][9][Co]), so that dX = conv3x3(dY, Wf)
 * with C = Co and N = Ci is the input gradient of Y = conv3x3(X, Wt). */
ddflb_status ddflb_nn_conv3x3_flip(const void* Wt, int32_t Co, int32_t Ci, void* Wf, void* stream);
/* 3x3 patches of X (BF16 NHWC [B][H][W][C], stride cs, zero padding):
 * col [B*H*W][9*C] (tap-major then channel), or transposed [9*C][B*H*W]. */
ddflb_status ddflb_nn_im2col(const void* X, int32_t B, int32_t H, int32_t W, int32_t C,
                             int32_t cs, void* col, int32_t transposed, void* stream);
/* Adjoint of im2col: dX[b][h][w][c] (FP32, stride cs) = sum of the 9 patch
 * entries dcol [B*H*W][9*C] (FP32) that read (h, w). */
ddflb_status ddflb_nn_col2im(const float* dcol, int32_t B, int32_t H, int32_t W, int32_t C,
                             float* dX, int32_t cs, void* stream);
/* dst [N][M] = src [M][N] (BF16, src row stride lds). */
ddflb_status ddflb_nn_transpose(const void* src, int32_t M, int32_t N, int32_t lds, void* dst,
                                void* stream);
/* 2x2 average pooling (BF16) and its adjoint (FP32, optionally accumulating). */
ddflb_status ddflb_nn_pool(const void* X, int32_t B, int32_t H, int32_t W, int32_t C, int32_t csx,
                           void* Y, int32_t csy, void* stream);
ddflb_status ddflb_nn_pool_bwd(const float* dY, int32_t B, int32_t H, int32_t W, int32_t C,
                               int32_t csy, float* dX, int32_t csx, int32_t accumulate,
                               void* stream);
/* Nearest 2x upsampling (BF16, input H x W) and its adjoint (FP32). */
ddflb_status ddflb_nn_upsample(const void* X, int32_t B, int32_t H, int32_t W, int32_t C,
                               int32_t csx, void* Y, int32_t csy, void* stream);
ddflb_status ddflb_nn_upsample_bwd(const float* dY, int32_t B, int32_t H, int32_t W, int32_t C,
                                   int32_t csy, float* dX, int32_t csx, void* stream);
/* g *= act'(.) read from the activation output y (BF16); optional BF16 copy gb. */
ddflb_status ddflb_nn_act_bwd(float* g, const void* y, int64_t rows, int32_t C, int32_t csg,
                              int32_t csy, int32_t act, void* gb, int32_t csb, void* stream);
/* db[c] = sum over rows of g[r][c] (FP32), in a fixed order.  For 4096 rows or
 * more (and C <= 4096) the partial sums go through one scratch array of the
 * library, so such calls on different streams must not overlap. */
ddflb_status ddflb_nn_bias_grad(const float* g, int64_t rows, int32_t C, int32_t cs, float* db,
                                void* stream);
/* Mean squared error of n FP32 values into *dev_loss (FP64), optional gradient
 * 2 (pred - target) / n; dev_partial: 256 doubles of caller scratch. */
ddflb_status ddflb_nn_mse(const float* pred, const float* target, int64_t n, float* grad,
                          double* dev_partial, double* dev_loss, void* stream);
/* Adam step t >= 1 on FP32 weights w with moments m, v (decoupled weight
 * decay wd); refreshes the BF16 copy wb if not NULL. */
ddflb_status ddflb_nn_adam(float* w, const float* g, float* m, float* v, void* wb, int64_t n,
                           float lr, float beta1, float beta2, float eps, int64_t t, float wd,
                           void* stream);
/* y (BF16, stride csy) = x (FP32, stride csx), rows x C. */
ddflb_status ddflb_nn_cast_bf16(const float* x, int64_t rows, int32_t C, int32_t csx, void* y,
                                int32_t csy, void* stream);

/* Initial fields for a learned warm start, computed on the device from the
 * network's prediction pred ([ny][nx][cs] FP32, channels: 0 u_x / U, 1 u_y / U,
 * 2 phi, 3 omega n / (U omega_scale) with n = nx, 4 (rho - 1) / U^2; cs >= 5):
 * rho, ux, uy, phi ([ny][nx] each) and grads ([6][ny][nx]: d_x u_x, d_y u_x,
 * d_x u_y, d_y u_y, d_x phi, d_y phi), ready for ddflb_init / ddflb_batch_init,
 * which add the Chapman-Enskog non-equilibrium part of Secs. 2 and 3.  phi is
 * clamped to [phi_lo, phi_hi]; the derivatives are central differences of the
 * predicted u and phi (one-sided on the outer rows and columns), except that
 * the antisymmetric part of the velocity gradient is the predicted vorticity:
 * d_x u_y = S_xy + omega / 2, d_y u_x = S_xy - omega / 2 with S_xy from the
 * differences.  Each operation is rounded once in a fixed order.  The paper
 * has no network; this serves the warm start only.  Asynchronous on stream.
 * Errors: EINVAL (NULL pointers, sizes, u_lid <= 0, phi_lo > phi_hi), ECUDA. */
ddflb_status ddflb_warm_fields(const float* pred, int32_t nx, int32_t ny, int32_t cs,
                               double u_lid, double omega_scale, double phi_lo, double phi_hi,
                               float* rho, float* ux, float* uy, float* phi, float* grads,
                               void* stream);

/* Message of the last error on the calling thread ("" if none). */
const char* ddflb_last_error(void);

/* Library version string. */
const char* ddflb_version(void);

#ifdef __cplusplus
}
#endif
#endif /* DDFLB_H */
