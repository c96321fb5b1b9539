/*
 * lbve.h -- C ABI of the GB300 library for the coupled lattice Boltzmann (LB) +
 * Oldroyd-B time step of Kuron, Stewart, de Graaf and Holm, "An extensible lattice
 * Boltzmann method for viscoelastic flows: complex and moving boundaries in Oldroyd-B
 * fluids" (arXiv:2009.12279).
 *
 * One context holds one solve: a D3Q19 PDF field, the 6-component polymer stress,
 * a flag field and up to LBVE_MAX_PARTICLES spheres, all resident in device memory.
 * Every call runs its work as CUDA kernels on the context's stream; nothing falls
 * back to the CPU.
 *
 * Conventions shared by all calls:
 *   - grid nx*ny*nz, cell index x + nx*(y + ny*z) (x fastest), lattice units
 *     (dx = dt = 1, cell volume 1);
 *   - vector fields are 3 consecutive arrays of n cells (x, y, z components);
 *   - stress fields are 6 consecutive arrays of n cells (xx, yy, zz, xy, xz, yz);
 *   - PDFs are 19 consecutive arrays of n cells in the D3Q19 order
 *       0:(0,0,0) 1:(+x) 2:(-x) 3:(+y) 4:(-y) 5:(+z) 6:(-z)
 *       7:(+x+y) 8:(-x-y) 9:(+x-y) 10:(-x+y) 11:(+x+z) 12:(-x-z)
 *       13:(+x-z) 14:(-x+z) 15:(+y+z) 16:(-y-z) 17:(+y-z) 18:(-y+z);
 *   - flags: 0 fluid, 1 no-slip wall, LBVE_FLAG_WALL0 + k moving-wall class k,
 *     LBVE_FLAG_PARTICLE0 + p cells covered by particle p (set by the library).
 *
 * Errors: every call returns an lbve_status and never aborts the process.  On an
 * error the context stays valid (except after LBVE_ECUDA from a sticky CUDA error)
 * and lbve_last_error() describes the cause.  Host buffers are owned by the caller
 * and are only read or written during the call (the call synchronises the
 * context's stream before returning whenever it touches host memory).
 */
#ifndef LBVE_H
#define LBVE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lbve_ctx lbve_ctx;

typedef enum {
    LBVE_OK = 0,
    LBVE_EINVAL = 1,    /* invalid argument or parameter combination */
    LBVE_ENOMEM = 2,    /* device allocation failed */
    LBVE_ECUDA = 3,     /* a CUDA call failed; lbve_last_error() has the CUDA message */
    LBVE_EUNSTABLE = 4, /* NaN, rho <= 0 or |u| above the stability limit detected */
    LBVE_ETIMEOUT = 5,  /* a bounded device-side wait gave up */
    LBVE_ESTATE = 6     /* call not valid in the context's current state */
} lbve_status;

/* Storage precision of the PDFs (arithmetic is FP64 for LBVE_F64, else FP32).
 * All reduced modes store the deviation f_i - w_i rho0 (FP16: times 2^pdf_scale_log2).
 * The 16-bit modes round the stream-collide's stores stochastically (unbiased: the
 * hardware's stochastic-rounding conversion of two values at a time, with random bits
 * from a counter-based hash of the step, the cell and the direction pair, so results are
 * deterministic and the same alone, in a pool or in z-slabs): round-to-nearest would drop
 * per-step changes smaller than half a unit of the stored deviation, and slow flows would
 * stall.  The price is a noise floor in the steady-state residual (~2e-5 per step in
 * BF16, ~2.5e-6 in FP16). */
typedef enum { LBVE_F64 = 0, LBVE_F32 = 1, LBVE_F16_SHIFTED = 2, LBVE_BF16_SHIFTED = 3 } lbve_pdf_prec;

#define LBVE_FLAG_FLUID 0
#define LBVE_FLAG_NOSLIP 1
#define LBVE_FLAG_WALL0 2
#define LBVE_MAX_WALL 16
#define LBVE_FLAG_PARTICLE0 64
#define LBVE_MAX_PARTICLES 64

/* Finite-volume terms (Sec. "Finite volume method"): bit 0 advective flux, bit 1 source.
 * When neither bit is set both are selected.  Two variants may be added:
 * LBVE_FV_CTU scales each D3Q7 face flux by the corner-transport-upwind transverse
 * overlap (1 - |u_a|)(1 - |u_b|) of the donor cell (Sec. "Stability improvements": the
 * donor cell displaced by its velocity overlaps the face neighbour along k by
 * |u_k|(1 - |u_a|)(1 - |u_b|); the edge and corner overlaps stay in the donor cell).
 * LBVE_FV_DIVU adds the tau_ij div(u) term of Eq. (source), which the paper sets to 0,
 * with div(u) the trace of the central-point velocity gradient. */
#define LBVE_FV_FLUX 1
#define LBVE_FV_SOURCE 2
#define LBVE_FV_CTU 4
#define LBVE_FV_DIVU 8

/* Kernel schedule: two kernels per step (LB, then FV), or one fused kernel per step.
 * SPLIT: the per-cell stream-collide (the LB half, Eqs. (lb), (guo), (force), (ubb)) and
 * the tiled stress update.  PIPELINED: the split schedule with the row-pipelined
 * stream-collide and the two-cell stress update wherever the grid allows them (see
 * lbve_stream_collide_kernel, lbve_stress_kernel).  AUTO: PIPELINED for large grids (the
 * row pipeline from 2^22 cells in FP32 and 16-bit storage, the two-cell stress update
 * from 2^21, where they were measured faster on GB300), SPLIT below.  All three give
 * bitwise the same results. */
#define LBVE_SCHED_AUTO 0
#define LBVE_SCHED_SPLIT 1
#define LBVE_SCHED_FUSED 2
#define LBVE_SCHED_PIPELINED 3

/*
 * Parameters of one solve.  eta is the total viscosity eta_n + eta_p, beta = eta_p/eta
 * (Sec. "Dimensionless numbers"), lambda_p the polymer relaxation time in steps
 * (Eq. (oldroydb)), body_force a force density applied to every fluid cell
 * (F in Eq. (stokes-general)).  The LB rates follow the TRT relations of Sec.
 * "Lattice Boltzmann": omega+ = 1/(3 eta_n/rho0 + 1/2),
 * (1/omega+ - 1/2)(1/omega- - 1/2) = magic (3/16 in the paper; 0 selects 3/16).
 * A non-periodic direction needs non-fluid cells in its first and last layer.
 */
typedef struct {
    int nx, ny, nz;
    int periodic[3];
    double eta, beta, lambda_p, rho0;
    double body_force[3];
    double magic;
    int pdf_prec;        /* lbve_pdf_prec */
    int pdf_scale_log2;  /* FP16 storage scale 2^k of the shifted PDFs (-1: k = 15); FP32
                            and BF16 keep the FP32 exponent range and store unscaled */
    int fv_terms;        /* LBVE_FV_* bits; no FLUX or SOURCE bit selects both */
    int schedule;        /* LBVE_SCHED_* */
    int block_x;         /* per-cell kernels: threads per block along x (32, 64 or 128; blocks
                            hold 128 threads); 0 selects the default */
    double giesekus_alpha; /* Giesekus mobility alpha in [0, 1/2]; 0 (the default) is
                            Oldroyd-B.  The paper names the Giesekus law among those its
                            finite-volume scheme extends to (Sec. "Oldroyd-B fluids") without
                            printing it; the textbook law tau + lambda tau_(1) +
                            (alpha lambda / eta_p) tau.tau = eta_p (grad u + grad u^T) adds
                            -(alpha / eta_p) tau.tau to the source of Eq. (source) */
    double fene_L2;      /* FENE-P maximum extensibility L^2 (> 3); 0 (the default) is
                            Oldroyd-B.  The paper names FENE-P among the laws its scheme
                            extends to without printing it; the textbook Peterlin closure is
                            written for the conformation tensor A, which the stress arrays
                            then hold: A_(1) = -(f A - I) / lambda_p, tau = (eta_p / lambda_p)
                            (f A - I), f = 1 / (1 - tr A / L^2).  Fields are still given and
                            read as stress tau (converted per cell).  Needs beta > 0 and
                            giesekus_alpha = 0; runs with lbve_step on the split schedule
                            only (no particles, pools, fused schedule or lbve_step_noalloc) */
} lbve_params;

/* Optional device allocator (e.g. a framework's caching allocator).  alloc returns a
 * device pointer of at least `bytes` usable on `stream`, or NULL on failure; blocks must
 * be at least 8-byte aligned.  With 16-byte aligned stress and velocity arrays (as from
 * cudaMalloc) and nx a multiple of 4, the stress kernel stages its planes by 16-byte
 * copies, else by 4-byte copies; the results are the same. */
typedef void *(*lbve_alloc_fn)(size_t bytes, void *stream, void *user);
typedef void (*lbve_free_fn)(void *ptr, size_t bytes, void *stream, void *user);

/* Fill *p with defaults (periodic box, eta 1/6, beta 0.5, lambda 1000, rho0 1, FP32). */
void lbve_default_params(lbve_params *p);

/* Device bytes a context with these parameters allocates (for admission control). */
size_t lbve_device_bytes(const lbve_params *p);

/*
 * Create a solve on the current CUDA device.  cuda_stream is a cudaStream_t (NULL =
 * legacy default stream) on which every kernel of the context runs.  The initial state
 * is rho = rho0, u = 0, tau = 0 everywhere and an all-fluid flag field.
 * Errors: EINVAL (bad parameters; *out stays NULL), ENOMEM, ECUDA.
 */
lbve_status lbve_create(const lbve_params *p, void *cuda_stream, lbve_ctx **out);
lbve_status lbve_create_with_allocator(const lbve_params *p, void *cuda_stream, lbve_alloc_fn alloc,
                                       lbve_free_fn dealloc, void *user, lbve_ctx **out);
lbve_status lbve_destroy(lbve_ctx *ctx);

/*
 * Fixed geometry (Sec. "Lattice Boltzmann", Eq. (ubb)): flags is a host array of n
 * bytes; values 0, 1 or LBVE_FLAG_WALL0 + k with k < n_wall.  wall_vel holds n_wall
 * velocities (host, 3 doubles each) of the moving-wall classes; NULL if n_wall = 0.
 * Links from fluid into a wall cell bounce back with the moving-wall term; wall
 * classes also get their momentum-exchange force reported (lbve_read_body_forces).
 * Must be called before any particle is added.  Errors: EINVAL (bad flag value,
 * fluid cell in the outer layer of a non-periodic direction), ESTATE.
 */
lbve_status lbve_set_geometry(lbve_ctx *ctx, const uint8_t *flags, const double *wall_vel, int n_wall);

/*
 * Initial fields (host arrays, each may be NULL): rho (n), u (3n), tau (6n).  The
 * PDFs are set to the equilibrium of Eq. (lb-equilibrium) at (rho, u); tau is copied
 * into the fluid cells (non-fluid cells hold zero stress, here and after
 * lbve_set_geometry, which zeroes it in the cells it makes solid).
 * Resets the time counter to 0.  Particle cells keep their state.  Page-locked arrays
 * the device can address (cudaHostAlloc, cudaHostRegister) are read in place by one
 * kernel; other host memory goes through device staging in z-slabs.  Synchronises.
 */
lbve_status lbve_init_fields(lbve_ctx *ctx, const double *rho, const double *u, const double *tau);

/* Same as lbve_init_fields with device pointers (FP64, same layouts; each may be NULL). */
lbve_status lbve_init_fields_device(lbve_ctx *ctx, const double *rho, const double *u, const double *tau);

/*
 * Add a rigid sphere (Sec. "Moving boundaries"): centre X, radius R, density rho_p
 * (mass rho_p 4/3 pi R^3, moment of inertia 2/5 m R^2), velocity v, angular velocity
 * w, constant external force and torque (all host arrays of 3 doubles; NULL = 0).
 * Fluid cells whose centre lies within R of X (minimum image on periodic sides) become
 * particle cells.  *id receives the particle index.  Errors: EINVAL, ESTATE (too many
 * particles).
 */
lbve_status lbve_add_particle(lbve_ctx *ctx, const double X[3], double R, double rho_p, const double v[3],
                              const double w[3], const double Fext[3], const double Text[3], int *id);

/*
 * Advance nsteps time steps (Eqs. (lb), (continuity)-(source), moving boundaries).
 * Asynchronous on the context's stream unless the context has particles with a
 * host-side check pending; returns after enqueueing.  Errors: EINVAL, ECUDA, EUNSTABLE.
 *
 * Instability: every stream-collide checks each fluid cell for rho <= 0, |u|^2 >= 1/3
 * (the lattice sound speed squared, beyond which the equilibrium of Eq.
 * (lb-equilibrium) has no meaning) or a NaN, and sets a flag in page-locked host memory
 * when it finds one (no synchronisation, no extra traffic).  lbve_step returns
 * LBVE_EUNSTABLE without stepping once the flag of an earlier step has reached the
 * host; lbve_synchronize returns it after synchronising.  The state stays readable.
 * lbve_init_fields[_device] and lbve_write_pdfs clear the flag.
 */
lbve_status lbve_step(lbve_ctx *ctx, int nsteps);

/*
 * Decomposition of one domain into z-slabs (the paper's runs are distributed over
 * waLBerla's block forest, Sec. "Implementation and extensibility"), one context per
 * slab, with the halo exchange done by the caller between steps (same device, peer
 * devices or ranks).  A slab context holds its planes
 * plus one ghost plane on each side: create it with nz = planes + 2 and periodic[2] = 0,
 * call lbve_set_z_range(ctx, 1, nz - 1, z_origin) before lbve_set_geometry (z_origin: the
 * domain's plane index of the slab's first computed plane, which keeps the rounding keys of
 * the 16-bit stores those of the undecomposed domain), and give the ghost
 * planes the flags (and initial fields) of the neighbouring slabs' boundary planes (solid
 * planes beyond a closed domain).  Only planes [z_lo, z_hi) are computed; wall links of
 * the ghost planes are left out, so body forces of the slabs add up to the domain's.
 * Particles, pools and the fused schedule are not combined with z-slabs.
 *
 * One step of a decomposed domain, every slab on the same schedule:
 *   lbve_step_phase(s, 0) on every slab          (stream-collide)
 *   exchange LBVE_HALO_F and LBVE_HALO_U           (between neighbouring slabs)
 *   lbve_step_phase(s, 1) on every slab          (stress update; the step completes)
 *   exchange LBVE_HALO_TAU
 * Exchanging `what` between a lower slab A and an upper slab B: pack(A, what, 1, buf),
 * unpack(B, what, 0, buf), and pack(B, what, 0, buf2), unpack(A, what, 1, buf2).  Buffers
 * are device memory of lbve_halo_bytes(ctx, what) bytes: plane-major values, one x-y plane
 * of the slab per value, x fastest:
 *   LBVE_HALO_F    the 5 PDFs per cell that cross the face in the step just taken (raw
 *                  storage elements; which slots depends on that step's parity of the
 *                  in-place layout, handled by the library): 5 storage elements per cell;
 *   LBVE_HALO_U    u of the boundary plane, 3 reals per cell (into the ghost plane);
 *   LBVE_HALO_TAU  the stress of the boundary plane, 6 reals per cell (into the ghost).
 * A decomposed run gives bitwise the fields of the undecomposed one.  Calls enqueue on
 * the context's stream.  Errors: EINVAL, ESTATE (not a z-slab, phases out of order).
 */
#define LBVE_HALO_F 0
#define LBVE_HALO_U 1
#define LBVE_HALO_TAU 2
lbve_status lbve_set_z_range(lbve_ctx *ctx, int z_lo, int z_hi, int z_origin);
/* phase 0: the stream-collide of the next step (with the momentum exchange before it);
 * phase 1: its stress update, completing the step.  lbve_step refuses while a phase 0
 * awaits its phase 1. */
lbve_status lbve_step_phase(lbve_ctx *ctx, int phase);
size_t lbve_halo_bytes(const lbve_ctx *ctx, int what);
lbve_status lbve_halo_pack(lbve_ctx *ctx, int what, int side, void *dev_buf);
lbve_status lbve_halo_unpack(lbve_ctx *ctx, int what, int side, const void *dev_buf);

/* 1 if the context's instability flag is set (see lbve_step), 0 if not, -1 for NULL.
 * Does not synchronise: steps still in flight may set it later. */
int lbve_is_unstable(const lbve_ctx *ctx);

/*
 * Which stream-collide kernel lbve_step launches for this context (split schedule).
 * LBVE_LB_ROWS: the row pipeline -- a block walks a strip of x-rows of one plane, and a
 * producer warp moves each row's 19 PDF rows (AA layout of the step's parity), its mask
 * row and the stress rows its polymer force reads (Eq. (force): the rows y -+ 1 and
 * z -+ 1) into shared memory with bulk asynchronous copies completing on mbarriers.  It
 * is taken with schedule PIPELINED (AUTO: from 2^22 cells, FP32 and 16-bit storage) when
 * nx is a multiple of 32 in [64, 512], the PDF, stress and mask arrays are 16-byte
 * aligned (always with the library's own allocations), the layout fits one block's
 * shared memory (FP64: nx up to 384) and the stress law is not FENE-P.  LBVE_LB_CELLS:
 * the per-cell kernel (one thread per cell, global loads).  Every cell runs the same
 * arithmetic in both, so results are bitwise equal.  -1 for NULL.  A bounded wait of the
 * row pipeline that gives up (a copy that never lands; not expected) makes the next
 * lbve_step / lbve_synchronize return LBVE_ETIMEOUT.
 */
#define LBVE_LB_CELLS 0
#define LBVE_LB_ROWS 1
int lbve_stream_collide_kernel(const lbve_ctx *ctx);

/*
 * Which stress-update kernel (the finite-volume step, Eqs. (continuity)-(source))
 * lbve_step launches (split schedule).  Both march a column of cells through a z-chunk
 * with the tau and u planes staged in a shared-memory ring.  LBVE_FV_PAIRS: 64 x 8
 * columns, each thread updating two neighbouring cells of a row in the two lanes of
 * paired FP32 instructions; taken with schedule PIPELINED (AUTO: from 2^21 cells) for
 * FP32, FP16 and BF16 storage when the solve uses the method's own update (flux and
 * source on; no CTU, tau div u, Giesekus or FENE-P term), nx is a multiple of 4 and the
 * arrays are 16-byte aligned (always with the library's own allocations).
 * LBVE_FV_TILES: 32 x 8 columns, one cell per thread.  Results are bitwise equal.  -1 for
 * NULL.
 */
#define LBVE_FV_TILES 0
#define LBVE_FV_PAIRS 1
int lbve_stress_kernel(const lbve_ctx *ctx);

/*
 * Copy the macroscopic fields to host arrays (each may be NULL): rho (n), u (3n, the
 * physical velocity (j + F/2)/rho of Eq. (macroscopic-velocity) with F = g + F^p),
 * tau (6n), flags (n).  Non-fluid cells read 0.  Page-locked arrays the device can
 * address are written in place by one kernel; other host memory goes through device
 * staging in z-slabs, after one byte per page of it has been written (outputs only:
 * copies into pages never touched before are slow).  Synchronises the stream.
 */
lbve_status lbve_read_fields(lbve_ctx *ctx, double *rho, double *u, double *tau, uint8_t *flags);

/* Same fields into device buffers of FP64 (each may be NULL); asynchronous. */
lbve_status lbve_read_fields_device(lbve_ctx *ctx, double *rho, double *u, double *tau);

/* PDFs f_i (19n, unshifted, FP64) to / from host memory, in the D3Q19 order above
 * (pageable output pages are touched before the copy, as for lbve_read_fields). */
lbve_status lbve_read_pdfs(lbve_ctx *ctx, double *f);
lbve_status lbve_write_pdfs(lbve_ctx *ctx, const double *f);

/* Probe `count` cells (host array of cell indices): out (host, 29 doubles per cell) gets
 * f_0..f_18 (unshifted), rho, u (physical velocity as in lbve_read_fields) and tau (6).
 * Non-fluid cells read f as stored and rho = u = tau = 0.  Synchronises the stream. */
lbve_status lbve_probe(lbve_ctx *ctx, const int64_t *cells, int count, double *out);

/* Fill/drain totals since creation: out[0..5] stress dropped because a destroyed cell
 * had no fluid neighbour, [6] cells destroyed, [7] cells created. */
lbve_status lbve_read_conversions(lbve_ctx *ctx, double out[8]);

/* Particle state: out[0..2] X, [3..5] v, [6..8] w, [9..11] momentum-exchange force
 * and [12..14] torque of the last step, [15..17] fill/drain impulse dP and [18..20]
 * angular impulse dL of the last step, [21] m, [22] I, [23] R. */
lbve_status lbve_read_particle(lbve_ctx *ctx, int id, double out[24]);

/* Momentum-exchange force of the last step per flag value: out[256][3] (host). */
lbve_status lbve_read_body_forces(lbve_ctx *ctx, double *out);

/* Global sums over fluid cells, FP64 on the device: out[0] mass, [1..3] momentum
 * sum f c, [4] fluid cell count, [5] 1 if a NaN/Inf or rho <= 0 was seen. */
lbve_status lbve_reduce(lbve_ctx *ctx, double out[6]);

/* Kernel timing.  While enabled, every kernel that lbve_step launches is bracketed by
 * CUDA events on the context's stream.  lbve_read_kernel_times synchronises the stream
 * and returns, per kernel kind (LBVE_KT_*), the summed device milliseconds and the
 * launch counts since timing was (re)enabled. */
#define LBVE_KT_LB 0        /* stream-collide (split schedule) */
#define LBVE_KT_FV 1        /* finite-volume stress update (split schedule) */
#define LBVE_KT_FUSED 2     /* fused FV(t) + LB(t+1) */
#define LBVE_KT_ME 3        /* momentum exchange + body reduction */
#define LBVE_KT_PARTICLE 4  /* particle update, re-voxelisation, fill/drain */
#define LBVE_KT_COUNT 8
lbve_status lbve_set_kernel_timing(lbve_ctx *ctx, int enable);
lbve_status lbve_read_kernel_times(lbve_ctx *ctx, double ms[LBVE_KT_COUNT], long long launches[LBVE_KT_COUNT]);

/*
 * Time steps on caller-owned device buffers, allocating no device memory.
 *
 * The paper has no counterpart: this serves callers that cannot call cudaMalloc, such
 * as code that runs inside a framework which owns all device memory through its own
 * pool, or a host that forbids allocation after start-up.  Such a caller keeps the
 * state in its own buffers and this call advances it with the split-schedule kernels.
 * The intermediates the kernels need (the velocity field passed from the stream-collide
 * kernel to the stress kernel, and the per-cell neighbour masks derived from the flags
 * at the start of every call) live in fixed file-scope device arrays of
 * 3 * LBVE_NOALLOC_MAX_CELLS doubles and LBVE_NOALLOC_MAX_CELLS 32-bit words (14 MiB in
 * all), which every GPU that loads the library holds until the process exits.
 *
 * Buffers (device, caller-owned, same layouts as a context uses internally), with
 * n = nx*ny*nz and np = n rounded up to a multiple of 64:
 *   f      19 * np PDF storage elements of p->pdf_prec: FP64 stores f_i itself; the
 *          reduced modes store (f_i - w_i rho0) * 2^k (k = 15 for FP16 by default,
 *          else 0; see pdf_scale_log2), w = 1/3, 1/18 (1..6), 1/36 (7..18).  At even t0
 *          slot i of cell r holds f_i(r) (the plain layout); at odd t0 the in-place
 *          (AA) layout of an odd step, i.e. the state after an odd number of steps.
 *   tau_a  6 * np stress values (FP64 in FP64 mode, else FP32) at time t0;
 *   tau_b  6 * np values of scratch for the other stress time level; after the call
 *          the stress at t0 + nsteps is in tau_a if nsteps is even, else in tau_b;
 *   flags  n bytes: 0 fluid, 1 no-slip, LBVE_FLAG_WALL0 + k wall class k < n_wall
 *          (velocities in wall_vel, host, 3 doubles each); particle flags act as
 *          resting walls.  Momentum-exchange forces are not computed by this call.
 *          The call sets the stress of every non-fluid cell to zero in tau_a and tau_b
 *          (a solid cell carries no stress; the stress update relies on it).
 * Schedule: always the split kernels (the per-cell stream-collide and the tiled stress
 * update).  p->schedule must be LBVE_SCHED_AUTO or LBVE_SCHED_SPLIT (LBVE_SCHED_FUSED and
 * LBVE_SCHED_PIPELINED are rejected with EINVAL); p->block_x is honoured as
 * by lbve_create, but schedules recorded by lbve_autotune are not applied and the stress
 * kernel takes its default z-chunk.  None of these choices changes a result.
 * Validation: EINVAL for bad parameters, NULL buffers or more than
 * LBVE_NOALLOC_MAX_CELLS cells.  The first call on each device (with that device
 * current) looks up the address of the static array and keeps it for the life of the
 * process; make that first call before any stream capture.  A reset of the device's
 * primary context (cudaDeviceReset) discards the array and invalidates that address:
 * do not call this entry point on a device after resetting it.  Every call shares the array, which keeps the last call's contents;
 * nothing in it needs to start at zero.  Calls that overlap on the GPU (other streams,
 * other threads) race on it: serialise them.  Enqueues the kernels on cuda_stream and
 * returns without synchronising.  Errors are described by lbve_noalloc_last_error().
 */
#define LBVE_NOALLOC_MAX_CELLS (1 << 19)
lbve_status lbve_step_noalloc(const lbve_params *p, void *f, void *tau_a, void *tau_b, const uint8_t *flags,
                              const double *wall_vel, int n_wall, long long t0, int nsteps, void *cuda_stream);
const char *lbve_noalloc_last_error(void);

/*
 * Residual of a solve (steady-state test): out[0] = |u - u_prev| / |u| (L2 over fluid
 * cells, FP64 with a fixed-shape reduction, so the value does not depend on what else
 * runs), where u is the velocity of the last completed step and u_prev the one seen by
 * the previous call (zero at the first call); out[1] = |u|.  The first call allocates
 * the snapshot buffer.  Synchronises the stream.
 */
lbve_status lbve_residual(lbve_ctx *ctx, double out[2]);

/*
 * Pools: resident solves that advance together.  lbve_pool_step runs each time step as
 * one persistent stream-collide kernel and one persistent stress kernel over a packed
 * list of (solve, block) work items, plus the per-solve momentum-exchange and particle
 * kernels; each cell is computed exactly as in lbve_step, so a solve's result does not
 * depend on the other members.  Members must share the pool's PDF precision and stream.
 * Admission is checked against the pool's device-memory budget (lbve_device_bytes of
 * the member's parameters); the pool never owns or frees member contexts.
 * With graphs enabled (default) the launch sequence of a step call is captured into a
 * CUDA graph and replayed while the membership and step count are unchanged (not on
 * the legacy default stream, which cannot be captured: there the kernels launch
 * directly).
 */
typedef struct lbve_pool lbve_pool;
lbve_status lbve_pool_create(int pdf_prec, size_t budget_bytes, void *cuda_stream, lbve_pool **out);
lbve_status lbve_pool_destroy(lbve_pool *pool);
/* 1 if a solve with these parameters fits the remaining budget, else 0. */
int lbve_pool_fits(const lbve_pool *pool, const lbve_params *p);
/* Errors: ENOMEM (over budget), ESTATE (precision or stream differ, already a member). */
lbve_status lbve_pool_admit(lbve_pool *pool, lbve_ctx *ctx);
lbve_status lbve_pool_remove(lbve_pool *pool, lbve_ctx *ctx);
/* Errors: EUNSTABLE, without stepping, when a member's instability flag (lbve_step) is
 * set: remove the members for which lbve_is_unstable returns 1 and step again. */
lbve_status lbve_pool_step(lbve_pool *pool, int nsteps);
/* Residuals of all members in admission order: 2 doubles each as in lbve_residual. */
lbve_status lbve_pool_residuals(lbve_pool *pool, double *out);
int lbve_pool_size(const lbve_pool *pool);
size_t lbve_pool_bytes_in_use(const lbve_pool *pool);
lbve_status lbve_pool_set_graphs(lbve_pool *pool, int enable);
const char *lbve_pool_last_error(const lbve_pool *pool);

/*
 * Schedule autotuning.  No launch shape changes a result (every cell runs the same
 * arithmetic in whatever block it falls), so the tuner times candidate schedules on the
 * solve's own steps: the solve advances by the steps measured.
 *
 * lbve_autotune (split schedule; LBVE_ESTATE for the fused schedule or a pool member):
 * for every candidate -- stream-collide block width 32, 64 or 128 (up to the width nx
 * needs) times stress z-planes per block at half, one and two times the default --
 * `steps` untimed steps, then `steps` steps timed with CUDA events on the context's
 * stream.  The
 * fastest is kept for this context and recorded in a process-wide table keyed by
 * (precision, nx, ny, nz); contexts created later with that key start from it (unless
 * their params set block_x).  steps <= 0: apply a recorded choice only, measuring
 * nothing.  out may be NULL.
 */
typedef struct {
    int block_x;                 /* chosen stream-collide block width */
    int fv_zchunk;               /* chosen stress z-planes per block */
    int candidates;              /* schedules measured by this call */
    long long steps_taken;       /* steps the context advanced */
    double ms_per_step;          /* chosen schedule, as measured (0 if not measured) */
    double ms_per_step_default;  /* the schedule before the call, as measured */
} lbve_tuning;
lbve_status lbve_autotune(lbve_ctx *ctx, int steps, lbve_tuning *out);

/* Pool tile autotuning.  Members are grouped into classes by nx.  Class by class, in
 * decreasing order of cells, the stream-collide tile width (16, 32, 64 or 128 cells of a
 * 128-thread block, up to the width nx needs) and then the stress tile width (16, 32 or
 * 64 cells of a 256-thread block; FP64: 32) are chosen by coordinate descent, each
 * candidate timed over `steps` pool steps after two untimed calls of `steps` steps (which
 * leave the step graphs of both call parities captured).  The choices are
 * recorded per (precision, nx) and applied to contexts admitted to any pool later.  Every
 * member advances by the steps measured.  The first max_classes classes are reported
 * (arrays of max_classes entries, NULL allowed): nx, chosen tile widths; ms_before /
 * ms_after: pool step time with the tiles before the call and with the choices. */
lbve_status lbve_pool_autotune(lbve_pool *pool, int steps, int max_classes, int *n_classes, int *class_nx,
                               int *lb_tx, int *fv_tx, double *ms_before, double *ms_after);

/*
 * Checkpoint and restore of a solve at a step boundary (for restarts; the paper has no
 * counterpart).  The record holds the raw device state: the PDF storage (19 np elements
 * of the storage type, in the in-place layout of the current step parity), the current
 * stress (6 np reals), the flag field (n bytes, particle cells included), the particle
 * table, the conversion diagnostics and body forces of the last step, the step counter
 * and the stress / velocity ping-pong indices, behind a header naming the grid, the
 * precision and the particle count.  lbve_checkpoint_bytes gives its size.
 * lbve_save copies it into caller-owned host memory (synchronises the stream).
 * lbve_restore overwrites a context created with the same parameters, after
 * lbve_set_geometry with the same no-slip and wall-class cells and the same number of
 * lbve_add_particle calls (their link capacities), and rebuilds the neighbour masks and
 * the particle link lists; stepping it then gives bitwise the results of stepping the
 * saved solve.  The residual snapshot of lbve_residual is not part of the record.
 * Errors: EINVAL (buffer too small, another grid, precision, particle count or static
 * geometry), ESTATE (restore into a pool member), ECUDA.
 */
size_t lbve_checkpoint_bytes(const lbve_ctx *ctx);
lbve_status lbve_save(lbve_ctx *ctx, void *buf, size_t bytes);
lbve_status lbve_restore(lbve_ctx *ctx, const void *buf, size_t bytes);

/* Steps done since the last lbve_init_fields. */
long long lbve_time(const lbve_ctx *ctx);
lbve_status lbve_synchronize(lbve_ctx *ctx);
const char *lbve_last_error(const lbve_ctx *ctx);
const char *lbve_status_string(lbve_status s);

#ifdef __cplusplus
}
#endif
#endif
