/*
 * iblb.h -- C ABI of libiblb, a single-GPU (sm_103a) implementation of the
 * time step of the immersed boundary - lattice Boltzmann (IB-LB) method for
 * wetting of Bellantoni et al., "Immersed boundary - lattice Boltzmann method
 * for wetting problems" (arXiv 2503.20605).
 *
 * One time step (Sec. II) advances a D3Q19 BGK lattice with Guo forcing and
 * bounce-back walls (Sec. II A, eqs. LBE, hydro_var1/2), coupled through the
 * four-point delta kernel (eqs. force_spread, vel_interpolation) to a closed
 * triangulated droplet membrane carrying surface-tension forces (Sec. II B)
 * and the regularised wall interaction Pi(h) that sets the contact angle
 * (Sec. II C, eqs. disjoin-p, A_choice); membrane nodes move by forward Euler.
 *
 * Conventions
 *   - Units: lattice units, dx = dt = 1 (Sec. III).
 *   - Box: nx * ny * nz lattice nodes, periodic in x and y.  With walls on,
 *     layers Z = 0 and Z = nz - 1 are solid (halfway bounce-back, resting
 *     walls) and the fluid is Z = 1 .. nz - 2; the bottom wall plane is
 *     z = 1/2.  With walls off the box is periodic in z too.
 *   - Lattice arrays exchanged through this API cover the FLUID cells only,
 *     layout a[k][z'][y][x] (x fastest), z' = Z - 1 with walls, Z without.
 *   - Populations are absolute f_i (not offsets), velocity order:
 *       0 (0,0,0); 1 (+x) 2 (-x) 3 (+y) 4 (-y) 5 (+z) 6 (-z);
 *       7 (+x+y) 8 (-x-y) 9 (+x-y) 10 (-x+y) 11 (+y+z) 12 (-y-z)
 *       13 (+y-z) 14 (-y+z) 15 (+x+z) 16 (-x-z) 17 (+x-z) 18 (-x+z)
 *     (Tab. I groups; the order inside a group is this library's choice).
 *   - Membrane nodes are (x, y, z) triples in lattice coordinates; faces are
 *     int32 triples of node indices, counter-clockwise seen from outside.
 *
 * Ownership and threading
 *   - Every host pointer argument is owned by the caller and only read (or
 *     written, for outputs) during the call; the library keeps no reference.
 *     Output buffers are caller-allocated with the sizes stated per function.
 *   - A context owns all of its device memory and one CUDA stream of its own.
 *     Work is ordered after the work already queued on the caller's stream
 *     given at creation, and the caller's stream is made to wait for the
 *     context's work before each call returns (stream ordering both ways).
 *   - Calls that return data to the host synchronise; iblb_step does not.
 *   - A context must not be used from two host threads at once.
 *
 * Errors
 *   - Every int-returning function returns IBLB_OK (0) or a negative
 *     IBLB_E_* code and stores a message readable with iblb_last_error().
 *   - Device-side conditions (NaN, a node moving more than half a lattice
 *     unit in one step, a list overflow) set a status word that iblb_sync()
 *     and the data-returning calls report as IBLB_E_UNSTABLE / IBLB_E_OVERFLOW.
 *   - No exception or longjmp crosses the ABI.
 */
#ifndef IBLB_H
#define IBLB_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------- */
#define IBLB_OK 0
#define IBLB_E_ARG -1       /* invalid argument (sizes, tau <= 1/2, ...)      */
#define IBLB_E_MESH -2      /* membrane mesh not closed / not orientable / V<=0 */
#define IBLB_E_NOMEM -3     /* device or host allocation failed               */
#define IBLB_E_CUDA -4      /* a CUDA call failed                             */
#define IBLB_E_UNSTABLE -5  /* NaN, non-positive density or node jump > 0.5  */
#define IBLB_E_TIMEOUT -6   /* a bounded device wait gave up                  */
#define IBLB_E_STATE -7     /* call not valid in the context's state          */
#define IBLB_E_IO -8        /* checkpoint file error                          */
#define IBLB_E_OVERFLOW -9  /* a per-tile or per-column list exceeded its cap */

/* ---- population storage (the arithmetic is FP32 in every case) ---------- */
#define IBLB_STORE_F32 0   /* offsets f_i - w_i rho0 stored as float          */
#define IBLB_STORE_F16 1   /* offsets stored as IEEE half, round-to-nearest   */
#define IBLB_STORE_BF16 2  /* offsets stored as bfloat16, round-to-nearest    */

/* ---- wetting models ------------------------------------------------------ */
#define IBLB_WET_OFF 0     /* no wall interaction                              */
#define IBLB_WET_THETA 1   /* A from theta_eq by eq. A_choice                  */
#define IBLB_WET_RAW 2     /* A given directly                                 */

/* Lattice and fluid (Sec. II A, Sec. III). */
typedef struct {
    int nx, ny, nz;        /* full box in lattice nodes; nx, ny >= 8; nz >= 8 with walls */
    int walls;             /* 1: bounce-back walls at Z = 0 and Z = nz-1; 0: periodic z  */
    double tau_out;        /* BGK relaxation time outside the droplet, > 1/2            */
    double lambda;         /* viscosity ratio mu_in/mu_out (eq. def_lambda); inside
                              tau_in = 1/2 + lambda (tau_out - 1/2); 1 disables the
                              in/out classification                                     */
    double rho0;           /* initial density (Sec. III: 1)                             */
    int storage;           /* IBLB_STORE_*; the same for every droplet of a context     */
    double body_force[3];  /* uniform force density on every fluid cell                 */
} iblb_lattice_desc;

/* Membrane physics (Sec. II B, II C). */
typedef struct {
    double sigma;          /* surface tension                                           */
    int wetting;           /* IBLB_WET_*                                                */
    double theta_eq_deg;   /* equilibrium contact angle, degrees (IBLB_WET_THETA)       */
    double A;              /* interaction strength (IBLB_WET_RAW)                      */
    double xi;             /* regularising length scale xi > 0                          */
    int n, m;              /* exponents of Pi(h), n > m > 1 (the paper uses 6, 3)      */
    double h_min_frac;     /* near-wall guard: h_eff = max(h, h_min_frac * xi); 0 = off */
    int volume_correction; /* 1: after each step rescale the mesh about its node
                              centroid to the initial volume (not in the paper)       */
    double shear_modulus;  /* k_s >= 0 and k_alpha >= 0 of a Skalak membrane energy   */
    double area_modulus;   /* w = k_s/12 (I1^2 + 2 I1 - 2 I2) + k_alpha/12 I2^2 per unit
                              reference area (I1 = 2b, I2 = e^(2a) - 1 with the
                              invariants of eq. strain_inv), added to the droplet's
                              sigma e^a; the reference is the mesh given to
                              iblb_set_membrane.  0, 0: the paper's droplet.  An
                              extension named by the paper's framework (Sec. II B),
                              not used in its results.                                */
} iblb_physics_desc;

/* Observables of one droplet (Sec. III, App. C), FP64. */
typedef struct {
    double mass;           /* sum over fluid cells of sum_i f_i                         */
    double volume;         /* enclosed mesh volume                                      */
    double area;           /* mesh area                                                 */
    double centroid[3];    /* mean of the node positions                                */
    double zmin, zmax;     /* lowest / highest node                                     */
    double theta_R0_deg;   /* angle from the half-height l = (zmax-zmin)/2, eq. angleh,
                              with R0 = radius of the initial volume                    */
    double theta_RV_deg;   /* same with the current volume-equivalent radius           */
    double rc_cut;         /* contact radius, protocol (i): mesh edges crossing the
                              plane z = 1/2 + zcut_frac*R0, mean distance from their
                              centre                                                    */
    double rc_flat;        /* contact radius, protocol (ii): sqrt(chi_eps / pi)         */
    double n_cut;          /* number of edges crossing the protocol (i) plane           */
    double chi_flat;       /* area of the flat lower-half faces, protocol (ii)          */
    int status;            /* IBLB_OK or the pending device status of this droplet      */
    int clamped;           /* nodes clamped by the near-wall guard in the last step     */
} iblb_obs;

/* Per-phase timing slots returned by iblb_get_profile. */
#define IBLB_PH_FORCES 0   /* nodal forces + binning (a1)                               */
#define IBLB_PH_SPREAD 1   /* scan, fill, deterministic gather-spread (a2)              */
#define IBLB_PH_INOUT 2    /* in/out ray casting (a3)                                   */
#define IBLB_PH_LB 3       /* fused stream-collide (a4)                                 */
#define IBLB_PH_ADVECT 4   /* interpolation + advection (a5)                            */
#define IBLB_PH_REDUCE 5   /* FP64 reductions + volume correction (a6)                  */
#define IBLB_NPHASE 6

/* Options for iblb_set_option. */
#define IBLB_OPT_GRAPHS 0     /* 1: replay captured CUDA graphs of one step (or of
                                 IBLB_OPT_GRAPH_CHUNK steps); 0 (default): launch the
                                 kernels of each step directly, which with
                                 IBLB_OPT_PDL measured faster on GB300 (81 against 84 us
                                 per step at 128^3); results are bit-identical           */
#define IBLB_OPT_PROFILE 1    /* 1: record CUDA events around each phase; 2: around the
                                 whole step only; 3: around the stream-collide kernel
                                 only (its time is reported as the IBLB_PH_LB phase);
                                 each adds a host sync per step; 0 (default): off       */
#define IBLB_OPT_LB_BLOCKS_PER_SM 2 /* resident blocks per SM of the persistent
                                 stream-collide kernel (0..8; 0 = as many as fit)       */
#define IBLB_OPT_LB_ROW_MULT 3 /* cell rows per stream-collide group, in units of
                                 max(1, 256 / nx) rows (1..4; 0 = 1); setting it sets
                                 IBLB_OPT_LB_GROUP_CELLS to 0                            */
#define IBLB_OPT_LB_STAGES 4  /* shared-memory stages of the stream-collide pipeline:
                                 the most groups in flight per block (2..8; default 3;
                                 lowered to the most that fit in shared memory)          */
#define IBLB_OPT_FUSED_IB 5   /* 1: the membrane work of a step runs as two cooperative
                                 kernels (forces + spread; advection + volume
                                 correction) with grid barriers between their phases,
                                 reported as the forces and advect phases; 0 (default):
                                 one kernel per stage.  Results are bit-identical
                                 either way; on GB300 the separate kernels are faster. */
#define IBLB_OPT_IB_BLOCKS_PER_SM 6 /* blocks per SM of the two cooperative membrane
                                 kernels (0..8; 0 = as many as fit; default 1)           */
#define IBLB_OPT_SPLIT_LB 7   /* 1: stream-collide groups whose rows cannot meet the
                                 step's band (more than one tile row from the previous
                                 step's band) run on a second stream while the membrane
                                 kernels compute the forces; the others run after the
                                 spread.  0 (default): one stream-collide launch after
                                 the spread.  Results are bit-identical; on GB300 the
                                 two launches compete for the SMs and gain nothing.    */
#define IBLB_OPT_PDL 9         /* 1: the kernels of a step are launched with programmatic
                                 dependent launch (each may start while the previous one
                                 finishes, and waits for it before reading its results);
                                 1 (default); 0: plain stream order.  Bit-identical.     */
#define IBLB_OPT_LB_FAR_BLOCKS_PER_SM 8 /* resident blocks per SM of those far groups
                                 (0..8; 0 = as many as fit; default 1, which leaves room
                                 for the membrane kernels)                               */
#define IBLB_OPT_LB_GROUP_CELLS 10 /* about this many cells per stream-collide group
                                 (whole rows: max(1, round(cells / nx)) rows, at most ny),
                                 in place of IBLB_OPT_LB_ROW_MULT (1..16384; 0 = use the
                                 multiplier; default 768)                                */
#define IBLB_OPT_GRAPH_CHUNK 11 /* steps per replayed CUDA graph (1..64; default 1): with
                                 K > 1, iblb_step runs whole chunks of K steps as one
                                 captured graph each and the rest one step per graph,
                                 so the host launches once per K steps.  Not used while
                                 IBLB_OPT_PROFILE is on.  Results are bit-identical.    */

typedef struct iblb_ctx iblb_ctx;

/* Library version string (static storage). */
const char *iblb_version(void);

/* Message of the last error on ctx (ctx may be NULL for creation errors);
 * static or context-owned storage, valid until the next call on ctx. */
const char *iblb_last_error(const iblb_ctx *ctx);

/* Eq. A_choice: A = sigma (m-1)(n-1) / ((n-m) xi) (1 + cos theta_eq).
 * Writes *A; IBLB_E_ARG if xi <= 0 or n <= m. */
int iblb_wetting_A(double sigma, double theta_eq_deg, double xi, int n, int m, double *A);

/* Create a context holding one droplet (lattice + membrane) on the current
 * CUDA device.  stream: cudaStream_t of the caller (NULL = legacy default).
 * The lattice starts at rest, f_i = w_i rho0 (Sec. III).  The membrane is set
 * with iblb_set_membrane.  IBLB_E_ARG on invalid descriptors. */
int iblb_create(const iblb_lattice_desc *lat, const iblb_physics_desc *phys, void *stream,
                iblb_ctx **out);

/* Create a context holding n independent droplets with their own boxes and
 * parameters (arrays of n descriptors, all with the same storage).  Each
 * phase of a step runs as one launch over all droplets; a droplet of a batch
 * evolves bitwise as it would alone. */
int iblb_batch_create(int n, const iblb_lattice_desc *lat, const iblb_physics_desc *phys,
                      void *stream, iblb_ctx **out);

/* Free all device and host memory of ctx (NULL is ignored). */
void iblb_destroy(iblb_ctx *ctx);

/* Number of droplets, and for droplet k its fluid cells and membrane sizes. */
int iblb_info(const iblb_ctx *ctx, int k, int *n_drops, int64_t *cells, int *n_nodes, int *n_tri);

/* Set the membrane of droplet k (Sec. II A: closed triangular mesh).
 * xyz: host, 3*n_nodes doubles; tri: host, 3*n_tri int32, CCW from outside.
 * The mesh must be closed and orientable with Euler characteristic 2 and
 * positive volume (IBLB_E_MESH otherwise).  Records the initial volume V0.
 * All membranes of a batch must be set before the first step; calling it
 * again replaces the membrane (and resets V0). */
int iblb_set_membrane(iblb_ctx *ctx, int k, const double *xyz, int n_nodes, const int32_t *tri,
                      int n_tri);

/* Host-only check of a membrane mesh, the one iblb_set_membrane applies
 * (Sec. II A: the droplet is a closed triangular mesh; the in/out test and
 * the volume need it closed and consistently oriented).  No context and no
 * GPU needed.  xyz: host, 3*n_nodes doubles; tri: host, 3*n_tri int32.
 * Returns IBLB_OK and writes the enclosed volume to *volume (if not NULL),
 * IBLB_E_MESH with the reason in iblb_last_error(NULL) when the mesh is not
 * closed, orientable, of Euler characteristic 2, with every node used,
 * finite and of positive volume (faces counter-clockwise seen from
 * outside), and IBLB_E_ARG for NULL arrays. */
int iblb_check_mesh(const double *xyz, int n_nodes, const int32_t *tri, int n_tri, double *volume);

/* Overwrite / read the node positions of droplet k (host, 3*n_nodes doubles,
 * x, y, z per node; pinned host memory makes the transfer asynchronous up to
 * the call's return).  iblb_set_nodes makes the positions final (no volume
 * correction pending) and returns once xyz has been copied, so the caller may
 * reuse it; the device work it queued runs in stream order.  iblb_get_nodes
 * returns the positions with any pending volume correction applied and
 * synchronises the context's stream.  IBLB_E_STATE for a droplet without a
 * membrane; CUDA errors as elsewhere. */
int iblb_set_nodes(iblb_ctx *ctx, int k, const double *xyz);
int iblb_get_nodes(iblb_ctx *ctx, int k, double *xyz);

/* Overwrite / read the populations of droplet k: host, 19*cells doubles,
 * absolute f_i, fluid-cell layout (see Conventions).  Values are rounded to
 * the context's storage on set. */
int iblb_set_populations(iblb_ctx *ctx, int k, const double *f);
int iblb_get_populations(iblb_ctx *ctx, int k, double *f);

/* Density and velocity of droplet k at the end of the last step, evaluated
 * from the stored post-collision populations and that step's force density:
 * rho = sum_i f*_i, U = (sum_i c_i f*_i - F/2) / rho (equal to eq. hydro_var2
 * of the step).  rho: cells doubles, u: 3*cells doubles ([k][cell]). */
int iblb_get_macros(iblb_ctx *ctx, int k, double *rho, double *u);

/* Evaluate, for the current node positions and without advancing time, the
 * nodal forces (Sec. II B, II C), the spread force density (eq. force_spread)
 * and, with lambda != 1, the in/out classification of every cell. */
int iblb_compute_forces(iblb_ctx *ctx);

/* Results of the last force evaluation (iblb_compute_forces or a step) for
 * droplet k: phi (3*n_nodes doubles), F (3*cells doubles, [k][cell], body
 * force included), inside (cells bytes, 1 inside / 0 outside). */
int iblb_get_node_forces(iblb_ctx *ctx, int k, double *phi);
int iblb_get_force_density(iblb_ctx *ctx, int k, double *F);
int iblb_get_inside(iblb_ctx *ctx, int k, uint8_t *inside);

/* Advance every droplet by nsteps time steps (asynchronous on the context's
 * stream; replays a captured graph per step unless IBLB_OPT_GRAPHS is 0). */
int iblb_step(iblb_ctx *ctx, int nsteps);

/* Wait for the context's work; returns the device status (IBLB_OK,
 * IBLB_E_UNSTABLE or IBLB_E_OVERFLOW) and clears it. */
int iblb_sync(iblb_ctx *ctx);

/* Run ONE time step (the same work as iblb_step(ctx, 1), launched eagerly)
 * with tracing on: every warp of the step's kernels records the GPU's global
 * timer once its wait on the previous kernel returned (programmatic dependent
 * launch), and a one-warp marker kernel launched after the step does the
 * same.  Synchronises the context's stream.  out (host, IBLB_TRACE_KERNELS x
 * 5 doubles, kernel-major in the order of IBLB_TRACE_*) receives per kernel,
 * in microseconds from the earliest stamp of the step: the first, median and
 * last warp start, the kernel's end = the first start of the next kernel that
 * ran (or of the marker), which comes after its last warp's exit, and the
 * number of warps recorded (0, and NaN times, for a kernel that did not run,
 * such as the volume correction with none requested).  The first call
 * allocates a 1.5 MB stamp buffer, freed by iblb_destroy.  Only the
 * one-kernel-per-stage path is traced (the cooperative kernels of
 * IBLB_OPT_FUSED_IB record nothing), and with IBLB_OPT_SPLIT_LB the two
 * stream-collide launches share their stamps.  The stamps are separate
 * instantiations of the kernels, launched only by this call: iblb_step runs
 * none of their code.  Not thread-safe: trace one context at a time.
 * Returns IBLB_E_ARG for a null out; CUDA errors as elsewhere. */
#define IBLB_TRACE_KERNELS 5
#define IBLB_TRACE_FORCE 0    /* node forces and tile lists */
#define IBLB_TRACE_SPREAD 1   /* deterministic spread */
#define IBLB_TRACE_LB 2       /* fused stream-collide */
#define IBLB_TRACE_INTERP 3   /* interpolation and advection */
#define IBLB_TRACE_VC 4       /* volume correction */
int iblb_trace_step(iblb_ctx *ctx, double *out);

/* Observables of droplet k (synchronises).  zcut_frac: protocol (i) plane
 * height over R0 (the paper's optimum 0.05); eps_flat: protocol (ii)
 * flatness parameter (the paper's optimum 0.1). */
int iblb_observe(iblb_ctx *ctx, int k, double zcut_frac, double eps_flat, iblb_obs *out);

/* Observables of every droplet of the context, out[ndrops] (synchronises);
 * one pass over the lattice for all the masses. */
int iblb_observe_all(iblb_ctx *ctx, double zcut_frac, double eps_flat, iblb_obs *out);

/* IBLB_OPT_* switches; IBLB_E_ARG for unknown options or values. */
int iblb_set_option(iblb_ctx *ctx, int option, int value);

/* Accumulated per-phase device time (ms, IBLB_NPHASE doubles), whole-step
 * device time and number of profiled steps since the last reset.  Times are
 * taken with CUDA events on the context's stream while IBLB_OPT_PROFILE is on. */
int iblb_get_profile(iblb_ctx *ctx, double *phase_ms, double *step_ms, int64_t *steps);
int iblb_reset_profile(iblb_ctx *ctx);

/* Time candidate launch shapes of the stream-collide kernel on this context's
 * lattice (a few steps each, state restored afterwards), keep the fastest and
 * append it to the text file cache_path (NULL: no cache).  A cached entry for
 * the same shape class is used without timing.  Results are bitwise
 * identical for every candidate. */
int iblb_autotune(iblb_ctx *ctx, const char *cache_path);

/* Checkpoint: write / read the complete dynamic state (populations, nodes,
 * V0, the volume correction computed in the last step, step counter) of
 * every droplet to / from a binary file.  Loading needs
 * a context created with the same descriptors and membranes.  A resumed run
 * is bitwise identical to an uninterrupted one. */
int iblb_save(iblb_ctx *ctx, const char *path);
int iblb_load(iblb_ctx *ctx, const char *path);

/* Stateless mesh observables on DEVICE arrays (same definitions as
 * iblb_observe without the mass): d_xyz 3*n_nodes doubles (xyz triples),
 * d_tri 3*n_tri int32 (node indices), results written to the HOST array
 * out[13] in the order of iblb_obs from volume to chi_flat (volume, area,
 * centroid[3], zmin, zmax, theta_R0_deg, theta_RV_deg, rc_cut, rc_flat,
 * n_cut, chi_flat).  R0 > 0 is the reference radius of eq. angleh.
 * Allocates its scratch with cudaMallocAsync on `stream` (NULL = legacy
 * default stream), frees it the same way and synchronises the stream. */
int iblb_mesh_observe_dev(const double *d_xyz, int n_nodes, const int32_t *d_tri, int n_tri,
                          double R0, double zcut_frac, double eps_flat, void *stream,
                          double *out);

/* The same observables as iblb_mesh_observe_dev, with the same arguments and
 * output, computed without allocating any memory: the scratch is a fixed
 * array in device global memory, one per device.  The paper has no
 * counterpart to this call; it serves callers that cannot allocate device
 * memory at that moment (all free memory held by a caching allocator, or an
 * out-of-memory handler).
 *   Limit: n_tri <= 1,048,576 and n_nodes <= 524,288; larger meshes return
 *   IBLB_E_ARG without touching the device.
 *   Nothing needs to be zeroed beforehand.
 *   Set-up: the first call in a CUDA context (with that device current)
 *   loads the library's array and observation kernels into the context
 *   (CUDA loads modules lazily, and loading allocates device memory) and
 *   looks up the array's address with cudaGetSymbolAddress.  Only that first
 *   call may allocate, so make it early, while device memory is still free,
 *   and before capturing any stream.  The address is kept with the identity
 *   of its context; a new context on the device (after cudaDeviceReset, say)
 *   gets the set-up again.  Any CUDA error returns IBLB_E_CUDA.
 *   Not reentrant: calls in flight at the same time on the same device (other
 *   host threads, other streams) share the array and race.  Each call
 *   synchronises `stream` before it returns. */
int iblb_mesh_observe_dev_noalloc(const double *d_xyz, int n_nodes, const int32_t *d_tri, int n_tri,
                                  double R0, double zcut_frac, double eps_flat, void *stream,
                                  double *out);

/* Self-test of the bounded waits (no counterpart in the paper).  Every wait
 * of the stream-collide pipeline on an mbarrier gives up after a cycle limit
 * (about 2 s) and reports IBLB_E_TIMEOUT instead of hanging.  This call runs
 * that same wait, with a limit of `cycles` SM clock cycles (1e3 .. 1e10), on
 * a barrier that nothing completes, on `stream` (synchronised before the
 * call returns).  Returns IBLB_E_TIMEOUT when every waiting thread gave up
 * (the expected outcome), IBLB_E_ARG for a limit out of range, IBLB_E_CUDA
 * if a CUDA call failed, IBLB_E_STATE for any other outcome. */
int iblb_selftest_wait_timeout(long long cycles, void *stream);

/* ---- learned warm start ---------------------------------------------------
 * Not in the paper: a network that predicts the equilibrium shape so that a
 * run can start from it instead of from a sphere.  The shape is the App. B
 * parametrisation: the radial distance r = G(phi) of the surface from the
 * droplet's centre (node centroid), phi the polar angle from +z, made
 * dimensionless as g = G / R0 and averaged over the azimuth (as in eq.
 * L2-error_equilibrium), sampled at nphi polar angles phi_k = (k + 1/2) pi /
 * nphi (nphi = 64 for the network).  These four calls need no GPU.          */

/* Profile of a mesh: nodes xyz[3 * n_nodes] (host); node j falls in bin
 * floor(phi_j nphi / pi); g[k] = mean radial distance of the bin's nodes / R0;
 * empty bins interpolate linearly between the nearest filled bins (constant
 * beyond the first / last).  Writes g[nphi].  IBLB_E_ARG on bad arguments,
 * IBLB_E_MESH if every node sits at the centroid. */
int iblb_mesh_profile(const double *xyz, int n_nodes, double R0, int nphi, double *g);

/* Deform a sphere-like closed mesh (xyz[3 * n_nodes], faces tri[3 * n_tri],
 * host) to the profile g[nphi]: each node moves onto the surface of
 * revolution r = R0 g(phi) about the centroid (g linear between samples,
 * constant beyond the end samples), keeping its azimuth and its fraction of
 * the surface area measured from the top pole, so that nodes stay evenly
 * spread; the result is scaled about the centroid to the input mesh's
 * enclosed volume, centred at (cx, cy) and shifted so that its lowest node
 * is at z = z_bottom.  Writes xyz_out[3 * n_nodes].  IBLB_E_ARG /
 * IBLB_E_MESH on bad input (non-positive g, bad indices, non-positive
 * volume). */
int iblb_deform_mesh(const double *g, int nphi, double R0, const double *xyz, int n_nodes,
                     const int32_t *tri, int n_tri, double cx, double cy, double z_bottom,
                     double *xyz_out);

/* The spherical-cap start of Sec. III B as a profile for iblb_deform_mesh:
 * g[k] = G(phi_k) / R0, phi_k = (k + 1/2) pi / nphi, of the exact spherical
 * cap with contact angle theta_eq_deg (0 < theta < 180) and the volume of
 * the unit sphere (App. B normalisation), measured from the centroid of the
 * cap's surface (curved part and base disc, weighted by area).  Host only.
 * IBLB_E_ARG on bad arguments. */
int iblb_cap_profile(double theta_eq_deg, int nphi, double *g);

/* Message of the last failed iblb_mesh_profile / iblb_deform_mesh /
 * iblb_cap_profile call of this thread. */
const char *iblb_warmstart_last_error(void);

/* The network: multilayer perceptron 3 -> 256 -> 256 -> 256 -> 64, tanh
 * hidden units, linear output g at the 64 polar samples.  Inputs per sample:
 * (theta_eq in degrees, R0, lambda), mapped to the features
 * ((theta_eq - 90) / 70, (R0 - 16) / 8, log10 lambda).  Parameters: one
 * float vector, layer by layer W_l (out x in, row major) then b_l
 * (iblb_mlp_param_count() = 149056 values).  The three 256-input layers run
 * on the tensor cores (tcgen05, BF16 operands, FP32 accumulation); the
 * input layer, the reductions and Adam in FP32.  An iblb_mlp owns its device
 * memory and works on the stream given at creation; it must not be used from
 * two host threads at once. */
typedef struct iblb_mlp iblb_mlp;

int64_t iblb_mlp_param_count(void);

/* Create from initial parameters (host, n_params = iblb_mlp_param_count());
 * max_batch (1 .. 2^20) bounds the batch of iblb_mlp_grad / iblb_mlp_train
 * and the chunk of iblb_mlp_predict.  Adam's moments start at zero. */
int iblb_mlp_create(const float *params, int64_t n_params, int max_batch, void *stream,
                    iblb_mlp **out);
void iblb_mlp_destroy(iblb_mlp *m);
const char *iblb_mlp_last_error(const iblb_mlp *m);

/* Copy the current FP32 parameters to out[n] (n = iblb_mlp_param_count()). */
int iblb_mlp_get_params(iblb_mlp *m, float *out, int64_t n);

/* Inference: x[3 * S] raw inputs (host) -> y[64 * S] (host).  Any S >= 1
 * (processed in chunks of max_batch).  lambda must be > 0. */
int iblb_mlp_predict(iblb_mlp *m, const double *x, int S, double *y);

/* Loss L = mean over the S x 64 outputs of (yhat - y)^2 and its gradient
 * with respect to the parameters, for one batch (1 <= S <= max_batch):
 * grad[iblb_mlp_param_count()] and *loss (host).  Parameters unchanged. */
int iblb_mlp_grad(iblb_mlp *m, const double *x, const double *y, int S, double *grad, double *loss);

/* Training: `epochs` passes over the S samples (x[3 * S], y[64 * S], host),
 * each in a fresh order (Fisher-Yates with a splitmix64 stream from `seed`)
 * cut into floor(S / batch) batches; one Adam step per batch (beta1 0.9,
 * beta2 0.999, eps 1e-8, learning rate lr, bias-corrected; the step counter
 * continues across calls).  loss_per_epoch[epochs] (may be NULL) receives
 * the mean batch loss of each epoch.  IBLB_E_TIMEOUT if a bounded wait in
 * the tensor-core kernel gave up. */
int iblb_mlp_train(iblb_mlp *m, const double *x, const double *y, int S, int epochs, int batch,
                   double lr, uint64_t seed, double *loss_per_epoch);

#ifdef __cplusplus
}
#endif
#endif
