/*
 * osbli.h -- C ABI of the B300-native (sm_103a) residual / RK-stage path of the OpenSBLI method
 * (Lusher, Jammy & Sandham, arXiv:2007.14933).
 *
 * What one RK step computes (paper sections):
 *   - compressible Navier-Stokes residual (Sec. 2.1, Eqs. 1-7) on a structured grid, curvilinear
 *     through metric terms evaluated once with the 4th-order central / one-sided schemes
 *     (Sec. 2.6-2.7, Eqs. 28-33);
 *   - convective terms by characteristic-space WENO5-JS, WENO-Z, TENO5 or TENO6 reconstruction
 *     with a Roe-averaged eigensystem and local Lax-Friedrichs splitting (Sec. 2.2 algorithm,
 *     Eqs. 9-27), or 4th-order central differences (Sec. 2.6);
 *   - viscous and heat-flux terms by 4th-order central differences (Eqs. 4-5, 28-33);
 *   - the low-storage 3-stage RK update dU = A dU + dt R, U = U + B dU (Sec. 2.8, Eqs. 36-38);
 *   - boundary conditions through ghost points (Sec. 3.1.3, Eqs. 40-46; Sec. 6 set-up).
 *
 * Data layout at the boundary: the state is five conserved variables (rho, rho u, rho v, rho w,
 * rho E) as structure of arrays [5][nz][ny][nx], FP64, x fastest, contiguous.  Pointers given to
 * osbli_set_state / osbli_get_state / osbli_residual / osbli_set_boundary_data may be host or
 * device pointers (unified addressing; page-locked host memory for asynchronous copies).  The
 * library owns every buffer it allocates; the caller owns every pointer it passes in and may
 * reuse it when the call returns.
 *
 * Errors: every int-returning call returns OSBLI_OK (0) or a negative code; osbli_last_error()
 * returns a message for the last failure on that handle.  No call throws.  A handle is not
 * thread-safe; different handles are independent.
 */
#ifndef OSBLI_H
#define OSBLI_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
    OSBLI_OK = 0,
    OSBLI_EINVAL = -1,     /* invalid argument or parameter combination */
    OSBLI_ENOMEM = -2,     /* device allocation failed */
    OSBLI_ECUDA = -3,      /* a CUDA call failed (message in osbli_last_error) */
    OSBLI_ENONFINITE = -4, /* the state became non-finite during osbli_rk_step */
    OSBLI_ETIMEOUT = -5,   /* a bounded device-side wait gave up */
    OSBLI_ESTATE = -6      /* stepping before osbli_set_state / missing face data */
};

/* convective scheme (Sec. 2.2-2.6) */
enum { OSBLI_CENTRAL4 = 0, OSBLI_WENO5JS = 1, OSBLI_TENO5 = 2, OSBLI_WENO5Z = 3, OSBLI_TENO6 = 4 };
/* time integrator (Sec. 2.8, Eqs. 36-38): low-storage 2N Runge-Kutta, 3rd order in 3 stages
 * (Williamson) or 4th order in 5 stages (Carpenter & Kennedy); or the 3rd-order
 * strong-stability-preserving scheme of Gottlieb & Shu (1998) in its convex form
 * (U1 = U^n + dt R(U^n), U2 = 3/4 U^n + 1/4 (U1 + dt R(U1)), U^{n+1} = 1/3 U^n + 2/3 (U2 + dt
 * R(U2)); the second register holds U^n, so the storage is the same two arrays) */
enum { OSBLI_RK3 = 0, OSBLI_RK4 = 1, OSBLI_SSPRK3 = 2 };

/* boundary conditions per direction and side (Sec. 3.1.3, Sec. 5-6 set-ups):
 *   PERIODIC   both sides of a direction must be periodic together
 *   ZEROGRAD   ghosts copy the boundary node (zero-order extrapolation; also used as outlet)
 *   WALL       isothermal no-slip wall on the boundary node (Eqs. 40-46), temperature T_wall
 *   DIRICHLET  ghosts and boundary node from osbli_set_boundary_data (rho, u, v, w, p)
 *   INFLOW     ghosts and boundary node: u, v, w, T from osbli_set_boundary_data (slot 0 unused),
 *              pressure extrapolated from the first interior node, rho = gamma Ma^2 p / T
 *   ADIABATIC  no-slip wall with zero heat flux (the laminar channel of Sec. 5.4): ghost
 *              temperatures mirror the interior; after each stage the wall node's temperature
 *              makes the one-sided 4th-order derivative vanish, (48T1 - 36T2 + 16T3 - 3T4)/25 */
enum { OSBLI_PERIODIC = 0, OSBLI_ZEROGRAD = 1, OSBLI_WALL = 2, OSBLI_DIRICHLET = 3,
       OSBLI_INFLOW = 4, OSBLI_ADIABATIC = 5 };

/* arithmetic of the reconstruction (Sec. 2.2-2.5) */
enum { OSBLI_FP64 = 0, OSBLI_MIXED = 1 };

typedef struct osbli osbli_t;

typedef struct {
    int nx, ny, nz;            /* interior points; 1 marks an inactive direction (Sod: 400,1,1);
                                  an active non-periodic direction needs >= 5 points, a periodic
                                  one >= 3 */
    double gamma, Re, Pr, Ma;  /* Re <= 0: inviscid (no viscous / heat-flux terms) */
    double dt;                 /* fixed time step */
    int scheme;                /* OSBLI_CENTRAL4 | OSBLI_WENO5JS | OSBLI_TENO5 | OSBLI_WENO5Z (Eq. 22) |
                                  OSBLI_TENO6 (K = 6: Eq. 27's tau_6, the 4-point candidate on
                                  i..i+3, linear weights of the 6-point reconstruction; same
                                  i-2..i+3 stencil and ghost width) */
    double teno_ct;            /* TENO cut-off C_T (Eq. 24), e.g. 1e-5 (TENO5 and TENO6) */
    int bc[3][2];              /* bc[direction][side], side 0 = low index */
    double T_wall;             /* isothermal wall temperature (Eq. 41) */
    double sutherland_ratio;   /* T_s/T_ref of Eq. 6; <= 0: constant mu = 1 */
    int precision;             /* OSBLI_FP64 | OSBLI_MIXED */
    int sensor;                /* 1: learned shock sensor gates the characteristic vs central
                                  fluxes (precision OSBLI_MIXED, a WENO/TENO scheme, uniform or
                                  rectilinear grid); 0: off */
    double h[3];               /* grid spacing per direction when coords == NULL */
    double L[3];               /* period of each periodic direction (coordinate unwrapping) */
    int rk;                    /* OSBLI_RK3 (3 stages, default) | OSBLI_RK4 (5 stages) |
                                  OSBLI_SSPRK3 (3 stages) */
    double force[3];           /* body force per unit volume on the momentum; its work f.u enters
                                  the energy equation (0, 0, 0: none) */
} osbli_params;

/* Create a solver for one grid.  coords: NULL (uniform grid, spacing h) or node coordinates of
 * the interior points, host memory, [3][nz][ny][nx] (x, y, z components); the metric terms are
 * computed on the device once (Sec. 2.7).  cuda_stream: the cudaStream_t every call enqueues
 * on (NULL: the handle creates its own blocking stream, ordered with the legacy default
 * stream).  On success *out receives the handle.  Errors: EINVAL (bad sizes/parameters),
 * ENOMEM, ECUDA. */
int osbli_create(const osbli_params *p, const double *coords, void *cuda_stream, osbli_t **out);

/* Release every device buffer of the handle.  NULL is ignored. */
void osbli_destroy(osbli_t *h);

/* Face data of a DIRICHLET or INFLOW face: [5][plane], plane = interior points of the two other
 * directions, lower direction fastest.  Copied in.  Errors: EINVAL (face is neither). */
int osbli_set_boundary_data(osbli_t *h, int dir, int side, const double *prims);

/* Copy a state in ([5][nz][ny][nx]).  Errors: EINVAL, ECUDA. */
int osbli_set_state(osbli_t *h, const double *U);

/* Copy the current state out (same layout).  Synchronises the handle's stream. */
int osbli_get_state(osbli_t *h, double *U);

/* Advance nsteps RK3 steps (3 stages each: ghost fill, residual, register update, boundary
 * nodes).  The first call captures one step into a CUDA graph that later calls replay.
 * Synchronises and checks the device error word before returning: ENONFINITE when any interior
 * value became non-finite, ESTATE before osbli_set_state, EINVAL for nsteps < 0. */
int osbli_rk_step(osbli_t *h, int nsteps);

/* Residual R(U) (the right-hand side dU/dt of Eqs. 1-3) of the current state, written to R in
 * the state layout.  Used for single-stage parity checks.  Synchronises. */
int osbli_residual(osbli_t *h, double *R);

/* Diagnostics of the current state (deterministic reductions over interior points):
 * out[0..4] = sum of the conserved variables, out[5] = mean kinetic energy 1/2 rho |u|^2,
 * out[6] = max Mach number, out[7] = min density, out[8] = min pressure, out[9] = fraction of
 * cells gated to the characteristic flux by the learned sensor at the last evaluation (0 when
 * the sensor is off), out[10..12] = fraction of interfaces along x, y, z taking the
 * characteristic flux under the sensor's gate (strong jumps aside), out[13..15] = 0. */
int osbli_diagnostics(osbli_t *h, double out[16]);

/* Time each kernel launch of one residual evaluation (ghost fill per direction, primitives,
 * convective flux difference per direction, viscous fluxes, viscous divergence) with CUDA events
 * on the handle's stream, averaged over reps >= 1 repetitions.  ms[i] (host, max entries)
 * receives the mean duration of launch i in milliseconds; osbli_profile_name(h, i) names it.
 * Returns the number of launches (> 0) or a negative error code.  The state is unchanged. */
int osbli_profile_residual(osbli_t *h, int reps, double *ms, int max);

/* Name of launch i of the last osbli_profile_residual on h ("" when out of range). */
const char *osbli_profile_name(const osbli_t *h, int i);

/* ---- learned shock sensor (an addition to the method: the paper has no sensor) --------------
 * Per cell, features from the 3x3x3 neighbourhood (rho_n/rho_c - 1, (u_n - u_c)/a_c for three
 * components, p_n/p_c - 1: 135 values, padded to 144 BF16 per row) feed an MLP
 * 135 -> 32 -> 32 -> 1 (ReLU, ReLU, sigmoid) evaluated on BF16 tensor cores once per RK step.
 * Cells with probability above the threshold are flagged, and an interface takes the TENO/WENO characteristic flux when either adjacent cell
 * is gated (or its stencil holds a strong jump); otherwise the 4th-order central flux.
 * Weights: FP32 parameter vector of OSBLI_SENSOR_NPARAM values, W1[32][135], b1[32], W2[32][32],
 * b2[32], w3[32], b3 (host memory). */
#define OSBLI_SENSOR_NPARAM 5441
#define OSBLI_SENSOR_NFEAT 144

/* Install weights and decision threshold (probability in (0,1)) on a handle created with
 * params.sensor = 1; required before stepping.  Errors: EINVAL. */
int osbli_sensor_set_weights(osbli_t *h, const float *w, float threshold);

/* Install a fixed cell gate in place of the network's decision (handle created with
 * params.sensor = 1): flags [nz][ny][nx] bytes, host or device, nonzero = the cell is flagged.
 * The gate rule is the learned one -- an interface takes the characteristic flux when either
 * adjacent cell is flagged (a ghost cell takes the flag of its periodic image, else of the
 * nearest interior cell of its line) or its six-node stencil holds an adjacent pressure or
 * density ratio above 1.5, and the central 4th-order interface flux
 * [7 (F_i + F_{i+1}) - (F_{i-1} + F_{i+2})] / 12 (Sec. 2.6, Eq. 28 in flux form) otherwise --
 * and stays until the next osbli_sensor_set_gate or osbli_sensor_set_weights; no inference runs
 * while it holds.  Copied in; synchronises.  Errors: EINVAL (no sensor on the handle), ECUDA. */
int osbli_sensor_set_gate(osbli_t *h, const uint8_t *flags);

/* Training labels of the current state (TENO5 handles, any precision): 1 for a cell whose FP64
 * TENO5 residual used an interface where a candidate stencil was cut and the cut moved the
 * reconstruction by more than 5 % of the stencil's range and by more than 1e-5 x the interface's
 * mean density x its largest acoustic speed (a floor against rounding-noise cut-offs).  labels: [nz][ny][nx] bytes, host or
 * device.  Allocates temporary device memory. */
int osbli_sensor_labels(osbli_t *h, uint8_t *labels);

/* Features of the current state: d_feats device pointer, [nz*ny*nx][144] BF16 (the caller
 * allocates nz*ny*nx*288 bytes). */
int osbli_sensor_features(osbli_t *h, void *d_feats);

/* Sensor probabilities of the current state, [nz][ny][nx] FP32, host or device pointer. */
int osbli_sensor_probs(osbli_t *h, float *probs);

/* Sensor probabilities of n feature rows: d_feats [n][144] BF16 device, w host parameter vector,
 * d_probs [n] FP32 device.  Legacy default stream; synchronises the device. */
int osbli_mlp_forward(const void *d_feats, long long n, const float *w, float *d_probs);

/* One full-batch gradient of the mean weighted binary cross-entropy
 * L = -mean(pos_weight y log p + (1 - y) log(1 - p)) on the GPU kernels used for training:
 * d_feats [n][144] BF16 device, d_labels [n] bytes device, w host parameter vector, grad host
 * (OSBLI_SENSOR_NPARAM), *loss host.  Allocates temporary device memory. */
int osbli_mlp_grad(const void *d_feats, const uint8_t *d_labels, long long n, float pos_weight,
                   const float *w, float *grad, double *loss);

/* Train with Adam (beta 0.9 / 0.999) for `steps` mini-batches of `batch` rows (multiple of 16)
 * drawn by a counter-based hash of (seed, step, row); w (host, in/out) holds the FP32 master
 * parameters; loss_hist (host, steps values, may be NULL) the batch losses.  Runs on the legacy
 * default stream.  Allocates temporary device memory. */
int osbli_mlp_train(const void *d_feats, const uint8_t *d_labels, long long n, int steps, int batch,
                    float lr, float pos_weight, unsigned seed, float *w, float *loss_hist);

/* Kernel launches one RK step enqueues (for launch accounting). */
int osbli_launches_per_step(const osbli_t *h);

/* Largest ghosted grid osbli_residual_noalloc accepts: (nx+6)(ny+6)(nz+6) nodes, counting the
 * 6 ghost layers only on directions with more than one point (e.g. 34^3, 250^2 x 1). */
#define OSBLI_NOALLOC_MAX_NODES 65536

/* Residual R(U) of a state held in caller memory, computed without allocating device memory.
 * The paper has no counterpart: this is for callers that may not call cudaMalloc (a host
 * application that gives all device memory to its own pool, a real-time loop that cannot take
 * the synchronisation an allocation may imply, a plug-in whose framework forbids allocation).
 * The intermediate arrays live in one static device array of 30 doubles x
 * OSBLI_NOALLOC_MAX_NODES (15.7 MB) that every GPU using the library holds until the process
 * exits.  Same arithmetic as osbli_residual.
 *   p        parameters as for osbli_create (every scheme, Sutherland viscosity, body force);
 *            restricted to a uniform grid (spacing h), faces PERIODIC, ZEROGRAD or WALL
 *            (T_wall > 0) only -- no face data, so no DIRICHLET / INFLOW / ADIABATIC faces --,
 *            precision OSBLI_FP64 and no sensor (the mixed-precision path is not offered here)
 *   d_U      device pointer, [5][nz][ny][nx] FP64 state (read)
 *   d_R      device pointer, [5][nz][ny][nx] FP64 residual (written)
 *   stream   cudaStream_t the work is enqueued on; the call synchronises it before returning.
 * Returns OSBLI_OK, EINVAL (bad parameters, or a grid beyond OSBLI_NOALLOC_MAX_NODES: the message
 * from osbli_last_error(NULL) names both sizes), ENONFINITE (the residual written to d_R holds a
 * non-finite value) or ECUDA.  The first call on a device looks up
 * the array's device address (cudaGetSymbolAddress) with that device current; make that first
 * call before any stream capture.  All calls share the array and it keeps the previous call's
 * contents (the ghosted state is cleared at the start of each call); calls whose GPU work
 * overlaps -- other streams or other host threads -- race on it and must be serialised by the
 * caller. */
int osbli_residual_noalloc(const osbli_params *p, const double *d_U, double *d_R, void *stream);

/* Measured FP64 FMA throughput of the current device in TFLOP/s (independent DFMA chains; the
 * denominator of the FP64 path's ALU roofline).  A measurement helper: the paper has no
 * counterpart.  Uses the legacy default stream and a small temporary device buffer. */
int osbli_fp64_peak(double *tflops);

/* Same for FP32 FMAs (denominator of the mixed path's reconstruction kernels). */
int osbli_fp32_peak(double *tflops);

/* Message of the last failure on h (or of the last failed osbli_create when h is NULL). */
const char *osbli_last_error(const osbli_t *h);

/* ---------------------------------------------------------------------------------------------
 * Ensembles: many independent problems advanced together (the paper's 2D Riemann tubes of
 * Sec. 5.2 run as a batch).  Every phase of an RK stage is one launch over the blocks of all
 * members, and a step is one CUDA graph, so the launch count does not grow with the member count
 * and members of very different sizes share the GPU.  Each member computes exactly what its own
 * handle would (same kernels and arithmetic).
 * ------------------------------------------------------------------------------------------- */
typedef struct osbli_ens osbli_ens_t;

/* params: [nprob] member descriptions (uniform grids, own n, h, dt; inviscid, Re <= 0; WENO5-JS,
 * WENO-Z, TENO5 or TENO6, the same scheme and precision for every member; faces PERIODIC or ZEROGRAD; no
 * sensor).  cuda_stream: cudaStream_t for all work, or NULL for an ensemble-owned stream.
 * Errors: EINVAL (with the member index in the message), ENOMEM, ECUDA. */
int osbli_ensemble_create(int nprob, const osbli_params *params, void *cuda_stream, osbli_ens_t **out);

/* Release the members and tables.  NULL is ignored. */
void osbli_ensemble_destroy(osbli_ens_t *e);

/* State of member p in / out, [5][nz][ny][nx] FP64, host or device (as osbli_set/get_state). */
int osbli_ensemble_set_state(osbli_ens_t *e, int p, const double *U);
int osbli_ensemble_get_state(osbli_ens_t *e, int p, double *U);

/* The handle of member p (owned by the ensemble; for diagnostics / residuals), NULL if out of
 * range. */
osbli_t *osbli_ensemble_member(osbli_ens_t *e, int p);

/* nsteps RK3 steps of every member (one graph replay per step), then a synchronising check of
 * the members' error words.  Errors: ESTATE (a member without state), ENONFINITE (the message
 * names the lowest member that became non-finite), ECUDA. */
int osbli_ensemble_step(osbli_ens_t *e, int nsteps);

/* Marching chunk of the line kernels for every member (0: each member's own default, sized to fill
 * the GPU alone).  Changes launch shapes only: results are bitwise identical. */
int osbli_ensemble_set_chunk(osbli_ens_t *e, int chunk);

/* Time reps steps for each candidate chunk (0, 8, 16, 32, 64) on the current state, keep the
 * fastest, restore every member's state.  chunk_out / ms_out (may be NULL): the choice and its
 * milliseconds per step.  Allocates a copy of the states for the duration of the call. */
int osbli_ensemble_autotune(osbli_ens_t *e, int reps, int *chunk_out, double *ms_out);

/* Persistent form (on = 1): each osbli_ensemble_step call is ONE cooperative kernel launch that
 * runs all nsteps RK steps of every member.  Its blocks (as many as can be resident at once)
 * take each phase's virtual blocks over all members from a device ticket counter (the tile
 * queue) and meet at a grid barrier between phases.  Every barrier wait is bounded by
 * spin_limit polls of at least 64 ns each (0: the default, 2e7); a wait that runs out makes
 * every block leave and osbli_ensemble_step return OSBLI_ETIMEOUT, the members' states then
 * partly advanced (set them again).  Results are bitwise those of the graph form (on = 0, the
 * default: one launch per phase over all members, one graph per step).  Errors: EINVAL. */
int osbli_ensemble_set_persistent(osbli_ens_t *e, int on, long long spin_limit);

/* Blocks of the last persistent launch (0 before one). */
int osbli_ensemble_persistent_grid(const osbli_ens_t *e);

/* Kernel launches of one captured step (0 before the first step; 1 in the persistent form, whose
 * single launch covers a whole osbli_ensemble_step call), total interior points. */
int osbli_ensemble_launches_per_step(const osbli_ens_t *e);
long long osbli_ensemble_points(const osbli_ens_t *e);

/* Message of the last failure on e (or of the last failed osbli_ensemble_create when NULL). */
const char *osbli_ensemble_last_error(const osbli_ens_t *e);

/* ---------------------------------------------------------------------------------------------
 * Split grids: one grid divided into z-slabs, each a sub-domain with its own ghost layers, as
 * the paper's parallel runs divide their grids into blocks that exchange halos (Sec. 7.2).  The
 * slabs live on the current device.  Once per RK stage every slab's low and high ghost planes
 * are copied from its neighbours' interior planes into its own ghost buffers (the conserved
 * state, 3 planes: the i-2..i+3 stencil; on viscous runs also the z-direction viscous fluxes,
 * 2 planes, after they are formed), then each slab advances on its own.  Results are bitwise
 * those of one osbli_t on the whole grid.  Uniform grids (params.h) only, any scheme,
 * precision and face type; the learned sensor is not offered on split grids.
 * ------------------------------------------------------------------------------------------- */
#define OSBLI_DOMAIN_MAX_SLABS 64
typedef struct osbli_dom osbli_dom_t;

/* The split of nz planes into nslab contiguous slabs (the first nz % nslab slabs one plane
 * longer): slab s holds global planes k0[s] .. k0[s] + nzs[s] - 1; lo[s] / hi[s] are the slabs
 * across its low / high z face (periodic: wrapping), -1 for a physical face.  Host only (no
 * device work).  Arrays of nslab entries.  Errors: EINVAL (nslab outside 1..min(nz, 64)). */
int osbli_domain_plan(int nz, int nslab, int periodic, int *k0, int *nzs, int *lo, int *hi);

/* Split the grid of p (uniform, nz > 1) into nslab z-slabs per osbli_domain_plan.  Every slab
 * needs >= 3 planes, >= 5 where it has a physical z face.  cuda_stream as for osbli_create.
 * Errors: EINVAL (with the reason; message from osbli_domain_last_error(NULL)), ENOMEM, ECUDA. */
int osbli_domain_create(const osbli_params *p, int nslab, void *cuda_stream, osbli_dom_t **out);
void osbli_domain_destroy(osbli_dom_t *d);

/* Whole-grid state in / out, [5][nz][ny][nx] FP64, host or device (split across the slabs). */
int osbli_domain_set_state(osbli_dom_t *d, const double *U);
int osbli_domain_get_state(osbli_dom_t *d, double *U);

/* Face data of the whole grid's DIRICHLET / INFLOW face, layout as osbli_set_boundary_data. */
int osbli_domain_set_boundary_data(osbli_dom_t *d, int dir, int side, const double *prims);

/* nsteps RK steps of the whole grid (one CUDA graph per step holding every slab's launches and
 * the halo copies); synchronises and checks every slab's error word (ENONFINITE names the
 * slab). */
int osbli_domain_step(osbli_dom_t *d, int nsteps);

/* Residual of the current whole-grid state, [5][nz][ny][nx], host or device.  Synchronises. */
int osbli_domain_residual(osbli_dom_t *d, double *R);

/* Slab count; the handle of slab s (owned by the domain); kernel launches of one captured step
 * (0 before the first step) and, in *copies, its halo copies. */
int osbli_domain_slabs(const osbli_dom_t *d);
osbli_t *osbli_domain_member(osbli_dom_t *d, int s);
int osbli_domain_launches_per_step(const osbli_dom_t *d, int *copies);
const char *osbli_domain_last_error(const osbli_dom_t *d);

#ifdef __cplusplus
}
#endif

#endif /* OSBLI_H */
