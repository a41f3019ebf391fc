/*
 * strm.h: C ABI of the GB300 (sm_103a) library that evaluates the right-hand side of the 3D
 * compressible Navier-Stokes equations and advances them with Wray's low-storage RK3, the
 * method of STREAmS (Bernardini, Modesti, Salvadore and Pirozzoli, arXiv 2004.02276, Section 2).
 *
 * Conventions shared by every entry point
 *   - Return value: STRM_OK (0) or a negative status below. strm_last_error() gives a
 *     thread-local message for the last failure. No C++ exception or abort crosses the ABI.
 *   - Device pointers: every `double*` state or residual argument is a device address
 *     (cudaMalloc'd or from a framework allocator) unless its name ends in `_host`.
 *   - State layout: the conserved variables w = [rho, rho u, rho v, rho w, rho E] (Section 2.2)
 *     as five SoA fields over the interior nodes only, x fastest:
 *         w[m*N + (k*ny + j)*nx + i],  N = nx*ny*nz,  0 <= m < 5.
 *     Residuals R and the RK register use the same layout. Ghost layers live in the workspace.
 *   - Ownership: the caller owns w, r_old, rhs and the workspace. The library owns only the
 *     opaque context (host memory) and, after the first strm_advance_n call, a CUDA graph and
 *     a private capture stream. It never allocates device memory.
 *   - Streams: all work is enqueued on the stream given to strm_init_grid, in stream order.
 *     Entry points that return host data (strm_conserved_totals, strm_get_time, the _host
 *     variants) synchronise that stream; the others return without waiting.
 *   - Concurrency: a context is not thread safe; use one context per host thread/stream.
 *
 * Grid (Sections 3.1-3.3): nx*ny*nz nodes; x and z uniform (x_i = (i + 1/2) lx/nx); y nodes at
 * eta_j = (j + 1/2)/ny mapped by one of the STRM_MAP_* maps (clustered toward both walls,
 * toward one wall at y = 0, or uniform), so that walls at eta = 0 and 1 fall on interfaces
 * (staggered wall). z is periodic; x and y periodic by default.
 * Non-dimensional gas: p = rho R T, E = cv T + |u|^2/2, H = E + p/rho, k = cp mu/Pr.
 */
#ifndef STRM_H
#define STRM_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
  STRM_OK = 0,
  STRM_EINVAL = -1,     /* bad argument or configuration */
  STRM_ECUDA = -2,      /* a CUDA runtime call failed */
  STRM_ENONFINITE = -3, /* a reduction met NaN or Inf (the state blew up) */
  STRM_ENOMEM = -4,     /* workspace smaller than strm_workspace_bytes() */
  STRM_ETIMEOUT = -5    /* reserved for bounded device-side waits */
};

/* Wall-normal maps y(eta), eta in [0, 1] (nodes at eta_j = (j + 1/2)/ny):
 *   UNIFORM          y = ly (eta - 1/2)
 *   TANH             y = (ly/2) tanh(beta (2 eta - 1)) / tanh(beta)   (both walls)
 *   TANH_ONESIDED    y = ly (1 - tanh(beta (1 - eta)) / tanh(beta))   (wall at y = 0)
 *   ERF              y = (ly/2) erf(beta (2 eta - 1)) / erf(beta)     (both walls; Section 3.1)
 *   SINH_ONESIDED    y = ly sinh(beta eta) / sinh(beta)               (wall at y = 0; Section 3.2) */
enum { STRM_MAP_UNIFORM = 0, STRM_MAP_TANH = 1, STRM_MAP_TANH_ONESIDED = 2, STRM_MAP_ERF = 3,
       STRM_MAP_SINH_ONESIDED = 4 };
enum {
  STRM_BC_PERIODIC = 0,        /* no params */
  STRM_BC_WALL_ISOTHERMAL = 1, /* y faces; no params */
  STRM_BC_CHARACTERISTIC = 2,  /* 5 params: reference rho, u, v, w, p */
  STRM_BC_RECYCLE_INFLOW = 3,  /* x-min; 7 params: reference rho, u, v, w, p, recycling plane i, delta_in */
  STRM_BC_SHOCK_TOP = 4,       /* y-max; 7 params: free stream rho, u, v, w, p, deflection theta
                                  (radians), x where the incident shock reaches the wall */
  STRM_BC_DF_INFLOW = 5        /* x-min; digital-filter inflow, set with strm_set_inflow_df */
};
enum { STRM_FACE_YMIN_YMAX = 0, STRM_FACE_XMIN = 1, STRM_FACE_XMAX = 2, STRM_FACE_YMIN = 3, STRM_FACE_YMAX = 4 };
enum { STRM_WENO_OFF = 0, STRM_WENO_SENSOR = 1, STRM_WENO_ALL = 2 };
enum { STRM_VISC_POWER = 0, STRM_VISC_SUTHERLAND = 1 };
/* STRM_PREC_FP64: every operation in FP64. STRM_PREC_MIXED: flux, sensor, WENO and viscous
 * arithmetic in FP32 (the x faces' central flux on deviations from a per-row reference formed
 * in FP64); FP64 for the stored state, the primitives rho, u, v, w, p, H, the projection of w
 * and of the flux into characteristic variables, the RK stage accumulation, forcing, the time
 * step (from FP32 wave-speed maxima) and totals. */
enum { STRM_PREC_FP64 = 0, STRM_PREC_MIXED = 1 };

typedef struct {
  int nx, ny, nz;        /* interior nodes, each >= 1 (ny >= 3 with walls) */
  double lx, ly, lz;     /* box lengths */
  int y_map;             /* one of STRM_MAP_* */
  double beta;           /* clustering parameter (> 0 for every map but STRM_MAP_UNIFORM) */
} strm_grid;

typedef struct {
  double gamma;          /* ratio of specific heats */
  double prandtl;        /* Pr (Section 2: 0.72) */
  double r_gas;          /* gas constant R in the chosen units */
  int visc_law;          /* STRM_VISC_POWER: mu_ref (T/t_ref)^visc_exp; SUTHERLAND: suth_s = S/t_ref */
  double mu_ref, t_ref, visc_exp, suth_s;
  double t_wall;         /* isothermal wall temperature */
  int forcing;           /* 1: constant mass flow rate in x (Eqs. 1b, 1c) */
} strm_phys;

typedef struct {
  int L;                 /* central scheme half width, order 2L: 2 or 3 (Eq. encflux) */
  int weno_mode;         /* STRM_WENO_OFF / SENSOR (Ducros switch, Eq. sensor) / ALL */
  double theta_thr;      /* sensor threshold for the WENO switch */
  double weno_eps;       /* WENO5 epsilon */
  double u0, l0;         /* sensor scales: the floor in the sensor denominator is (u0/l0)^2 */
  int convective;        /* 1: include convective terms (0 only for tests) */
  int viscous;           /* 1: include viscous terms (0 for inviscid runs) */
  int precision;         /* STRM_PREC_FP64 or STRM_PREC_MIXED */
} strm_scheme;

typedef struct strm_ctx strm_ctx;

/* Thread-local message describing the last non-OK status. */
const char* strm_last_error(void);

/* Device workspace (bytes) a context with this grid and scheme needs; 0 if invalid. */
size_t strm_workspace_bytes(const strm_grid* g, const strm_scheme* s);

/* Create a context (Section 2; grid of Section 3.1). `workspace` is a device buffer of at least
 * strm_workspace_bytes() bytes, 256-byte aligned, owned by the caller and kept alive until
 * strm_destroy. `stream` is a cudaStream_t (NULL: the legacy default stream). The y boundary
 * starts periodic; strm_set_bc selects walls. Uploads the wall-normal metrics (stream order). */
int strm_init_grid(strm_ctx** ctx, const strm_grid* g, const strm_phys* p, const strm_scheme* s,
                   void* workspace, size_t workspace_bytes, void* stream);

/* Boundary kind of a face (z faces are periodic). STRM_FACE_YMIN_YMAX sets both y faces to
 * periodic or wall. A periodic face needs a periodic opposite face (checked at the next
 * evaluation). Kinds:
 *   WALL_ISOTHERMAL: no-slip, T = t_wall, staggered (Section 3.1): mirrored ghosts, no mass,
 *     tangential-momentum or energy flux through the wall face.
 *   CHARACTERISTIC (Section 3.2, non-reflecting top and outflow): ghosts from the eigenvectors at
 *     the boundary node; outgoing characteristic variables extrapolated at zeroth order, incoming
 *     ones from a reference state: at y faces the reference primitives; at x faces (outflow) the
 *     boundary node's state at the reference pressure, since the outflow plane crosses the
 *     boundary layer and a subsonic outflow prescribes only the far-field pressure.
 *   RECYCLE_INFLOW (x-min): ghost plane -1-q copies interior plane i_recycle-q with heights
 *     stretched by delta_r/delta_in, delta_r where the spanwise-mean u of the recycling plane first
 *     reaches 0.99 u_ref (a rescaled recycling inflow; the paper's own inflow, the digital-filter
 *     inflow, is set with strm_set_inflow_df).
 *   SHOCK_TOP (y-max, Section 3.3): characteristic face whose reference is, downstream of the
 *     shock foot x_imp - ly/tan(beta), the weak oblique-shock post-shock state of deflection theta.
 * Returns STRM_EINVAL for a wrong face, kind or parameter count. */
int strm_set_bc(strm_ctx* ctx, int face, int kind, const double* params, int nparams);

/* rhs <- R(w): convective (central or WENO per the sensor), viscous and forcing terms
 * (Section 2.1, Eqs. 1a-c). w and rhs are device arrays of 5*N doubles; they must not alias. */
int strm_compute_rhs(strm_ctx* ctx, const double* w, double* rhs);

/* One RK3 step in place (Eq. RK, alpha = (0, -17/60, -5/12), beta = (8/15, 5/12, 3/4)).
 * dt > 0: fixed step; dt <= 0: CFL step dt = cfl / max(sum_d (|u_d| + c)/h_d), computed on the
 * device. r_old is a caller-owned device register of 5*N doubles (its contents on entry are
 * not used; on exit it holds the last stage's residual). */
int strm_rk_step(strm_ctx* ctx, double* w, double* r_old, double dt, double cfl);

/* nsteps RK3 steps (as strm_rk_step) replayed from a CUDA graph captured on first use. */
int strm_advance_n(strm_ctx* ctx, double* w, double* r_old, int nsteps, double dt, double cfl);

/* Host-buffer variant: copies w_host (5*N doubles) to the device buffer w, advances nsteps,
 * copies the state back to w_host and waits for the stream. A page-locked w_host that is mapped
 * into the device's address space (cudaHostRegister, cudaHostAlloc; 16-byte aligned) is copied
 * by a kernel through its device address; other host memory by cudaMemcpyAsync. w and r_old:
 * distinct device buffers of 5*N doubles (STRM_EINVAL if null or equal). */
int strm_advance_n_host(strm_ctx* ctx, double* w_host, double* w, double* r_old, int nsteps,
                        double dt, double cfl);

/* Metric-weighted totals out_host[m] = sum_interior w_m dx (y_eta deta) dz. Synchronises.
 * Returns STRM_ENONFINITE if any total is NaN or Inf. */
int strm_conserved_totals(strm_ctx* ctx, const double* w, double out_host[5]);

/* Simulated time accumulated by strm_rk_step/strm_advance_n and the last dt. Synchronises.
 * Returns STRM_ENONFINITE (outputs still written) when either is NaN or Inf: the CFL maximum
 * propagates a non-finite state into dt, so this is the cheap health check after a run. */
int strm_get_time(strm_ctx* ctx, double* t_host, double* dt_host);

/* Set the simulated time (and reset the last dt to 0). Stream-ordered. */
int strm_set_time(strm_ctx* ctx, double t);

/* Sensor diagnostics for parity checks: theta and node divergence at the interior nodes
 * (device, N doubles each, nullable), and the WENO face flags (device bytes, nullable) in the
 * layout x: [nz][ny][nx+1], y: [nz][ny+1][nx], z: [nz+1][ny][nx]; entry s along a direction
 * is the interface between nodes s-1 and s. */
int strm_sensor(strm_ctx* ctx, const double* w, double* theta, double* div,
                unsigned char* flags_x, unsigned char* flags_y, unsigned char* flags_z);

/* Number of WENO faces per direction in the last right-hand-side evaluation. Synchronises. */
int strm_weno_counts(strm_ctx* ctx, long long counts_host[3]);

/* ---- Digital-filter turbulent inflow (Section 3.2: Klein-type digital filter done as a sequence
 * of one-dimensional convolutions, strong Reynolds analogy, prescribed Reynolds stresses). Once
 * per time step a new random plane is drawn (SplitMix64 keyed by draw, velocity component, z
 * and extended-y index; r = sqrt(3)(2u - 1)), filtered along y with b_l = exp(-pi l^2/(2 n^2))
 * normalised to unit energy, l = -2n..2n, then along z (periodic), and blended into the
 * fluctuation plane Psi <- Psi exp(-pi dt/(2 tau)) + psi sqrt(1 - exp(-pi dt/tau)). Every ghost
 * layer of the x-min face takes u_i = U_i(y) + a_ij Psi_j (a: Cholesky factor of the Reynolds
 * stresses, R13 = R23 = 0), T = T(y) - U u'/cp, p = p_ref, rho = p/(R T). */
typedef struct {
  double p_ref;              /* inflow pressure */
  int ny_filter, nz_filter;  /* filter half-widths n in grid points along y and z (>= 1) */
  double tau;                /* integral time scale of the time correlation (> 0) */
  unsigned long long seed;   /* generator seed */
} strm_df;

/* Device bytes of the inflow buffer for this context and filter (0 if invalid). */
size_t strm_inflow_df_bytes(const strm_ctx* ctx, const strm_df* df);

/* Make the x-min face a digital-filter inflow. profiles_host[7][ny]: the mean U, V, T and the
 * Reynolds stresses R11, R12, R22, R33 at the wall-normal nodes (R must be positive
 * semi-definite). buffer: caller-owned device memory of strm_inflow_df_bytes() bytes, 8-byte
 * aligned, kept while the face is in use. Draws the first plane (stream-ordered). The x-max face
 * must not be periodic. STRM_EINVAL on bad arguments. */
int strm_set_inflow_df(strm_ctx* ctx, const strm_df* df, const double* profiles_host, void* buffer,
                       size_t bytes);

/* ---- Flow statistics (Section 3: Reynolds averages over the homogeneous directions and in
 * time; Favre averages are ratios of the mass-weighted ones, e.g. u~ = (rho u)/rho). Each
 * sample adds, in FP64 on the device, the spatial means of STRM_NSTAT point-wise quantities,
 * in this order:
 *   rho, u, v, w, p, T, rho u, rho v, rho w, rho T, rho uu, rho vv, rho ww, rho uv, rho uw,
 *   rho vw, uu, vv, ww, uv, p^2, T^2, rho^2, mu.
 * STRM_STATS_XZ averages over x and z (channel: one row of ny values per quantity);
 * STRM_STATS_Z averages over z only (spatially developing flows: ny x nx values, x fastest).
 * The accumulator lives in a caller-owned device buffer; the sums are taken in a fixed order
 * (one thread per (x, y) column walking z, then one block per row for the x sum). */
enum { STRM_NSTAT = 24 };
enum { STRM_STATS_XZ = 0, STRM_STATS_Z = 1 };

/* Device bytes of the statistics buffer for `mode` (0 if ctx is NULL or the mode unknown). */
size_t strm_stats_bytes(const strm_ctx* ctx, int mode);

/* Attach a caller-owned device buffer of strm_stats_bytes(ctx, mode) bytes (8-byte aligned) and
 * zero the sums (stream-ordered); resets the sample count and the step counter. buffer = NULL
 * detaches (no further samples). The buffer must outlive its use by the context. */
int strm_stats_bind(strm_ctx* ctx, int mode, void* buffer, size_t bytes);

/* Add one sample of the interior state w (stream-ordered). STRM_EINVAL without a buffer. */
int strm_stats_sample(strm_ctx* ctx, const double* w);

/* Sample automatically after every k-th step taken by strm_rk_step / strm_advance_n (k = 0:
 * never). Steps are counted from this call. The samples are stream-ordered launches after
 * the step (not part of the replayed step graph). */
int strm_stats_every(strm_ctx* ctx, int k);

/* Means over the samples taken so far, out_host[q * rows + r] with rows = ny (XZ) or ny * nx
 * (Z), and the number of samples (nullable). Synchronises. With no sample yet the means are 0. */
int strm_stats_read(strm_ctx* ctx, double* out_host, long long* nsamples_host);

/* Kernel classes of the per-kernel timing diagnostics. */
enum {
  STRM_K_PRIMS = 0, STRM_K_DT, STRM_K_GHOST_PRIMS, STRM_K_SENSOR, STRM_K_GHOST_SENSOR,
  STRM_K_FACES_X, STRM_K_FACES_Y, STRM_K_FACES_Z, STRM_K_WENO_X, STRM_K_WENO_Y, STRM_K_WENO_Z,
  STRM_K_ASSEMBLE, STRM_K_FORCE, STRM_K_RK_UPDATE, STRM_K_COUNT
};

/* Short name of kernel class k ("" if out of range). */
const char* strm_kernel_name(int k);

/* Turn per-kernel timing on or off and reset its accumulators. While on, every kernel the
 * context launches is bracketed by a CUDA event pair on the context's stream and
 * strm_advance_n launches eagerly instead of replaying its graph; the WENO face counts of
 * each evaluation are read back (which synchronises). Diagnostics only. */
int strm_timing(strm_ctx* ctx, int enable);

/* Accumulated milliseconds and launches per kernel class (arrays of STRM_K_COUNT, nullable)
 * and WENO faces processed per direction (array of 3, nullable) since strm_timing.
 * Synchronises the stream. */
int strm_timing_read(strm_ctx* ctx, double* ms_host, long long* launches_host,
                     long long* weno_faces_host);

/* Total kernels this context has launched (graph replays count every kernel in the graph). */
int strm_launch_count(strm_ctx* ctx, long long* launches_host);

/* ---- Batched ensemble: many independent grids advanced together (different sizes, gas and
 * flow parameters; the same central order L and precision). One RK3 step of the whole ensemble
 * is a CUDA graph replayed per step, under one of two schedules: each kernel of the right-hand
 * side and of the RK update as one launch over all instances, or (persistent) one cooperative
 * launch per RK stage that runs every phase of the stage with grid-wide barriers between them.
 * Every instance computes what a context of its own would (same kernel bodies), up to where the
 * compiler contracts a multiply and an add into an FMA and, in the persistent schedule, the
 * grouping of the CFL and forcing partial sums. */
typedef struct strm_ensemble strm_ensemble;

/* Device workspace for n instances (sum of the per-instance workspaces plus the instance
 * tables); 0 if any grid or scheme is invalid. */
size_t strm_ensemble_workspace_bytes(int n, const strm_grid* grids, const strm_scheme* schemes);

/* Create an ensemble of n instances: grids[e], phys[e], schemes[e] and the y boundary kind
 * bc_y[e] (STRM_BC_PERIODIC or STRM_BC_WALL_ISOTHERMAL). `workspace`: caller-owned device
 * memory of strm_ensemble_workspace_bytes() bytes, 256-byte aligned. Work goes to `stream`. */
int strm_ensemble_create(strm_ensemble** ens, int n, const strm_grid* grids, const strm_phys* phys,
                         const strm_scheme* schemes, const int* bc_y, void* workspace,
                         size_t workspace_bytes, void* stream);

/* Boundary kind of a face of instance e (as strm_set_bc on a single context: characteristic,
 * recycling inflow, shock top, ...), so that channel and boundary-layer instances advance
 * together. Takes effect at the next strm_ensemble_advance (the step graph is re-captured). */
int strm_ensemble_set_bc(strm_ensemble* ens, int e, int face, int kind, const double* params,
                         int nparams);

/* Device bytes of the inflow buffer of instance e (0 if invalid). */
size_t strm_ensemble_inflow_df_bytes(const strm_ensemble* ens, int e, const strm_df* df);

/* Digital-filter inflow of instance e (as strm_set_inflow_df; the caller-owned buffer serves that
 * instance). */
int strm_ensemble_set_inflow_df(strm_ensemble* ens, int e, const strm_df* df,
                                const double* profiles_host, void* buffer, size_t bytes);

/* nsteps RK3 steps of every instance (dt > 0 fixed for all, else each instance takes its own CFL
 * step with number cfl). w and r_old are host arrays of n device pointers (layout as for a
 * single grid, sized by each instance's grid). */
int strm_ensemble_advance(strm_ensemble* ens, double* const* w, double* const* r_old, int nsteps,
                          double dt, double cfl);

/* Autotuner: times one right-hand side of the ensemble (CUDA events, best of two) for the WENO
 * block size {32, 64, 128} x blocks per SM {4, 8, 16}, then the central-list grid {8, 16, 32}
 * blocks per SM, then the persistent schedule against the per-kernel one (not with a
 * digital-filter inflow), then the pencil tile of the slab traversal order of the assembly and
 * the z faces (slab height cap 32, 16, 8 or 0 = natural order); keeps the fastest and writes the
 * schedule {weno block, WENO blocks per SM, central blocks per SM, persistent 0/1, slab cap} to
 * choice_host[5] (nullable). The state is read, not modified. */
int strm_ensemble_tune(strm_ensemble* ens, double* const* w, double* const* r_old, int* choice_host);

/* Set the schedule the autotuner would choose: choice[5] as strm_ensemble_tune writes it.
 * STRM_EINVAL for a value outside the tuner's ranges (blocks per SM 1..64), for the persistent
 * schedule with a digital-filter inflow instance, or where the cooperative launch cannot run.
 * Each instance takes the largest admitted slab height not above the cap for its assembly, and
 * not above min(cap, 8) for its z faces (see the slab order of the assembly). Takes effect at
 * the next strm_ensemble_advance. */
int strm_ensemble_set_schedule(strm_ensemble* ens, const int* choice);

/* How long a grid-wide barrier of the persistent stage waits for the other blocks before it gives
 * up (default 10 s; seconds in [0, 3600], else STRM_EINVAL). Every phase of a stage must finish
 * within it. 0 makes the first block that has to wait give up, so the failure path (all blocks
 * leave, strm_ensemble_debug_flags reports 32) can be exercised without a fault. Takes effect at
 * the next strm_ensemble_advance. */
int strm_ensemble_set_barrier_limit(strm_ensemble* ens, double seconds);

/* Conserved totals of every instance, out_host[5*e + m]. Synchronises. */
int strm_ensemble_totals(strm_ensemble* ens, double* const* w, double* out_host);

/* Simulated time of every instance, t_host[e]. Synchronises. */
int strm_ensemble_times(strm_ensemble* ens, double* t_host);

/* The error words of all instances OR-ed together (bounds-checking build; see
 * strm_debug_flags), plus 32 (in every build) when a grid-wide barrier of the persistent stage
 * gave up waiting (strm_ensemble_set_barrier_limit); the blocks then left the kernel, the state
 * is not valid, and every later persistent stage leaves at its first barrier until this call
 * reports the bit, which also resets the barrier. Synchronises. */
int strm_ensemble_debug_flags(strm_ensemble* ens, unsigned* flags_host);

void strm_ensemble_destroy(strm_ensemble* ens);

/* ---- Overlap (Section 4: the paper overlaps the convective fluxes with the halo exchange).
 * mode is a set of bits; every later right-hand side of this context then runs
 *   STRM_OVERLAP_GHOST: the ghost-layer fill on a side stream while the Ducros sensor runs over
 *     the nodes at least L from every face of the box (their stencils read no ghost node); the
 *     sensor's boundary shell follows the join;
 *   STRM_OVERLAP_FACES: the x, y and z face stages (classification, central and WENO fluxes),
 *     which write separate flux arrays and lists, as three concurrent branches joined before
 *     the assembly.
 * Only the order of independent kernels changes: results are bit-identical to mode 0 (the
 * sequential order, the default). The two side streams and their events are created on the
 * first non-zero mode (with the context's device current) and released by strm_destroy; the
 * captured step graph of strm_advance_n is rebuilt on its next call. In timing mode
 * (strm_timing) all work stays on the context's stream. Concurrency pays on small grids, whose
 * kernels do not fill the GPU; on grids of millions of points each kernel fills it alone.
 * Null context or unknown bits: STRM_EINVAL; stream or event creation failure: STRM_ECUDA. */
#define STRM_OVERLAP_GHOST 1
#define STRM_OVERLAP_FACES 2
int strm_set_overlap(strm_ctx* ctx, int mode);

/* ---- Prescribed switch input: a test device of the hybrid scheme. The paper's switch (Eq.
 * sensor, Section 2.1) decides per face from the Ducros sensor of the current state; two runs
 * that differ by round-off (FP64 and mixed precision) eventually take different decisions at
 * faces whose sensor sits at the threshold, and each flip changes a flux by O(truncation). With
 * theta set, every later right-hand side of this context (sensor mode only) decides from the
 * caller's sensor values instead: theta is a device array of N doubles at the interior nodes
 * (layout of strm_sensor's theta), read at every evaluation, kept alive and unchanged by the
 * caller while set; the computed sensor still feeds the viscous terms (node divergence).
 * theta = NULL returns to the computed sensor. The step graph of strm_advance_n is rebuilt on
 * its next call. STRM_EINVAL: null context, or theta set outside STRM_WENO_SENSOR. */
int strm_set_theta(strm_ctx* ctx, const double* theta);

/* ---- Bounds checking. A library built with -DSTRM_DEBUG (paper_2004_02276_gb300/build.py,
 * debug=True: libstrm_debug.so) checks in every kernel the extreme nodes of each stencil, the
 * source node of each ghost and each face-list entry before using them; a violation ORs a code
 * into the context's error word (1 ghost fill, 2 node stencil, 4 face stencil or face index,
 * 8 list entry, 16 inflow plane) and the access is skipped instead of faulting. */

/* 1 if this library is the bounds-checking build, else 0. */
int strm_debug_build(void);

/* The context's error word (always 0 in the release build). Synchronises. */
int strm_debug_flags(strm_ctx* ctx, unsigned* flags_host);

/* ---- Precision conversions of the mixed-precision kernels. On GB300 (sm_103) the FP64 <-> FP32
 * conversion instructions issue on the FP64 pipe; the mixed-precision kernels convert with
 * integer operations on the IEEE-754 bit patterns instead. These two calls apply the same
 * conversions elementwise to device arrays, so that they can be checked against IEEE-754
 * conversion:
 *   FP64 -> FP32: round to nearest, ties away from zero (IEEE ties-to-even differs only for
 *   values exactly halfway between two floats); magnitudes that round below 2^-126 give a
 *   signed zero; magnitudes that round to 2^128 or above, infinities and NaNs give a signed
 *   infinity.
 *   FP32 -> FP64: exact for normal floats; subnormals give a signed zero; infinities and NaNs
 *   stay infinities and NaNs.
 * x and y are device arrays of n elements (n = 0: nothing is done); the work is enqueued on
 * `stream` (NULL: the legacy default stream) and the call does not synchronise. n < 0, or a
 * null pointer with n > 0: STRM_EINVAL. */
int strm_convert_f64_f32(const double* x, float* y, long long n, void* stream);
int strm_convert_f32_f64(const float* x, double* y, long long n, void* stream);

/* ---- FMA issue-rate probe: the denominator of the ALU roofline. The paper has no counterpart
 * (its P100 ran FP64 at half the FP32 rate; on GB300 the FP64 pipe issues two DFMA per clock per
 * SM against 128 FP32 FMA, so every FP64 kernel of this library is bound by it). Launches
 * launches + 1 kernels (the first untimed) of independent FMA chains, kChains per thread, four
 * 256-thread blocks per SM, about 40 ms each at the nominal rate, on `stream` (NULL: the legacy
 * default stream), timed with CUDA events, and writes the best launch's rate in TFLOP/s
 * (2 flops per FMA) and its milliseconds (nullable). precision: STRM_PREC_FP64 for FP64 FMA,
 * STRM_PREC_MIXED for FP32 FMA. Synchronises. STRM_EINVAL for another precision, launches
 * outside 1..1000 or a null rate pointer; STRM_ECUDA if a CUDA call fails. */
int strm_peak_fma(int precision, int launches, void* stream, double* tflops_host, double* ms_host);

/* Largest grid (nx*ny*nz) strm_conserved_totals_static accepts. */
#define STRM_STATIC_MAX_NODES 67108864

/* Conserved totals for callers that cannot allocate device memory. The paper has no
 * counterpart: this is a service of the library, not a step of the method.
 *
 * The totals of strm_conserved_totals (out_host[m] = sum w_m dx (y_eta deta) dz over the
 * interior, for any of the STRM_MAP_* wall-normal maps), up to rounding: the node volumes are
 * evaluated on the device here rather than uploaded from the host. It needs no context and no
 * workspace and allocates nothing, so it can be called by code that must not call cudaMalloc:
 * an in-situ monitor attached to a solver whose allocator already holds the device memory, or
 * a tool running where allocation is not allowed. The caller passes the grid, the device state
 * w (layout as above, on the current device) and a stream (NULL: the legacy default stream);
 * the call synchronises that stream.
 *
 * Its scratch (partial sums and results, about 0.66 MB) is a file-scope __device__ array of
 * the library: every GPU that loads the library holds it until the process exits, and every
 * call on a device shares it. Calls that overlap on the GPU (for example on two streams) race
 * on that array; serialise them. Each call looks up the array's device address
 * (cudaGetSymbolAddress, in the current device's context); make the first call on a device
 * before any stream capture, since the lookup may load the module. Grids above
 * STRM_STATIC_MAX_NODES nodes, unknown maps and non-positive sizes are rejected with
 * STRM_EINVAL and a message naming the cause. */
int strm_conserved_totals_static(const strm_grid* g, const double* w, double out_host[5],
                                 void* stream);

/* Release the context (not the caller's buffers). Safe on NULL. */
void strm_destroy(strm_ctx* ctx);

#ifdef __cplusplus
}
#endif
#endif
