/*
 * goc.h -- C ABI of the B300 GOC-LBM library (libgoc.so).
 *
 * The library advances lattice Boltzmann solutions of the Navier-Stokes
 * equations in general orthogonal coordinates (GOC): the central-moment MRT
 * GOC-LBM for D2Q9 (Appendix E, "Summary of the Algorithmic Steps of the
 * Central Moment GOC-LBM") coupled, optionally, with the D2Q5 vector GOC-LB
 * scheme for the magnetic induction equation (Appendix G).  Every step runs
 * in the library's own CUDA kernels for sm_103a.
 *
 * Conventions
 *  - Plain C types only.  Every call returns a goc_status (0 = success, < 0 =
 *    error); goc_last_error() gives a thread-local message for the last error.
 *    No call aborts the process.
 *  - Ownership: the library owns all device memory it allocates (freed by
 *    goc_destroy / goc_batch_destroy).  The caller owns every host buffer it
 *    passes; the library never keeps a host pointer after a call returns.
 *  - Streams: all device work of a lattice runs on goc_exec.cuda_stream
 *    (a cudaStream_t; NULL = the legacy default stream).  goc_step returns
 *    after enqueueing; calls that return data to the host synchronise that
 *    stream only.
 *  - Layout of host field arrays: row-major [ny][nx], node (i, j) at j*nx + i,
 *    i along xi1, j along xi2.  Lattice units: Delta xi = Delta t = 1.
 *  - Geometry: straight orthogonal grids x = x(xi1), y = y(xi2) (Appendix B,
 *    case (i); theta12 = theta21 = 0) from the per-axis maps, the curvilinear
 *    annular sector of Sec. 8.1 (ANNULUS), or any orthogonal grid given node
 *    by node (TABLE).  Node placement: wall axes are cell-centred (eta_j =
 *    (j + 1/2)/N, walls half a spacing outside the first and last node,
 *    physical length N); periodic axes use eta_i = i/N.
 */
#ifndef GOC_H
#define GOC_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    GOC_OK = 0,
    GOC_EINVAL = -1,       /* invalid argument (message says which) */
    GOC_ENOMEM = -2,       /* device or host allocation failed */
    GOC_ECUDA = -3,        /* a CUDA runtime call failed */
    GOC_EDIVERGED = -4,    /* NaN/Inf or non-positive density detected */
    GOC_ETIMEOUT = -5,     /* a bounded device-side wait ran out */
    GOC_EBUSY = -6,        /* batch is full / HBM budget exhausted */
    GOC_EUNSUPPORTED = -7  /* valid request that the library does not support (message says which) */
} goc_status;

/* Opaque handle of one lattice; owned by the library. */
typedef struct goc_lattice goc_lattice;

/* Boundary of one side of the lattice. Sides: 0 = W (xi1 = 0), 1 = E,
 * 2 = S (xi2 = 0), 3 = N.  Opposite sides must both be periodic or both walls. */
typedef enum { GOC_BC_PERIODIC = 0, GOC_BC_WALL = 1 } goc_bc;

/* Stretching maps of one axis (Sec. 6).
 *  UNIFORM  x = xi.
 *  TANH2    clustering at both walls, Eq. hypertanh_transformation1 /
 *           Eq. metriccoefficient (Sec. 6.1): x = (N/2)[1 + tanh(beta(2 eta-1))/tanh beta].
 *  SINE     periodic stretching x = xi + (a N/2pi) sin(2 pi xi/N) (|a| < 1).
 *  ROBERTS  Roberts boundary-layer map, Eq. y_Roberts / Eq. h2_Roberts
 *           (Sec. 6.2), lambda = (gamma+1)/(gamma-1).
 *  TANH1    clustering at the wall xi = 0 only, Eq. hypertanh_transformation /
 *           Eq. metriccoefficientB (Sec. 6.3) with the prefactor N (the printed
 *           N/2 maps onto half the domain): x = N[1 - tanh(beta(1 - eta))/tanh beta].
 *  SINH     clustering around an interior point x_c = yc N, Eq. Holst_transformation,
 *           Eq. B_Holst, Eq. h_2_Holst (Sec. 6.4):
 *           x = x_c [1 + sinh(mu(eta - B))/sinh(mu B)].
 *  ANNULUS  (xi1 only) the curvilinear annular sector of Sec. 8.1 between radii
 *           r_inner and r_outer spanning 2 pi / sectors of the circle, by the
 *           conformal map of Eq. 2_annularsector scaled to the lattice (Eq.
 *           5_annularsector) with cell-centred radial nodes:
 *           r = r_inner exp(ln(r_outer/r_inner) xi1/nx), h1 = r ln(r_outer/r_inner)/nx,
 *           h2 = 2 pi r/(sectors ny), theta11 = theta21 = 1/r, theta12 = theta22 = 0.
 *           Needs W/E walls, periodic S/N, kind[1] = UNIFORM; schemes 0, 2, 3;
 *           not for batches.  Wall speeds (wall_u[W], wall_u[E]) are azimuthal.  With the
 *           MIE, Appendix G's curvature terms (theta21 in the local gradient
 *           formula, g^corr and J3, the source Y of Eq. 6ab_C) are active and
 *           the MIE populations are stored without a reference field.
 *  TABLE    (kind[0]; kind[1] ignored) a general orthogonal grid given node by
 *           node: `table` holds six [ny][nx] planes h1, h2, theta11, theta12,
 *           theta21, theta22 (Eq. metricfactor, Eq. curvaturematrix) and
 *           `wall_table` the metric factors at the wall points: first the
 *           wall-normal one (h1 at the W wall over j, h1 at E over j, h2 at S
 *           over i, h2 at N over i: 2 ny + 2 nx values), then the tangential
 *           one in the same order (h2 at W and E, h1 at S and N).  Moving walls
 *           use the normal factor, the MIE wall condition h1 h2; any values on
 *           periodic sides.  Both are host arrays read during goc_create only;
 *           every h > 0.  Schemes 0, 2, 3, not for batches; the MIE as for
 *           ANNULUS.
 * Wall maps (TANH2 with beta > 0, ROBERTS, TANH1, SINH) need a wall axis; SINE a
 * periodic one. */
typedef enum { GOC_MAP_UNIFORM = 0, GOC_MAP_TANH2 = 1, GOC_MAP_SINE = 2, GOC_MAP_ROBERTS = 3,
               GOC_MAP_TANH1 = 4, GOC_MAP_SINH = 5, GOC_MAP_ANNULUS = 6, GOC_MAP_TABLE = 7 } goc_map_kind;

typedef struct {
    int nx, ny;             /* nodes along xi1, xi2; >= 3 along a wall axis, >= 1 otherwise */
    int bc[4];              /* goc_bc per side W, E, S, N */
    double wall_u[4];       /* tangential wall velocity: S/N along xi1, W/E along xi2
                               (momentum-augmented bounce-back, Eq. 101 / Eq. 103) */
    double wall_b[4][2];    /* (B1, B2) imposed at each wall for the MIE anti-bounce-back
                               (Appendix G, "Boundary Conditions for the Magnetic Field") */
} goc_grid;

typedef struct {
    int kind[2];            /* goc_map_kind for xi1, xi2 */
    double beta[2];         /* TANH2 clustering parameter (0 = uniform); TANH1 (> 0) */
    double a[2];            /* SINE amplitude */
    double gamma[2];        /* ROBERTS gamma (> 1) */
    double alpha[2];        /* ROBERTS alpha (0 or 1/2) */
    double mu[2];           /* SINH clustering strength (> 0) */
    double yc[2];           /* SINH clustering point as a fraction of the axis length, in (0, 1) */
    double r_inner, r_outer;  /* ANNULUS radii, 0 < r_inner < r_outer */
    double sectors;           /* ANNULUS: the sector spans 2 pi / sectors (> 0) */
    const double *table;      /* TABLE: [6][ny][nx] h1, h2, theta11, theta12, theta21, theta22 */
    const double *wall_table; /* TABLE: [2][2 ny + 2 nx] wall-normal, then tangential metric at W, E, S, N */
} goc_map;

typedef struct {
    double rho0;            /* reference density (initial state), > 0 */
    double tau;             /* shear relaxation time: omega4 = omega5 = 1/tau (used if nu <= 0) */
    double nu;              /* kinematic viscosity nu = cs^2 (1/omega5 - 1/2) (Eq. 73); > 0 overrides tau */
    double tau_zeta;        /* omega3 = 1/tau_zeta, zeta = cs^2 (tau_zeta - 1/2) (Eq. 76); 0 -> 1 */
    double omega_free;      /* omega0,1,2,6,7,8 (preparatory step (d)); 0 -> 1 */
    double fext[2];         /* external body force, GOC components F_ext,1, F_ext,2 */
    int gi_correction;      /* 1: full coefficients of Eqs. 83/85 (default);
                               0: the cubic Galilean-invariance terms dropped */
} goc_flow;

typedef struct {
    int enabled;            /* couple the D2Q5 MIE scheme (Appendix G) */
    double tau_m;           /* magnetic relaxation time (used if eta <= 0) */
    double eta;             /* magnetic resistivity eta = csm^2 (tau_m - 1/2); > 0 overrides tau_m */
    double mu_m;            /* magnetic permeability (current density J = curl B / mu_m); 0 -> 1 */
    double b_init[2];       /* uniform initial field (B1, B2); on per-axis grids also the storage
                               reference state */
} goc_mhd;

/* Population storage in HBM.  All arithmetic is FP32.  Populations are
 * stored as deviations from the node's rest equilibrium at rho0
 * (f_rest = P^-1 (h1 h2 rho0, 0, 0, h2/h1 rho0 cs^2, h1/h2 rho0 cs^2, 0, 0, 0, rho0 cs^4));
 * FP16/BF16 store them divided by one per-lattice scale. */
typedef enum { GOC_FP32 = 0, GOC_FP16_DEV = 1, GOC_BF16_DEV = 2 } goc_storage;

typedef struct {
    int storage;            /* goc_storage */
    void *cuda_stream;      /* cudaStream_t for all work of this lattice; NULL = default stream */
    int device;             /* CUDA device ordinal; < 0 = current device */
    int check_every;        /* goc_run_until: steps between residual checks; 0 -> 100 */
    int rounding;           /* FP16/BF16 storage: 0 = stochastic rounding of every stored value
                               (unbiased, so increments below half a unit in the last place
                               are kept on average), 1 = round to nearest; ignored for FP32 */
    int scheme;             /* 0 = the GOC-LBM step (default); 1 = the standard uniform-grid
                               central-moment LBM (the comparator: the GOC step at h1 = h2 = 1,
                               local collision, no stored force); scheme 1 requires uniform
                               maps on both axes, gi_correction = 0 and no MIE (else
                               GOC_EINVAL); 2 = the GOC-LBM with the single-relaxation-time
                               collision in velocity space of Appendix F (one rate 1/tau for
                               every moment, zeta = nu; tau_zeta and omega_free are ignored;
                               any map, MIE allowed; it diverges on clustered grids at
                               tau < 1 where the central-moment step does not); 3 = the GOC-LBM
                               with the raw-moment MRT collision of Appendix D (rates as for
                               scheme 0); lattices added by goc_batch_add use scheme 0 */
    int fixed_launch;       /* 0 = the launch autotuner picks the tile order (dynamic queue or
                               static) and programmatic dependent launch on or off, by timing
                               each choice on 16 steps of the first goc_step call of at least
                               72 steps (choices are cached per lattice size, storage and MIE;
                               every choice gives bitwise the same populations);
                               1 = fixed: dynamic tile queue, dependent launch on */
    int plateau_checks;     /* goc_run_until also stops once this many successive checks bring
                               no new smallest residual (the FP32/FP16 rounding floor lies above
                               the tolerance); 0 = never */
    int reference_every;    /* FP16/BF16 storage on straight grids: the stored deviations of the
                               xi1 links (1, 3) are taken relative to a reference that carries
                               the row-mean velocity A1(j), and the MIE populations relative to
                               the row-mean field Bref(j); the reference is refreshed from the
                               state every this many steps (and at initialisation), so that at a
                               steady flow along xi1 the stored values -- and their rounding
                               noise -- shrink to what the row means do not capture.
                               0 -> every 1024 steps; < 0 = never (A1 = 0, Bref = B_init).
                               goc_step refreshes exactly at multiples of the period; in a
                               batch, at the end of the goc_batch_step call that reaches one.
                               Ignored for FP32 storage, curved grids and scheme 1. */
    int streaming;          /* 0 = two population buffers, read one and write the other (default);
                               1 = one buffer updated in place: two access patterns alternate
                               (the post-collision populations kept at their node with the link
                               reversed, then at the node they stream to), each step a fields
                               pass and a collision pass.  FP32: 56 B per node resident instead
                               of 88 B, 156 B moved per step instead of 88 B, the populations
                               bitwise those of streaming 0; the MIE populations follow the
                               same layouts (40 B resident instead of 80 B; the fields agree to
                               rounding: the wall nodes' multiply-adds may fuse differently);
                               16-bit storage: 34 B instead of 44 B, the fields buffer staying
                               FP32, stochastic rounding from the same random streams (results
                               within the storage's rounding of streaming 0).  Scheme 0,
                               per-axis maps (else GOC_EUNSUPPORTED); not in batches or slabs;
                               goc_get_state / goc_set_state keep the layout, so a state moves
                               only between lattices of the same streaming. */
} goc_exec;

/* ---- lifecycle --------------------------------------------------------- */

/* q = min(min h1, min h2) and cs^2 = q^2/3 of a grid/map pair (Eq. GOC-LBE_CFL),
 * computed by the library's FP64 metric kernel (for a TABLE map, from the
 * table on the host).  Either output may be NULL. */
goc_status goc_metric_info(const goc_grid *grid, const goc_map *map, double *q, double *cs2);

/* Create a lattice: FP64 metric precompute (preparatory step (a)), cs rule
 * (step (c)), relaxation rates (step (d)), device allocation and the initial
 * state at rest with rho = rho0, U = 0, B = b_init (Appendix C.1).
 * mhd may be NULL (no MIE); exec may be NULL (FP32, default stream).
 * On success *out owns the lattice; on failure *out is NULL. */
goc_status goc_create(const goc_grid *grid, const goc_map *map, const goc_flow *flow,
                      const goc_mhd *mhd, const goc_exec *exec, goc_lattice **out);

/* Re-initialise from host fields (each [ny][nx] doubles, NULL = default:
 * rho0, 0, 0, b_init): f = P^-1 m^eq,eff(rho, U) with finite-difference
 * gradients (Appendix C.1), g = g^eq(B, U) + g^corr, stored force F = 0.
 * The fields are copied straight from the caller's buffers (page-locked
 * buffers copy fastest) into a device staging area of 5 nx ny doubles that
 * the lattice keeps (it is also the goc_moments buffer).  Resets the step
 * counter.  Synchronises the stream. */
goc_status goc_init_fields(goc_lattice *lat, const double *rho, const double *u1,
                           const double *u2, const double *b1, const double *b2);

/* NULL-safe.  Synchronises the stream and frees all device memory. */
void goc_destroy(goc_lattice *lat);

/* The launch configuration in use: *dynamic_tiles = 1 for the dynamic tile
 * queue (0: static tile order), *pdl = 1 for programmatic dependent launch,
 * *tuned = 1 once chosen (by the autotuner or fixed).  Any output may be NULL.
 * No counterpart in the paper: a property of this implementation. */
goc_status goc_launch_config(const goc_lattice *lat, int *dynamic_tiles, int *pdl, int *tuned);

/* Set the launch configuration (dynamic_tiles, pdl: 0 or 1) and turn the
 * autotuner off for this lattice.  Takes effect from the next step. */
goc_status goc_set_launch_config(goc_lattice *lat, int dynamic_tiles, int pdl);

/* Grid of the step kernel: *balanced = 0 launches as many persistent blocks
 * as fit on the device (or one per tile), 1 the fewest blocks that take the
 * same number of rounds of tiles, so every block gets an equal share (512
 * blocks for the 1024 tiles of a 512^2 lattice instead of 592 with 1.73
 * rounds).  Chosen by the autotuner with the other launch settings; the set
 * call fixes it (and turns the autotuner off).  Results are bitwise the same
 * under either.  No counterpart in the paper. */
goc_status goc_launch_grid(const goc_lattice *lat, int *balanced);
goc_status goc_set_launch_grid(goc_lattice *lat, int balanced);

/* Tile shape of the step kernel on straight grids with the central-moment
 * collision: *rows = 8 (tiles of 32 x 8 nodes, one node per thread) or 16
 * (32 x 16, two nodes per thread, so the per-tile work and the ring of halo
 * nodes are shared by twice the nodes).  Other lattices always use 8.  Chosen
 * by the autotuner with the other launch settings; the set call fixes it
 * (GOC_EINVAL for a height other than 8 or 16, or 16 on a lattice that cannot
 * use it) and turns the autotuner off.  Results are bitwise the same under
 * either.  No counterpart in the paper. */
goc_status goc_tile_height(const goc_lattice *lat, int *rows);
goc_status goc_set_tile_height(goc_lattice *lat, int rows);

/* ---- the hot loop ------------------------------------------------------ */

/* Enqueue nsteps time steps (each one fused launch: pull-streaming with
 * boundary conditions, hydrodynamic fields, normal gradients, stresses,
 * effective and Lorentz forces, central-moment collision, MIE collision,
 * store).  Asynchronous: returns launch errors, and the device status word
 * as a copy taken behind the previous call's work, if it has arrived (no
 * wait): GOC_EDIVERGED once a step saw NaN/Inf or a non-positive density,
 * GOC_ETIMEOUT if a staged tile copy did not complete in its bounded wait; the
 * status is sticky until goc_init_fields or goc_set_state.  nsteps >= 0. */
goc_status goc_step(goc_lattice *lat, long long nsteps);

/* Step until the residual R = ||U^n - U^(n-1)||_2 / ||U^n||_2 (max with the
 * B residual when the MIE is on; Sec. 7.3) falls below tol, checking every
 * exec.check_every steps, or max_steps is reached, or (exec.plateau_checks > 0)
 * that many checks in a row found no new smallest residual.  *done (may be
 * NULL) receives the steps taken, *residual (may be NULL) the last residual.
 * Synchronises.  Returns GOC_EDIVERGED on NaN. */
goc_status goc_run_until(goc_lattice *lat, double tol, long long max_steps,
                         long long *done, double *residual);

/* Block the host until the lattice's stream has drained; then returns the
 * device status word as goc_step describes (GOC_EDIVERGED, GOC_ETIMEOUT). */
goc_status goc_sync(goc_lattice *lat);

/* ---- results ----------------------------------------------------------- */

/* Macroscopic fields of the current state into caller-owned host arrays
 * ([ny][nx] doubles each; any may be NULL): rho, U1, U2 (with the stored
 * force, Eq. GOChydrodynamicfields), B1, B2 (Eq. 13_C; zero without MIE).
 * cartesian != 0 maps vector components with Eq. vectormapping: on the
 * straight grids the GOC unit vectors coincide with the Cartesian ones (the
 * values are the same); on the ANNULUS (radial xi1, azimuthal xi2) they are
 * rotated by the azimuth phi = (pi/sectors)(2 j/ny - 1) of node row j; a
 * TABLE map carries no coordinates (GOC_EUNSUPPORTED).  Synchronises; the
 * arrays are filled even when the status word reports a diverged lattice
 * (then GOC_EDIVERGED is returned). */
goc_status goc_moments(goc_lattice *lat, int cartesian, double *rho, double *u1,
                       double *u2, double *b1, double *b2);

/* Same fields as FP32 into caller-owned DEVICE memory out[5][ny][nx]
 * (rho, U1, U2, B1, B2), enqueued on the lattice stream (no sync). */
goc_status goc_moments_device(goc_lattice *lat, float *out);

/* FP64 reductions of the current state: total mass sum f = sum h1 h2 rho,
 * and the residuals of the last goc_run_until check (0 before any).
 * Any pointer may be NULL.  Synchronises. */
goc_status goc_diagnostics(goc_lattice *lat, double *mass, double *residual_u,
                           double *residual_b);

/* Total mass sum f of the current state, like goc_diagnostics(mass), for
 * callers that cannot allocate device memory at the time they ask:
 * real-time loops that must not stall on the allocator, and applications
 * whose device memory is all handed to their own pool at start-up (a
 * cudaMalloc there fails or fragments that pool).  This call allocates
 * nothing: its scratch is a fixed array of
 * GOC_NOALLOC_MAX_BLOCKS + 1 doubles (32 KiB) inside the library, held by every
 * GPU that loads the library until the process exits.  The paper has no
 * counterpart; it is a service of this library.
 *  - Lattices of more than GOC_NOALLOC_MAX_NODES nodes are rejected with
 *    GOC_EINVAL and a message giving the limit.
 *  - The first call on a device looks up the scratch address (set-up); make
 *    that first call before any stream capture.
 *  - All calls share the scratch array and it keeps the last call's contents;
 *    calls whose work overlaps on the GPU (other streams or threads) race.
 *  - Every grid kind (per-axis maps, the annular sector, node tables) and
 *    every storage format is supported; the sum is taken in a fixed order
 *    (deterministic) and agrees with goc_diagnostics to FP64 rounding.
 *  - Runs on the lattice's device and restores the caller's current device
 *    before returning.  Waits for the lattice's stream (a synchronous
 *    device-to-host copy of the result), so that stream must not be under
 *    stream capture when this is called; *mass is a host pointer. */
#define GOC_NOALLOC_MAX_BLOCKS 4096
#define GOC_NOALLOC_MAX_NODES 8388608LL
goc_status goc_mass_noalloc(goc_lattice *lat, double *mass);

/* Steps taken since creation / the last goc_init_fields. */
long long goc_steps_done(const goc_lattice *lat);

/* Number of nodes and bytes of device memory held by the lattice. */
goc_status goc_footprint(const goc_lattice *lat, long long *nodes, long long *device_bytes);

/* Algorithmic HBM bytes one node update moves (populations and stored force
 * read and written once, plus the per-node share of the metric tables: the
 * per-axis tables amortised over the other axis, or the 10 FP32 values per
 * node of a TABLE map). */
double goc_bytes_per_node(const goc_lattice *lat);

/* ---- checkpoint / resume ----------------------------------------------- */

/* Serialise the full state (populations, stored force, MIE populations,
 * step counter) into a caller buffer.  With buf == NULL only *bytes is set.
 * Restoring into a lattice created with the same arguments and stepping
 * gives bitwise the same results as never stopping. */
goc_status goc_get_state(goc_lattice *lat, void *buf, size_t *bytes);
goc_status goc_set_state(goc_lattice *lat, const void *buf, size_t bytes);

/* ---- batched execution of many independent lattices -------------------- */

typedef struct goc_batch goc_batch;

/* A batch holds up to max_lattices lattices whose total device footprint
 * stays within hbm_budget_bytes; all run on one stream. */
goc_status goc_batch_create(long long hbm_budget_bytes, int max_lattices,
                            const goc_exec *exec, goc_batch **out);
void goc_batch_destroy(goc_batch *b);

/* Admit a lattice (same arguments as goc_create; exec's stream and storage
 * come from the batch unless exec != NULL).  Returns GOC_EBUSY if the budget
 * or the slot count would be exceeded.  Every grid kind may join: per-axis
 * maps, the annular sector and node tables are grouped by kind (one batch
 * kernel per storage type, MIE on/off and grid kind).  *slot receives the
 * slot id. */
goc_status goc_batch_add(goc_batch *b, const goc_grid *grid, const goc_map *map,
                         const goc_flow *flow, const goc_mhd *mhd, int storage, int *slot);

/* Remove a lattice and free its memory. */
goc_status goc_batch_remove(goc_batch *b, int slot);

/* Advance every resident lattice by nsteps with one persistent launch per
 * time step (work items = (lattice, tile) over all lattices). */
goc_status goc_batch_step(goc_batch *b, long long nsteps);

/* Mark a slot for residual checks (on != 0): the last two steps of every
 * later goc_batch_step of >= 2 steps record that lattice's successive fields
 * and reduce R = ||U^n - U^(n-1)|| / ||U^n|| (Sec. 7.3) and the B residual
 * on the device.  Allocates the lattice's two snapshot buffers on first use. */
goc_status goc_batch_check(goc_batch *b, int slot, int on);

/* Residuals from the last goc_batch_step of a checked slot.  Synchronises the
 * batch stream.  Returns GOC_EDIVERGED if that lattice has diverged. */
goc_status goc_batch_residual(goc_batch *b, int slot, double *residual_u, double *residual_b);

/* Access one resident lattice (owned by the batch; do not destroy). */
goc_status goc_batch_lattice(goc_batch *b, int slot, goc_lattice **lat);

/* Bytes the batch currently holds on the device and its budget. */
goc_status goc_batch_usage(const goc_batch *b, long long *used, long long *budget, int *count);

/* ---- one lattice over several GPUs: slabs along xi2 -------------------- */
/* The lattice is cut into bands of xi2 rows ("slabs", one per GPU), as the
 * lattice Boltzmann update allows: a node's new populations depend on its
 * neighbours one row away, and through the second-order normal derivatives of
 * the fields (Appendix E) on rows two away, so two ghost rows per internal cut
 * suffice.  A slab is a lattice of its own rows plus two ghost rows on each
 * side that has a neighbouring slab (both sides on a periodic xi2 axis); it
 * treats its cuts as walls, which makes only the ghost rows wrong, and after
 * every step the ghost rows are overwritten with the two rows of the
 * neighbouring slab nearest the cut (populations, stored force, MIE
 * populations, and the per-row storage reference of 16-bit storage).  The
 * owned rows are then bitwise those of the single lattice: the metric is the
 * global one (q, hence c_s^2, the minimum over the whole lattice, Eq.
 * GOC-LBE_CFL) and the random streams of stochastic rounding follow global
 * node indices.  Per-axis maps (straight grids) only. */

/* A slab owning the global rows [row_begin, row_end) of the lattice `grid`
 * (the whole lattice's grid and map; its nx and W/E sides are the slab's).
 * Needs row_end - row_begin >= 2, and on a periodic xi2 axis at least 2 rows
 * left to the other slabs.  The slab's local rows are: ghost_lo ghost rows,
 * the owned rows, ghost_hi ghost rows (goc_slab_info); goc_moments,
 * goc_moments_device, goc_get_state and goc_init_fields work on all local
 * rows, goc_diagnostics' mass on the owned rows (add the slabs' shares).
 * goc_step takes at most one step per call on a slab, goc_run_until is
 * GOC_EUNSUPPORTED (the residual is a global sum).  Protocol, per slab: after
 * creation, after goc_init_fields / goc_set_state and after every
 * goc_step(slab, 1): goc_slab_pack, send send_lo to the slab below and
 * send_hi to the slab above, receive theirs, goc_slab_unpack (recv_lo from
 * the slab below, recv_hi from the one above). */
goc_status goc_create_slab(const goc_grid *grid, const goc_map *map, const goc_flow *flow,
                           const goc_mhd *mhd, const goc_exec *exec, int row_begin, int row_end,
                           goc_lattice **out);

/* Global rows [*row_begin, *row_end) owned and ghost rows below / above (0, ny,
 * 0, 0 for a whole lattice).  Any pointer may be NULL. */
goc_status goc_slab_info(const goc_lattice *lat, int *row_begin, int *row_end, int *ghost_lo,
                         int *ghost_hi);

/* Bytes of one side's ghost-row message (0 for a whole lattice): every plane
 * of the state, two rows of nx values each, in the storage type, then (16-bit
 * storage) the FP64 per-row storage reference of those rows. */
long long goc_slab_halo_bytes(const goc_lattice *lat);

/* Copy the two owned rows nearest each cut into caller-owned DEVICE buffers
 * of goc_slab_halo_bytes bytes (NULL: that side is skipped; ignored on a side
 * without a neighbour).  Enqueued on the lattice stream; no sync. */
goc_status goc_slab_pack(goc_lattice *lat, void *send_lo, void *send_hi);

/* Overwrite the ghost rows from the neighbours' messages (DEVICE buffers as
 * for goc_slab_pack; NULL skips a side).  Enqueued on the lattice stream. */
goc_status goc_slab_unpack(goc_lattice *lat, const void *recv_lo, const void *recv_hi);

/* ---- errors ------------------------------------------------------------ */
const char *goc_last_error(void);

/* Guard bands (a debug aid in place of a device memory checker): when the
 * environment variable GOC_GUARD_BANDS is set at goc_create, the padding
 * columns of every population, force and MIE plane and a 64 KB tail after
 * each such buffer are filled with a canary byte, which no kernel writes.
 * goc_check_guards counts the guard bytes that changed (*bad; 0 when no stray
 * write happened).  Synchronises.  GOC_EINVAL if the lattice has no guards.
 * goc_set_state rewrites the padding with the saved state's bytes. */
goc_status goc_check_guards(goc_lattice *lat, long long *bad);

/* Failure-detection self-test: one block waits on a device barrier that
 * nothing completes and gives up after `polls` polls (1 .. 2^26), the way
 * every device-side wait of the step kernels is bounded.  Returns
 * GOC_ETIMEOUT when the wait ran out (the expected outcome); the device stays
 * usable.  GOC_EINVAL for a poll count out of range. */
goc_status goc_selftest_bounded_wait(long long polls);

#ifdef __cplusplus
}
#endif

#endif /* GOC_H */
