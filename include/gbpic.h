/*
 * gbpic — C-ABI of the GB300 (sm_103a) hot path of the relativistic-reference-frame (RRF,
 * boosted-frame) particle-in-cell method of arXiv 2411.04703.
 *
 * The calls follow the paper's statement of the problem: a Maxwell solver and current
 * weighting in a frame moving at gamma_R (Sec. "Relativistic booster frame", Eq. Max1-Max4),
 * a beam defined in the laboratory frame and transformed by the code (Eq. Lor1, Lor2,
 * RRFVel; the beam paragraph of Sec. "Electron propagation in vacuum"), static lab elements
 * (undulator, plasma) transformed into the RRF (Eq. M1-M4, Nnormi, Vprime), a moving window
 * with absorbing field boundaries and dummy particles, and a leap-frog push.
 *
 * Units (normalisation rule stated with Table I): c = 1, time in 1/w_n, length in c/w_n,
 * momentum u = p/(m_e c), fields in m_e c w_n / e, densities in n_n = eps0 m_e w_n^2/e^2.
 * Then dE/dt = curl B - J, dB/dt = -curl E, div E = rho.
 *
 * Conventions shared by every call:
 *  - Every function returns an int status: PIC_OK (0) or a negative PIC_ERR_* code.  No
 *    exception or signal crosses the ABI.  pic_last_error() gives a message.
 *  - Errors are sticky: after a device-side error (PIC_ERR_DEVICE) or a CUDA error the
 *    context refuses further work and only pic_last_error / pic_destroy are valid.
 *  - Host arrays are borrowed for the duration of the call only.  Pointers documented as
 *    "host or device" may be either (the copy uses cudaMemcpyDefault).
 *  - Grid arrays are float, x fastest: index = (k * ny + j) * nx + i.  Yee staggering:
 *    E_x at (i+1/2, j, k), E_y at (i, j+1/2, k), E_z at (i, j, k+1/2), B_x at
 *    (i, j+1/2, k+1/2), B_y at (i+1/2, j, k+1/2), B_z at (i+1/2, j+1/2, k), J like E,
 *    rho at the nodes (i, j, k).
 *  - Every call that launches work enqueues it on the context's stream and returns without
 *    waiting, except the getters, which synchronise that stream.
 *  - Limits: nx, ny <= 1024; bits(nx) + bits(ny) + bits(nz) <= 31 (the cell index is packed
 *    into one int32); 8 nx ny nz < 2^31 (sort keys); fewer than 2^31 particles per species.
 */
#ifndef GBPIC_H
#define GBPIC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define PIC_OK 0
#define PIC_ERR_ARG (-1)       /* invalid argument (message says which) */
#define PIC_ERR_CUDA (-2)      /* a CUDA runtime call failed */
#define PIC_ERR_ALLOC (-3)     /* device allocation failed (allocator returned NULL) */
#define PIC_ERR_STATE (-4)     /* call not valid in the context's state (e.g. poisoned) */
#define PIC_ERR_DEVICE (-5)    /* a kernel raised its device error word (see message) */
#define PIC_ERR_CAPACITY (-6)  /* a species' particle storage is full */

enum { PIC_BC_PERIODIC = 0, PIC_BC_PML = 1, PIC_BC_OPEN = 2 };
enum { PIC_FRAME_LAB = 0, PIC_FRAME_BOOSTED = 1 };
enum {
    PIC_EX = 0, PIC_EY, PIC_EZ, PIC_BX, PIC_BY, PIC_BZ, PIC_JX, PIC_JY, PIC_JZ, PIC_RHO
};
enum { PIC_EXT_NONE = 0, PIC_EXT_PLANAR_UNDULATOR = 1, PIC_EXT_PLANAR_UNDULATOR_3D = 2 };
enum { PIC_PUSHER_BORIS = 0, PIC_PUSHER_VAY = 1 };
enum { PIC_GATHER_MOMENTUM = 0, PIC_GATHER_ENERGY = 1 };

typedef struct pic_ctx pic_ctx;

typedef struct { int nx, ny, nz; } pic_grid;

/* Field boundaries per face (face[d][0] low, face[d][1] high; a periodic dim must be
 * periodic on both faces).  PIC_BC_PML: convolutional PML of pml_cells cells ("the fields
 * are absorbed upon interaction with the boundaries", Sec. "Relativistic booster frame");
 * PIC_BC_OPEN: field values outside the grid are zero.  Particles whose cell leaves
 * [margin_lo, n-1-margin_hi] of a non-periodic dim become dummy (inactive) particles
 * (margins 1/2 for CIC, 2/3 for TSC).  moving_window: the window moves along +z at
 * window_v (units of c) in whole cells, floor(window_v n dt / dz) shifts by step n
 * (the paper's moving window "adjusted to the RRF time-step"). */
typedef struct {
    int face[3][2];
    int pml_cells;
    int moving_window;
    double window_v;
} pic_boundaries;

/* Device memory and stream supplied by the caller (e.g. PyTorch's caching allocator and
 * current stream).  alloc/free may be NULL (then cudaMalloc/cudaFree are used); stream may
 * be NULL (then the context creates its own non-blocking stream).  device: CUDA ordinal. */
typedef struct {
    void *(*alloc)(size_t bytes, void *user);
    void (*free)(void *ptr, size_t bytes, void *user);
    void *user;
    void *stream;
    int device;
} pic_device;

/* Create a simulation context: grid of nx*ny*nz cells of size dx[3] (normalised), time step
 * dt, frame Lorentz factor gamma_boost >= 1 (beta_R = sqrt(1 - 1/gamma^2), Eq. RRFVel),
 * boundaries bc, particle shape order 1 (CIC) or 2 (TSC).  Fields start at zero.  dt must
 * satisfy the Yee Courant limit dt < 1/sqrt(sum 1/dx_i^2).  On success *out owns all device
 * state (allocated through dev); on failure *out is NULL and the status says why
 * (pic_last_error(NULL) gives the message of a failed create).
 * A 2-D geometry (the x-z plane of the paper's runs, everything uniform along y) is a grid with
 * ny = 1 and a periodic y: the particle shape then sums to one on the single y node, the
 * Esirkepov current's y component becomes the out-of-plane current q w v_y (shape of the
 * average x-z position), and the curl's y derivatives vanish.  Any periodic dim may be shorter
 * than the stencil; its indices wrap modulo its size. */
int pic_create(pic_ctx **out, pic_grid grid, const double dx[3], double dt, double gamma_boost,
               const pic_boundaries *bc, int shape_order, const pic_device *dev);

/* Ensemble of `runs` independent simulations in one context (batched sweeps of undulator K and
 * plasma density with uneven beam sizes): every run has the grid `grid`, cell size, time step,
 * boost, boundaries and shape order given here, and its own particles, plasma density and
 * undulator K.  The runs are stacked along z (run r owns rows r*nz .. (r+1)*nz - 1 of a grid of
 * nx x ny x runs*nz cells; grid arrays and particle cells use that stacked index), z must be
 * periodic and is periodic inside each run, so no field, particle or current crosses between
 * runs.  One pic_step advances every run with one launch per kernel (the particle kernel's work
 * items span all runs).  nz must be a multiple of the tile's z size.  Per-run setup:
 * pic_load_species_batch, pic_set_external_field_batch, pic_set_plasma_batch; per-run
 * diagnostics: pic_get_moments_run.  runs = 1 is the same as pic_create. */
int pic_create_batch(pic_ctx **out, int runs, pic_grid grid, const double dx[3], double dt,
                     double gamma_boost, const pic_boundaries *bc, int shape_order,
                     const pic_device *dev);

/* Tile size for the per-tile sort and the particle kernel (cells, each 1..16), number of
 * steps between sorts (>= 1), and the margin (cells, 0..2) a particle may drift outside its
 * tile between sorts before it takes the slower global-memory path.  Defaults 8x8x8, 8, 1. */
typedef struct {
    int tile[3];
    int sort_every;
    int margin;
} pic_tuning;
int pic_set_tuning(pic_ctx *ctx, const pic_tuning *t);

/* A particle population (beam electrons, plasma electrons and ions are separate
 * populations, Sec. "Relativistic booster frame").  q, m in units of e and m_e; frozen:
 * momentum never pushed (lab-immobile ions drift at -beta_R in the RRF and carry their own
 * current j_i = v_R rho_i, deposited with the same weighting).  capacity: maximum particles
 * held (>= n of the load).  origin: grid coordinate (cells) of the loaded positions' zero.
 * match_undulator (lab frame only): the beam is already inside the undulator — before the
 * transform, u_x += -(q/m) A_x(z_lab) at the event's lab coordinate z + gamma_R origin_z dz
 * and u_z is lowered so that the lab energy is unchanged. */
typedef struct {
    double q, m;
    int frozen;
    int64_t capacity;
    double origin[3];
    int match_undulator;
} pic_species;

/* Create a species and load n particles (n may be 0).  x, u: host FP64 arrays [3][n]
 * (component-major), w: host FP64 [n] weights (real particles per macroparticle,
 * normalised) or NULL for 1.  frame PIC_FRAME_LAB: x are lab positions at lab time 0 relative
 * to the reference point, u lab momenta; each event is Lorentz-transformed (Eq. Lor1-Lor2),
 * its momentum boosted, and the particle drifted ballistically to t' = 0 (Eq. BGauss/Belon
 * take the distribution at t' = 0); all in FP64 on the device.  frame PIC_FRAME_BOOSTED: x
 * are RRF positions at t' = 0.  Grid coordinate = x/dx + origin; particles outside the active
 * region are dropped.  Particle ids are 0..n-1 in load order.  *species_id receives the id. */
int pic_load_species(pic_ctx *ctx, const pic_species *sp, int64_t n, const double *x,
                     const double *u, const double *w, int frame, int *species_id);

/* Ensemble form of pic_load_species: one species spanning every run, n_run[r] particles loaded
 * into run r (host int64[runs]).  x, u: host FP64 [3][n] and w: [n] or NULL, with n the sum of
 * n_run, run-major (the particles of run 0 first).  origin is in each run's own cell
 * coordinates; run r's particles wrap inside its rows; each run's undulator K is used for
 * match_undulator.  Ids are numbered 0..n-1 across the runs in that order.  Also valid on a
 * single-run context (n_run[0] = n). */
int pic_load_species_batch(pic_ctx *ctx, const pic_species *sp, const int64_t *n_run,
                           const double *x, const double *u, const double *w, int frame,
                           int *species_id);

/* Static lab element transformed into the RRF.  PIC_EXT_PLANAR_UNDULATOR: lab field
 * B_y = B0 f(z) cos(k_u z + phase), B0 = K k_u (K = e B0/(m c k_u)), k_u = 2 pi/lambda_u;
 * f = 0 before z_start, linear to 1 over ramp_len (the entrance "gentle slope", Sec.
 * "Electron propagation ... under external field"), 1 after; ramp_len < 0 or
 * z_start = -inf: f = 1 everywhere.  In the RRF the element moves at -c beta_R (Eq. Vprime):
 * the particle at RRF z', t' sees lab z = gamma_R (z' + beta_R t') and Eq. M1-M4 give
 * B'_y = gamma_R B_y, E'_x = -beta_R B'_y.  Evaluated analytically at each particle, added to
 * the gathered self fields.  lambda_u, z_start, ramp_len: lab, normalised.
 * PIC_EXT_PLANAR_UNDULATOR_3D: the same element with the transverse dependence of a planar
 * undulator's vacuum field (poles above and below in y), B_y = B0 f(z) cosh(k_u y) cos(k_u z +
 * phase), B_z = -B0 f(z) sinh(k_u y) sin(k_u z + phase) (divergence- and curl-free where f = 1),
 * y measured from the undulator axis, which is the grid's y mid-plane (y = ny dy / 2).  The
 * longitudinal component is unchanged by the boost (Eq. M1-M4: B'_z = B_z); B'_y and E'_x as
 * above.  A matched load (match_undulator) then uses A_x = (B0/k_u) cosh(k_u y) sin(k_u z +
 * phase).  The adjoint (pic_checkpoint) supports PIC_EXT_PLANAR_UNDULATOR only. */
typedef struct {
    int type;
    double K, lambda_u, phase, z_start, ramp_len;
} pic_external;
int pic_set_external_field(pic_ctx *ctx, const pic_external *f);

/* Ensemble form: f[runs] (host), one element per run; the runs may differ in K only (same
 * type, lambda_u, phase, z_start and ramp_len, and no entrance ramp: the undulator fills each
 * periodic run).  On an ensemble, pic_set_external_field gives every run the same K. */
int pic_set_external_field_batch(pic_ctx *ctx, const pic_external *f);

/* Background plasma (Sec. "Relativistic booster frame": N'_e = gamma_R N_e, Eq. Nnormi;
 * static lab elements move at -c beta_R, Eq. Vprime; plasma enters the window on one side
 * and leaves on the other).  Creates two species, electrons (q = -1, m = 1) and co-located
 * frozen ions (q = +1, same weighting), with cold momentum u'_z = -gamma_R beta_R, on a
 * regular lattice of ppc[0]*ppc[1]*ppc[2] per cell in the transverse cell range
 * x_range = {x0, x1, y0, y1}.  Lattice plane m sits at RRF z' = ((m + 1/2)/ppc_z) dz -
 * beta_R t'; its lab position gamma_R (m + 1/2) dz / ppc_z sets the lab density
 * n(z_lab) (piecewise linear through n_nodes points (z_nodes, density), zero outside) and
 * the weight gamma_R n dx dy dz / (ppc_x ppc_y ppc_z).  Fills the window now; every later
 * step injects the planes whose grid coordinate fell below nz - margin_hi.  Particles are
 * ordered and numbered by (plane, y cell, x cell, y sub, x sub).  Arrays are host FP64. */
typedef struct {
    int ppc[3];
    int x_range[4];
    int n_nodes;
    const double *z_nodes;
    const double *density;
    int64_t capacity;   /* per species; 0: computed from the window and the sort cadence */
} pic_plasma;
int pic_set_plasma(pic_ctx *ctx, const pic_plasma *p, int *electron_id, int *ion_id);

/* Periodic z (a single run or an ensemble): the lattice fills the whole box once (planes
 * 0 .. ppc_z * nz - 1, each run's planes with the profile in the run's own coordinates) and
 * drifts around it; no plane is injected later.  Ensemble form: density_scale (host FP64
 * [runs], >= 0) multiplies the profile of run r. */
int pic_set_plasma_batch(pic_ctx *ctx, const pic_plasma *p, const double *density_scale,
                         int *electron_id, int *ion_id);

/* Advance n steps (Sec. "Relativistic booster frame": leap-frog push and current weighting
 * for Eq. Max3-Max4, Maxwell Eq. Max1-Max2).  Per step: every `sort_every` steps a per-tile
 * counting sort of each species by cell; per species a fused kernel gathers E^n, B^n (same
 * shape as the deposit, each component at its Yee point) plus the external field at t'_n,
 * pushes u^{n-1/2} -> u^{n+1/2} (Boris; frozen species skip it), moves x^n -> x^{n+1} and
 * deposits the Esirkepov current J^{n+1/2}; then B^{n+1/2} = B^n - dt/2 curl E^n,
 * E^{n+1} = E^n + dt (curl B^{n+1/2} - J), B^{n+1} = B^{n+1/2} - dt/2 curl E^{n+1} (with CPML);
 * then the window shifts due by step n+1 and plasma planes entering the front are injected.
 * The current of a tile is summed exactly in fixed point (order-independent) with a scale set per
 * species and step from four times the largest displacement of the previous step; a particle
 * moving further, and every particle of a tile holding fewer than 32, adds its current with
 * float atomics instead.  Without a moving window or plasma injection (periodic z) and with
 * tracing off, whole pairs of sort periods are captured once into a CUDA graph and replayed
 * (see pic_use_graphs); a step counter on the device gives each replayed step its time.
 * Asynchronous on the context stream. */
int pic_step(pic_ctx *ctx, int64_t n);

/* Momentum push of every mobile species.  PIC_PUSHER_BORIS (default): the Boris rotation, the
 * reading of the paper's second-order leap-frog.  PIC_PUSHER_VAY: Vay's pusher, the modified
 * pusher the paper cites for boosted-frame runs (Sec. 1): a half kick with the old velocity and
 * a rotation whose Lorentz factor solves a quadratic, exact for E + v x B = 0 drifts (a
 * lab-static plasma inside the undulator, seen from the RRF).  The adjoint needs Boris. */
int pic_set_pusher(pic_ctx *ctx, int pusher);

/* Field gather of every mobile species.  PIC_GATHER_MOMENTUM (default): each component is
 * interpolated with the deposit's shape at its Yee point (the reading of the paper's scheme).
 * PIC_GATHER_ENERGY: one order lower along the dims where the component is staggered (CIC -> nearest
 * grid point, TSC -> CIC there), the transpose of the Esirkepov deposit: the x-shape of J_x is
 * the lower-order shape at the half-integer nodes, so for a gradient field E = -grad_h phi the
 * gathered E_x is exactly -d/dx of phi interpolated with the full shape, and B = curl_h A
 * gathers to the curl of the gathered A.  The adjoint needs PIC_GATHER_MOMENTUM.  PIC_ERR_ARG
 * for an unknown scheme; PIC_ERR_STATE while adjoint checkpoints are recorded. */
int pic_set_gather(pic_ctx *ctx, int gather);

/* Artificial neutralising ions (Sec. "Electron propagation in vacuum and under external field":
 * a background of ions compensating the beam's charge, damped linearly over T_ion so that the
 * beam's fields build up without the kick of a sudden charge).  From the current step, a static
 * charge density -rho_s (rho_s: species species_id's density now, with the deposit's shape)
 * fades to zero linearly over T_ion (normalised time).  Reading (the paper does not say how
 * Gauss's law survives the fading): in a charge-conserving scheme a charge fades only through a
 * current, so the ions carry J_z with div J = -d rho_ion/dt, J_z(i, j, k + 1/2) = -(dz/T_ion)
 * sum_{k' <= k} rho_s(i, j, k'), the prefix along z from the low face (the current leaves through
 * the high z face).  On a periodic z the column mean of rho_s cannot leave the box and stays as a
 * uniform neutralising background.  Fields must start at zero (the total charge is zero then);
 * the ions move down with a moving window.  Gauss's law div E = rho_particles + rho_ion(t) then
 * holds to rounding at every node through the ramp.  T_ion <= 0 removes the ions.  Replay of
 * captured steps (pic_use_graphs) is off while they exist.  PIC_ERR_ARG for an unknown species;
 * PIC_ERR_STATE while adjoint checkpoints are recorded. */
int pic_set_ion_ramp(pic_ctx *ctx, int species_id, double T_ion);


/* Replay of captured step sequences in pic_step (on = 1, the default) or one launch per kernel
 * (on = 0).  The capture is redone when species, the external field or the tuning change; if
 * capturing fails the context falls back to launching. */
int pic_use_graphs(pic_ctx *ctx, int on);

/* Autotuner of the tile-sort cadence at the context's current tile size (pic_autotune_tiles
 * below also chooses the tile).  Runs trials of whole sort periods (>= 32 steps each) with
 * sort_every = 1, 2, 3, 4, 6,
 * 8, 12, 16, 24, 32 (up to max_sort_every), each starting with a sort, in two passes (ascending,
 * then descending), times them with CUDA events on the context stream and keeps the fastest per
 * step (a rarer sort must win by 2 %).  The trial steps are real steps: the simulation advances
 * by their total (about 500 steps for max_sort_every = 16).  A fast drift (cells per step)
 * favours frequent sorts, a slow one rare sorts.  *sort_every_out (may be NULL) receives the
 * choice.  Synchronous. */
int pic_autotune(pic_ctx *ctx, int max_sort_every, int *sort_every_out);

/* Autotuner of the tile size and the sort cadence together.  tiles: host int[n_tiles][3],
 * candidate tile sizes (the first is the reference, e.g. the current 8 x 8 x 8); each must pass
 * pic_set_tuning's checks (1..16 cells per dim, the region within shared memory, for an ensemble
 * a z size dividing the rows of a run), else PIC_ERR_ARG.  Every candidate runs whole periods of
 * the current cadence (>= 32 steps, the first step sorting on the new tiles), in two passes
 * (ascending, then descending); the fastest per step is kept (a candidate must beat the best
 * before it in the list by 2 %), then pic_autotune picks the cadence for it.  The trials
 * advance the run.  Changing the tile reallocates the species' tile tables through the context's
 * allocator; the tile sizes 8 x 8 x 8 use the kernel's compiled region, others its runtime-sized
 * one.  tile_out (host int[3]) and sort_every_out receive the choice (either may be NULL).
 * PIC_ERR_STATE while adjoint checkpoints are recorded. */
int pic_autotune_tiles(pic_ctx *ctx, const int *tiles, int n_tiles, int max_sort_every, int *tile_out,
                       int *sort_every_out);

/* Wait for the context stream; returns PIC_ERR_DEVICE if a kernel raised the error word. */
int pic_sync(pic_ctx *ctx);

/* Force a per-tile sort of every species now (the sort also compacts dummy particles).  Order:
 * tiles x-fastest; inside a tile the cells x fastest, then z, then y; inside a cell the octant
 * of the offset (bit d set when offset_d >= 1/2); order among equal keys unspecified. */
int pic_sort(pic_ctx *ctx);

/* Copy one grid component (PIC_EX..PIC_JZ; J is the current of the last step) or the charge
 * density PIC_RHO (deposited now from every species with the particle shape) into dst
 * (host or device, n = nx*ny*nz floats).  Synchronous. */
int pic_get_fields(pic_ctx *ctx, int which, float *dst, size_t n);

/* Overwrite one grid component (PIC_EX..PIC_JZ) from src (host or device, n = nx*ny*nz
 * floats), e.g. to restart from saved fields.  Asynchronous on the context stream for device
 * sources; synchronous for host sources. */
int pic_set_fields(pic_ctx *ctx, int which, const float *src, size_t n);

/* Copy the live particles of a species to host arrays of capacity `cap`: cell indices
 * [3][cap] (int32 i, j, k), in-cell offsets [3][cap] (float, [0,1)), momenta [3][cap], weights
 * [cap] and ids [cap], in storage order (tile-sorted order after a sort).  Any output pointer
 * may be NULL.  *n_out receives the number of live particles (PIC_ERR_CAPACITY if > cap).
 * Synchronous. */
int pic_get_particles(pic_ctx *ctx, int species_id, int64_t cap, int64_t *n_out, int32_t *cell,
                      float *off, float *u, float *w, int64_t *id);

/* FP64 beam diagnostics (precision split: FP64 for back-transformed diagnostics
 * and conservation sums).  frame PIC_FRAME_BOOSTED: at t' = step dt, positions in
 * normalised RRF length (z' absolute, window shifts included).  PIC_FRAME_LAB: each
 * particle's RRF event and momentum are transformed back (inverse Eq. Lor1-Lor2) and drifted
 * ballistically to the weighted mean lab time (one RRF instant spans the lab times of
 * Eq. DT).  bunching = |sum w exp(-i k z)| / sum w at wavenumber k_bunch of that frame.
 * Normalised emittance sqrt(<dx^2><du^2> - <dx du>^2) (central, weighted); relative energy
 * spread std(gamma)/mean(gamma); kinetic energy sum w m (gamma - 1); field energy
 * (1/2) sum (E^2 + B^2) dV over the grid.  Synchronous. */
typedef struct {
    double count, sum_w, charge;
    double mean[3], rms[3], mean_u[3];
    double mean_gamma, rel_energy_spread;
    double emit_n[2];
    double bunching, kinetic_energy, mean_t, field_energy;
} pic_moments;
int pic_get_moments(pic_ctx *ctx, int species_id, int frame, double k_bunch, pic_moments *out);

/* Lab-frame reconstruction at one lab time (Sec. "Understanding the RRF", Eq. delta2electrons,
 * Eq. DT): the particles of one RRF instant sit at lab times spread by gamma_R beta_R dz', so a
 * lab snapshot at lab time t_lab is assembled particle by particle while the RRF steps pass
 * through it.  In every step a particle moves on a straight RRF segment from x^n to x^{n+1} with
 * momentum u^{n+1/2}; when the segment's lab times gamma_R (t' + beta_R z') span t_lab, its event
 * at t_lab is transformed to the lab (inverse Eq. Lor1-Lor2; x, y unchanged) with the lab
 * momentum of u^{n+1/2} and recorded in FP64 under the particle's id.  Lab coordinates are those
 * of the grid's absolute RRF coordinates (x' = cell + offset in units of d, z' counting window
 * shifts): the lab origin and clock coincide with the RRF's at the grid's origin node.
 * pic_lab_snapshot arms a snapshot of particle species species_id (ids 0 .. next id - 1; a
 * particle already at or past t_lab is marked missed); t_lab = NaN disarms and frees it.  While
 * armed, every step runs one more kernel over the species, and replay of captured steps is off.
 * pic_lab_snapshot_read copies the records (rec: host or device double[n][7] = lab x, y, z, u_x,
 * u_y, u_z, w) and states (host uint8[n]: 0 pending, 1 recorded, 2 missed) for n >= *n_ids ids;
 * rec and state may be NULL; *n_ids and *recorded (may be NULL) receive the number of ids and of
 * recorded particles.  pic_lab_snapshot_moments gives the moments of the recorded particles with
 * the definitions of pic_get_moments (bunching at the lab wavenumber k_bunch; mean_t = t_lab;
 * field_energy 0).  Synchronous.  A periodic z is taken in the box's own image.  PIC_ERR_ARG for a
 * lattice species, an unknown species or an ensemble; PIC_ERR_STATE when none is armed. */
int pic_lab_snapshot(pic_ctx *ctx, int species_id, double t_lab);
int pic_lab_snapshot_read(pic_ctx *ctx, double *rec, uint8_t *state, int64_t n, int64_t *n_ids, int64_t *recorded);
int pic_lab_snapshot_moments(pic_ctx *ctx, double k_bunch, pic_moments *out);

/* pic_get_moments restricted to the particles and field cells of one run of an ensemble
 * (0 <= run < runs); positions are in the run's own coordinates.  Synchronous. */
int pic_get_moments_run(pic_ctx *ctx, int species_id, int run, int frame, double k_bunch,
                        pic_moments *out);

/* Step count, window shifts and last injected plasma plane of the context: out[3]. */
int pic_get_time(pic_ctx *ctx, int64_t out[3]);

/* Number of live particles of a species (synchronous; dummy particles not yet compacted by
 * a sort are not counted). */
int pic_get_count(pic_ctx *ctx, int species_id, int64_t *n_out);

/* Tracing: per-kernel-class device time from CUDA events recorded on the context stream
 * around every launch group of pic_step / pic_sort, and the number of kernels launched.
 * Classes: 0 tile sort, 1 particle kernel of mobile species, 2 particle kernel of frozen
 * species, 3 field update (FDTD + CPML), 4 moving-window shift, 5 plasma injection, 6 other.
 * pic_trace_read synchronises the stream, returns the figures accumulated since the last read
 * (events[k]: timed launch groups of class k) and resets them.  Disabled by default. */
typedef struct {
    double ms[8];
    int64_t events[8];
    int64_t kernels;
    int64_t fallback;   /* particles whose current took global float atomics because they moved
                           beyond the step's fixed-point range (see pic_step) */
} pic_trace;
int pic_trace_enable(pic_ctx *ctx, int on);
int pic_trace_read(pic_ctx *ctx, pic_trace *out);

/* Allocation-free counting sort of caller-owned arrays, for callers that cannot let a library
 * allocate device memory (an application that reserves its whole device budget in its own
 * pool at start-up and forbids allocations afterwards, or code running where the CUDA
 * allocator must not be entered).  The paper has no counterpart: it is a tile counting sort like
 * the one pic_step runs internally, but with its own key (below; pic_step's internal key orders
 * the cells of a tile differently and adds the offset's octant).  cells: device int32[n], packed
 * cell indices i | j << 10 | k << 20 (-1 or a cell outside the grid = dummy, dropped); grid,
 * tile: host int[3] (grid <= 1024 x 1024 x 2048, 1 <= tile <= grid); order: device int32[n],
 * receives at sorted position q the index of the input element placed there (live elements
 * only, ascending key; order among equal keys unspecified).  The key of cell (i, j, k) with
 * nt_d = ceil(grid_d / tile_d) tiles per dim is
 *   key = ((k / T_z) nt_y + j / T_y) nt_x + i / T_x) * (T_x T_y T_z)
 *         + ((k % T_z) T_y + j % T_y) T_x + i % T_x,
 * i.e. tiles x-fastest, then the cells of a tile x-fastest.  key_start: device int32[n_keys + 1]
 * with n_keys = nt_x nt_y nt_z T_x T_y T_z, receives the exclusive start of each key
 * (key_start[n_keys] = number of live elements); stream: cudaStream_t or NULL.
 * Limits: n <= PIC_NOALLOC_MAX_N, n_keys <= PIC_NOALLOC_MAX_KEYS; larger sizes return
 * PIC_ERR_ARG with a message in pic_last_error(NULL).  Scratch comes from a fixed device array
 * inside the library (about 4 MB per GPU that loads the library, held until the process
 * exits); the first call on each device looks up its address (with that device current), so
 * make the first call before any stream capture.  The address found then is kept for the life of
 * the process: it belongs to the device's primary context, so do not call this entry point after
 * a cudaDeviceReset of that device or with another (non-primary) context current.  It calls no cudaMalloc/cudaFree.  All calls
 * share that scratch: calls whose work overlaps on the GPU race and give wrong results.
 * Asynchronous on `stream`. */
#define PIC_NOALLOC_MAX_N (1 << 20)
#define PIC_NOALLOC_MAX_KEYS (1 << 22)
int pic_tile_sort_noalloc(const int32_t *cells, int64_t n, const int grid[3], const int tile[3],
                          int32_t *order, int32_t *key_start, void *stream);

/* Adjoint (reverse-mode gradient) of a beam diagnostic with respect to the undulator K and the
 * plasma density profile, by a hand-written discrete adjoint of the step: the field update's
 * transpose runs time-reversed (the transpose of the forward-difference curl is the
 * backward-difference curl), the deposit's transpose gathers the adjoint current, the gather's
 * transpose scatters into the field adjoints, and Boris and the move are reversed per particle
 * from the recorded state.  Memory is traded for recomputation: pic_checkpoint(every_k) saves the
 * state at the start of the differentiated interval and every every_k steps after (pic_step then
 * also sorts at those steps); pic_backward restores each checkpoint in reverse order, recomputes
 * its segment recording every step, and runs the segment's adjoint.  Requirements: first-order
 * shape, Boris pusher, momentum-conserving gather, one run, periodic grid, no moving window or
 * PML, the 1-D planar undulator field without entrance ramp, no artificial ions; otherwise
 * PIC_ERR_ARG and nothing is recorded.  every_k <= 0 turns recording off
 * and frees the checkpoints.  The checkpoints and the per-step records of one segment are device
 * allocations of the context (about 250 MB per recorded step for 6.3M particles on 64x64x256). */
int pic_checkpoint(pic_ctx *ctx, int every_k);

/* Loss: the bunching factor of species_id in the boosted frame at the current step,
 * L = |sum w exp(-i k z')| / sum w (k = k_bunch, z' including window shifts).  The initial state
 * of the interval is held fixed: dL/dK is through the undulator field seen during the steps (a
 * beam loaded matched to the undulator keeps its loaded momenta), dL/dprofile through the
 * weights of the plasma electrons and the frozen ions, w = gamma_R n_lab(z_lab) dV / ppc with
 * n_lab piecewise linear through the profile nodes (Eq. Nnormi).  The context is left at the
 * state it had before the call.  Synchronous.  Errors: PIC_ERR_ARG for a NULL seed or out, a
 * seed species that is not a particle species, or more profile nodes than pic_grads holds;
 * PIC_ERR_STATE when pic_checkpoint was not called before the steps; PIC_ERR_ALLOC,
 * PIC_ERR_CUDA or PIC_ERR_DEVICE from the recomputation and the sweep.  out is caller-owned; its
 * contents are meaningful only when PIC_OK is returned. */
typedef struct {
    int species_id;
    double k_bunch;
} pic_adjoint_seed;
typedef struct {
    double loss;
    double dL_dK;
    int n_profile;               /* profile nodes given to pic_set_plasma (0 without plasma) */
    double dL_dprofile[64];
} pic_grads;
int pic_backward(pic_ctx *ctx, const pic_adjoint_seed *seed, pic_grads *out);

/* Relativistic resolution factor of the context's grid (Eq. Rrf1):
 * R_RF = (8 L_wind / N_z) sqrt((1 - beta_R)/(1 + beta_R)), L_wind / N_z the longitudinal cell
 * (of one run for an ensemble), i.e. eight RRF cells mapped back to the lab wavelength they
 * resolve.  *ok = (R_RF < lambda_lab): the radiation of lab wavelength lambda_lab (normalised
 * units, e.g. the resonant wavelength of Eq. RadLambda) gets at least eight cells per RRF
 * wavelength.  Host-only; no device work. */
int pic_resolution_factor(const pic_ctx *ctx, double lambda_lab, double *r_rf, int *ok);

/* FEL resonant wavenumber of the bunching diagnostic (Eq. RadLambda, Sec. "Relativistic booster
 * frame"): the lab wavelength lambda_l = lambda_u (1 + K^2/2) / (2 gamma_B^2) radiated by a beam of
 * lab Lorentz factor gamma_B in a planar undulator of strength K and lab period lambda_u
 * (normalised units).  frame PIC_FRAME_LAB: *k = 2 pi / lambda_l.  frame PIC_FRAME_BOOSTED: the
 * image of that wave pattern, moving with the beam's mean lab velocity beta_z (1 - beta_z =
 * (1 + K^2/2) / (2 gamma_B^2)), in the frame of Lorentz factor gamma_R: *k = gamma_R (1 - beta_z
 * beta_R) 2 pi / lambda_l, the inverse of the beam elongation of Eq. Belon at the mean velocity
 * (formed without cancellation at large gamma).  Host-only, FP64, no context and no device work.
 * Errors: PIC_ERR_ARG for k NULL, lambda_u <= 0, K < 0, gamma_B < 1, gamma_R < 1, a non-finite
 * argument or an unknown frame (message in pic_last_error(NULL)). */
int pic_resonant_wavenumber(double K, double lambda_u, double gamma_B, double gamma_R, int frame, double *k);

/* Release every device allocation of the context.  NULL is accepted. */
int pic_destroy(pic_ctx *ctx);

/* Message of the last error of ctx (of the last failed pic_create when ctx is NULL).  The
 * string is owned by the library and valid until the next call on ctx. */
const char *pic_last_error(const pic_ctx *ctx);

#ifdef __cplusplus
}
#endif
#endif /* GBPIC_H */
