/*
 * cgdem.h -- C ABI of the GB300 (sm_103a) library for the per-timestep
 * DEM contact and fluid-coupling step of the coarse-grained CFD-DEM method of
 * Kazidenov, Khamitov & Amanbek, "Coarse-graining of CFD-DEM for simulation
 * of sand production in the modified cohesive contact model" (arXiv
 * 2211.06142).
 *
 * What one step computes (Sec. 2.1-2.3):
 *   - Newton-Euler motion of spheres (Eq. 1-2), integrated by velocity Verlet
 *     with positions, velocities and the integrator update in FP64;
 *   - contact forces: the modified JKR law (Eq. 12-13, Table 1, Sec. 2.3:
 *     bonds break at point C and never reform; new contacts are Hertz),
 *     normal damping (Eq. 32-33), tangential spring-dashpot with per-contact
 *     history and Coulomb limit (Eq. 4, 35), contact torque (Eq. 5);
 *     Hertz walls of a cylindrical sample (Sec. 3.1 particle-wall contacts);
 *   - porosity n per fluid cell from a fixed-point particle-volume scatter
 *     (n of Eq. 6) and the Di Felice drag gathered back (Eq. 8-11),
 *     gravity and buoyancy (Eq. 1);
 *   - coarse-grained parameters by the SSW / SSP rules (Sec. 2.4, Eq. 14-35,
 *     Table 3): only the surface energy changes, gamma_g = k gamma_p.
 *
 * Conventions.
 *   - Units are SI.  Every function returns a cgdem_status (0 = OK, < 0 =
 *     error) unless stated.  Errors are also described by cgdem_last_error.
 *   - Particles are numbered by their position in the arrays passed to
 *     cgdem_init_particles (the "id"); samples are consecutive id ranges.
 *     Every host array that this library reads or writes is in id order.
 *   - "stream" is a cudaStream_t passed as void* (NULL = legacy default
 *     stream).  All device work of a call is enqueued on that stream; calls
 *     that copy to or from host memory synchronise it before returning.
 *   - Device memory belongs to the caller: the library carves one workspace
 *     (size from cgdem_workspace_size) and never calls cudaMalloc/cudaFree.
 *     The context object itself is host memory owned by the library.
 *   - A context is not thread-safe; calls on one context must not overlap.
 *   - Device-side errors (contact-list capacity exceeded, a bond that left
 *     the candidate list, a non-finite force) are latched in a status word on
 *     the device and returned by the next cgdem_status_sync or cgdem_get_*.
 */
#ifndef CGDEM_H
#define CGDEM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    CGDEM_OK = 0,
    CGDEM_E_INVALID = -1,   /* bad argument; nothing was enqueued */
    CGDEM_E_CAPACITY = -2,  /* a particle has more candidate neighbours than max_neighbors */
    CGDEM_E_CUDA = -3,      /* a CUDA runtime call failed */
    CGDEM_E_NONFINITE = -4, /* a force or position became NaN/Inf */
    CGDEM_E_TIMEOUT = -5,   /* a bounded device-side wait expired (the kernel gave up and returned) */
    CGDEM_E_STATE = -6      /* call out of order, or a bonded pair left the candidate list */
} cgdem_status;

typedef enum { CGDEM_FP64 = 0, CGDEM_MIXED = 1 } cgdem_precision;
typedef enum { CGDEM_PERIODIC_BOX = 0, CGDEM_CYLINDER = 1 } cgdem_domain_kind;
typedef enum { CGDEM_CG_NONE = 0, CGDEM_CG_SSW = 1, CGDEM_CG_SSP = 2 } cgdem_cg_scheme;

/*
 * Description of one sample, given at the FINE scale for the material:
 * the library applies the coarse-graining rules itself (gamma_g = k gamma,
 * Eq. 24; rho, E, nu, e, mu unchanged, Eq. 19, 28, 34, 35).  Radii passed to
 * cgdem_init_particles are grain radii (see cgdem_cg_scale_diameters).
 */
typedef struct {
    /* material, fine scale (Table 3) */
    double rho, E, nu, e, mu, gamma;
    /* coarse graining (Eq. 14-16): factor k >= 1 and scheme */
    double k_cg;
    int cg_scheme;          /* cgdem_cg_scheme */
    /* fluid (Table 4) */
    double rho_f, mu_f;
    int use_drag;           /* Di Felice drag Eq. 8-11 on/off */
    int use_buoyancy;       /* -rho_f V g on/off */
    /* domain: periodic cube [0,L)^3 (L[0]==L[1]==L[2] required in mixed
       precision), or a cylinder of radius Rc about the z axis, bottom plane
       z = 0 open over r < r_out (the outlet), top plane z = H */
    int kind;               /* cgdem_domain_kind */
    double L[3];
    double Rc, H, r_out;
    double g[3];
    double dt;              /* time step [s]; > 0 */
    int coulomb_mode;       /* 0: F_lim = F_ne + 2 F_C on bonds, F_ne otherwise; 1: |F_ne| */
    /* fluid grid: cell of x is floor((x - f_lo) * inv_hf) clamped per axis;
       cells numbered x fastest.  V_cell is the cell volume of Eq. 7. */
    int nf[3];
    double f_lo[3], hf[3], inv_hf[3];
    double V_cell;
    double n_min;           /* lower clamp of the porosity */
    int vf_mode;            /* 0 centroid, 1 equal-volume cube spread over cells */
    int couple_every;       /* recompute the porosity every k-th step (>= 1, equal in all samples) */
    double skin;            /* candidate-list skin [m]; > 2 |delta_C| required (2 |delta_S| with
                               jkr_mode 1) */
    double r_max;           /* largest grain radius the sample holds [m] (sizes the search grid) */
    /* fluid: 0 the superficial velocity of cgdem_set_fluid_velocity;
       1 (cylinders) two-way coupling by Darcy flow, the fluid of Eq. 6 in the
       slow-flow limit: after every porosity update the dynamic pressure p
       solves div(K(n) grad p) = 0 on the fluid grid with the Kozeny-Carman
       permeability K = perm_d^2 n^3 / (180 (1 - n)^2) (n capped at 0.95),
       p = p_inlet in the cells whose centre lies outside the cylinder wall
       and p = 0 at the outlet (the lower face of the bottom cells whose
       centre lies over it); the superficial velocity U = -(K / mu_f) grad p
       (cell centre: mean of its two face velocities per axis) replaces the
       prescribed one in the drag, every grain feels -V grad p (grad p =
       -mu_f U / K of its cell), and the drag reaction of Eq. 7 is summed per
       cell (cgdem_get_fluid) */
    int fluid_mode;
    double p_inlet;         /* injection (dynamic) pressure [Pa] */
    double perm_d;          /* grain diameter of the Kozeny-Carman permeability [m] */
    /* particle-particle contact model (cgdem_set_stage changes it later):
       0 the modified JKR (Sec. 2.3, Fig. 2): bonds only between the pairs
       that cgdem_init_particles bonds, broken at point C (Table 1) for good,
       new contacts Hertz; 1 the original JKR of the generation stage
       (Sec. 3.1, Fig. 1): a contact forms when two grains touch (point A:
       the force drops to -8/9 F_C), follows Eq. 12-13 loading and unloading,
       and separates at point S, the turning point of Eq. 13 (delta_S =
       -(3/4) (4 pi^2 gamma^2 R* / E*^2)^(1/3), F = -5/9 F_C); the pair forms
       a new contact the next time it touches */
    int jkr_mode;
} cgdem_sample_params;

/*
 * A preparation stage of a cylinder sample (Sec. 3.1: generation with the
 * original JKR, compression by the top plate to an overburden stress,
 * perforation by a penetrometer with the modified JKR).  The boundaries move
 * with the grains' drift, and their contacts are Hertz walls (Sec. 3.1) whose
 * relative velocity includes the wall's.
 */
typedef struct {
    int jkr_mode;           /* as in cgdem_sample_params */
    int plate_mode;         /* 0: the top plate holds its height; 1: after every force
                               evaluation its velocity becomes v = plate_gain (stress -
                               plate_stress), |v| <= plate_vmax, where stress is the force
                               along z the grains exert on it / (pi Rc^2) */
    double plate_H;         /* > 0: the plate's height from now on (<= the sample's H) [m] */
    double plate_stress;    /* target stress [Pa] (Sec. 3.1: 1 MPa) */
    double plate_gain;      /* [m / (s Pa)] */
    double plate_vmax;      /* [m/s] */
    int pen_mode;           /* 1: a penetrometer, a rigid cylinder of radius pen_radius on the
                               axis from its flat tip upwards, starts with its tip at
                               pen_z_start, moves down at pen_speed until the tip reaches
                               pen_z_stop, then up at the same speed until the tip is back at
                               pen_z_start, where it is removed; 2: the tool in place goes
                               back up from where it is (to pen_z_start); 0: none */
    double pen_radius, pen_speed, pen_z_start, pen_z_stop;
    double pen_force;       /* > 0: the driving force of the descent (Sec. 3.1: a constant
                               moving force): after each force evaluation the descent's speed
                               becomes pen_speed (1 - F / pen_force), clamped to [0, pen_speed],
                               F the force of the grains on the tool along z; 0: pen_speed */
    int outlet_closed;      /* 1: the bottom plane is closed over the outlet too (the stages
                               before the sand production); 0: open (grains leave through it) */
} cgdem_stage;

typedef struct {
    int precision;          /* cgdem_precision */
    int n_samples;          /* >= 1 */
    int max_neighbors;      /* candidate-list width per particle (ELL columns) */
    int block_size;         /* threads per block of the fused force kernel: 64, 128 or 256 */
    double cell_scale;      /* search cell edge = cell_scale * (2 R_max + skin), in [0.05, 1];
                               <= 0 selects 0.35 (pairs are searched from the larger sphere) */
    int steps_per_graph;    /* steps captured in one CUDA graph by cgdem_step (>= 1) */
    int closure;            /* 1: the context carries the learned closure (cgdem_set_closure);
                               its force kernel runs blocks of 128 (block_size 0 or 128) */
    int particles_per_warp; /* spheres per warp of the fused force kernel: 32 (0 selects it),
                               or 16 (twice the warps: for samples too small to fill the GPU) */
    int fluid_iters;        /* Darcy samples: conjugate-gradient iterations per solve at most
                               (0 selects 2000; each solve starts from the last pressure) */
    double fluid_tol;       /* stop when |residual| <= fluid_tol |right-hand side| (0 selects 1e-10) */
    int fluid_kernels;      /* 0: the solve's iterations in one cooperative launch (all blocks
                               resident, a grid barrier between phases, each wait bounded: a
                               wait that expires latches CGDEM_E_TIMEOUT) where the device
                               and graph capture allow it; 1: one kernel per phase of an
                               iteration, looped by a CUDA-graph WHILE node.  The two forms
                               sum in different orders, so they agree to rounding only */
} cgdem_config;

typedef struct cgdem_ctx cgdem_ctx;

/* ---------------------------------------------------------------------
 * Host-only helpers (no GPU needed).
 * ------------------------------------------------------------------- */

/* Rayleigh critical time step, Eq. 37-38, with G = E / (2 (1 + nu)). */
double cgdem_rayleigh_dt(double Rbar, double rho, double E, double nu);

/* Coarse-grained diameters from n_fine fine diameters (Sec. 2.4, Fig. 3):
 *   SSW: d_g = k d_p for the first floor(n_fine / k^3) fine particles;
 *   SSP: every grain has d_g = k (mean d_p^3)^(1/3), floor(n_fine / k^3) grains;
 *   NONE or k == 1: a copy.
 * d_out needs room for n_fine entries; *n_out receives the grain count. */
int cgdem_cg_scale_diameters(const double* d_fine, int64_t n_fine, double k, int scheme,
                             double* d_out, int64_t* n_out);

/* Device bytes needed for the given samples; counts[s] = grains of sample s. */
int cgdem_workspace_size(const cgdem_config* cfg, const cgdem_sample_params* sp,
                         const int64_t* counts, size_t* bytes);

/* ---------------------------------------------------------------------
 * Context.
 * ------------------------------------------------------------------- */

/* Create a context over a caller-owned device workspace of `bytes` bytes
 * (256-byte aligned, at least cgdem_workspace_size).  The workspace must
 * outlive the context.  sp has cfg->n_samples entries. */
int cgdem_create(const cgdem_config* cfg, const cgdem_sample_params* sp, const int64_t* counts,
                 void* workspace, size_t bytes, cgdem_ctx** out);
void cgdem_destroy(cgdem_ctx* ctx);
const char* cgdem_last_error(const cgdem_ctx* ctx);
/* Returns the latched device status (and clears nothing). Synchronises stream. */
int cgdem_status_sync(cgdem_ctx* ctx, void* stream);

/* ---------------------------------------------------------------------
 * The method (Sec. 2), one verb per step of the path.
 * ------------------------------------------------------------------- */

/* Copy the initial state from HOST arrays in id order: x, v, w [N,3] and
 * grain radii R [N] (N = sum of counts).  Forces, torques and all contact
 * history are reset to zero.  If bond_touching != 0, every pair with
 * d^2 < (Ri+Rj)^2 starts bonded (modified JKR, Sec. 2.3).  The porosity is
 * computed and the contact list built.  Synchronises stream.  The inputs are
 * checked on the device before anything uses them: CGDEM_E_INVALID names
 * the lowest particle whose radius lies outside (0, r_max] of its sample,
 * CGDEM_E_NONFINITE the lowest with a non-finite sum of its nine state
 * components (the radius test first at equal index); the context's state is
 * then left as it was. */
int cgdem_init_particles(cgdem_ctx* ctx, const double* x, const double* v, const double* w,
                         const double* R, int bond_touching, void* stream);

/* Prescribed superficial fluid velocity U_s per fluid cell (HOST array
 * [Cf,3], all samples' cells in sample order, cells x fastest).  The drag
 * (Eq. 8) uses the interstitial velocity U_s / n of the particle's cell.
 * The simple locally averaged fluid of the coupled model stands in for the
 * Navier-Stokes solve of Eq. 6.  Synchronises stream. */
int cgdem_set_fluid_velocity(cgdem_ctx* ctx, const double* Us, void* stream);

/* Re-sort particles by cell and rebuild the candidate list (pairs with
 * d < Ri + Rj + skin), carrying tangential history and bond state by id pair. */
int cgdem_build_contacts(cgdem_ctx* ctx, void* stream);

/* Bond every pair that touches now, d^2 < (Ri + Rj)^2 in IEEE double (Sec.
 * 3.1: the bonds of the modified JKR in the perforation stage, made on the
 * compressed sample); the other contacts keep their state and every contact
 * its tangential spring.  The candidate list of the current state holds
 * every touching pair, so this needs no rebuild.  Asynchronous on stream. */
int cgdem_bond_touching(cgdem_ctx* ctx, void* stream);

/* Porosity: scatter the fixed-point volume quanta round(V_i 2^40 / V_cell)
 * of every active particle into its fluid cell (Eq. 6-7 porosity n);
 * n = clamp(1 - S 2^-40, n_min, 1).  Integer atomics: bit-reproducible. */
int cgdem_couple_fluid(cgdem_ctx* ctx, void* stream);

/* Forces and torques at the current state (contacts, walls, gravity,
 * buoyancy, drag); advances the tangential history by dt and breaks bonds
 * (Eq. 1-5, 8-13, 32-35).  Uses the candidate list of the last build. */
int cgdem_compute_forces(cgdem_ctx* ctx, void* stream);

/* Velocity Verlet halves: half = 0: v += dt/2 F/m, w += dt/2 T/I, x += dt v
 * (wrapped into a periodic box); half = 1: v += dt/2 F/m, w += dt/2 T/I,
 * then particles below z < -2R in a cylinder leave through the outlet. */
int cgdem_integrate(cgdem_ctx* ctx, int half, void* stream);

/* nsteps full steps (half kick, drift, porosity every couple_every steps,
 * candidate-list rebuild when the skin may be exceeded, forces, half kick,
 * outlet), enqueued as CUDA graphs with no host round trip: the opening half
 * kick, blocks of steps_per_graph steps, blocks of the powers of two below
 * it for the remainder, and the closing step, each captured on first use
 * per stream.  Needs forces
 * consistent with the state (after init or compute_forces).  In FP64 each
 * candidate pair is evaluated once and its result passed between warps of
 * the force kernel in a fixed order; a warp's wait for another is bounded,
 * and one that runs out (never expected) latches CGDEM_E_TIMEOUT, returned
 * by the next readback or cgdem_status_sync. */
int cgdem_step(cgdem_ctx* ctx, int64_t nsteps, void* stream);

/* Self-check of the FP64 step's own reciprocal and cube root (Newton-
 * Raphson iteration from a single-precision seed, used by the FP64 contact
 * law for values that feed forces only).  x: n DEVICE doubles; out: 4 n
 * DEVICE doubles, out[4i..4i+3] = the step's 1/x, CUDA's 1.0 / x, the
 * step's cbrt(|x|), CUDA's cbrt(|x|).  Asynchronous on stream.  Errors:
 * CGDEM_E_INVALID (n < 0, or a null pointer with n > 0), CGDEM_E_CUDA. */
int cgdem_fp64_math_check(const double* x, int64_t n, double* out, void* stream);

/* Capture and upload on stream every CUDA graph that cgdem_step replays
 * there (the opening half kick, the block of steps_per_graph steps, the
 * blocks of the powers of two below it, the closing step), which cgdem_step
 * otherwise does at its first call on that stream.  Needs no particles: a
 * caller can pay the captures at creation instead of in the first step.
 * Graphs are captured again after cgdem_set_closure, cgdem_closure_record
 * and the first cgdem_set_stage, which change the kernels' variants.
 * A context without particles (N = 0) captures nothing.  Errors:
 * CGDEM_E_INVALID (null ctx), CGDEM_E_CUDA (capture or upload failed; the
 * message says which). */
int cgdem_prepare(cgdem_ctx* ctx, void* stream);

/* ---------------------------------------------------------------------
 * Readback (HOST arrays, id order).  Synchronise stream.
 * ------------------------------------------------------------------- */

/* Any pointer may be NULL.  Arrays are [N,3], owned by the caller (pinned
 * host memory makes the device-to-host copies faster).  Returns after the
 * stream has synchronised. */
int cgdem_get_state(cgdem_ctx* ctx, double* x, double* v, double* w, double* F, double* T,
                    void* stream);

/* Active particle contacts (those that applied a force at the last force
 * evaluation), as id pairs id_i < id_j sorted lexicographically, with the
 * bond flag.  *count receives the number; at most cap are written. */
int cgdem_get_contacts(cgdem_ctx* ctx, int32_t* id_i, int32_t* id_j, uint8_t* bonded,
                       int64_t cap, int64_t* count, void* stream);

/* The same active contacts, sorted the same way, with the tangential spring
 * xi of Eq. 4 of each ([count,3] doubles, SI): the spring as seen from id_i,
 * i.e. the one whose force k_t xi acts on id_i (the mixed precision keeps it
 * in FP32).  Any output pointer may be NULL; at most cap are written. */
int cgdem_get_contact_springs(cgdem_ctx* ctx, int32_t* id_i, int32_t* id_j, double* xi,
                              int64_t cap, int64_t* count, void* stream);

/* Porosity cell sums S (uint64 quanta) of all samples' fluid cells, sample
 * after sample; cap = room in cell_sums. */
int cgdem_get_voidfrac(cgdem_ctx* ctx, uint64_t* cell_sums, int64_t cap, void* stream);

/* Per sample, 8 doubles: translational KE, rotational KE, momentum x,y,z,
 * produced (outlet) mass, active particles, bonded contacts. */
int cgdem_get_diagnostics(cgdem_ctx* ctx, double* out, int64_t cap, void* stream);

/* Fluid state of the Darcy samples (fluid_mode 1), HOST arrays over all
 * samples' fluid cells (sample after sample, x fastest), any may be NULL:
 * p [Cf] dynamic pressure [Pa]; U [Cf,3] superficial velocity [m/s];
 * gradp [Cf,3] its driving gradient -mu_f U / K [Pa/m]; reaction [Cf,3] the
 * drag forces of the grains in each cell at the last force evaluation, the
 * one that ended the last cgdem_step or cgdem_compute_forces call (the steps
 * inside a call sum none: nothing reads them back, and the Darcy solve
 * does not use them) (Eq. 7: the fluid's force density is this over V_cell) in integer quanta
 * of 2^-60 N; *iters the iterations of the last solve (-1: it stopped at
 * fluid_iters short of fluid_tol).  Cells of other samples hold zeros.
 * Synchronises stream. */
int cgdem_get_fluid(cgdem_ctx* ctx, double* p, double* U, double* gradp, int64_t* reaction,
                    int64_t* iters, void* stream);

/* Start a preparation stage on cylinder sample `sample` (HOST struct): the
 * contact model, the top plate and the penetrometer take effect from the
 * next step (the boundaries move from the next drift on; a new penetrometer
 * starts without spring history).  CGDEM_E_INVALID for a periodic sample
 * with moving boundaries, a plate above the sample's H, non-positive speeds
 * or radii where a boundary moves, jkr_mode 1 with a skin below 2 |delta_S|
 * of the largest pair, or a context with the learned closure (nor may such
 * a context be created with jkr_mode 1).  The first call switches the
 * context's force kernels to the ones that run the stages (a few per cent
 * slower).  Synchronises stream. */
int cgdem_set_stage(cgdem_ctx* ctx, int sample, const cgdem_stage* stage, void* stream);

/* Per sample, 6 doubles (HOST, out[6 * n_samples]): the top plate's height
 * [m], its velocity for the next drift [m/s], the stress on it at the last
 * force evaluation [Pa], the penetrometer tip's height [m], its direction
 * (-1 down, +1 up, 0 none), and the force along z the grains exert on it at
 * the last force evaluation [N].  The forces are sums of integer quanta of
 * 2^-40 N.  Synchronises stream. */
int cgdem_get_boundaries(cgdem_ctx* ctx, double* out, int64_t cap, void* stream);

/* Produced sand by size class (Sec. 3.4, Fig. 11).  edges: nclass + 1
 * increasing fine-scale diameters [m] (HOST), 1 <= nclass <= 16, or nclass
 * = 0 to stop recording.  A grain of radius R in a sample coarse-grained at
 * ratio k stands for fine grains of diameter 2 R / k; it is counted in class
 * c when edges[c] <= 2 R / k < edges[c + 1] (below edges[0]: class 0; at or
 * above edges[nclass]: the last class).  From the call on, every grain that
 * leaves through the outlet adds 1 to its class's count and its mass
 * rho (4/3 pi) R^3 to its class's mass (integer quanta of 2^-40 of the
 * sample's largest grain mass, so the sums do not depend on the order of
 * the removals); the sums start at zero (and again at cgdem_init_particles).
 * Applies to every sample.  Synchronises stream. */
int cgdem_set_psd_classes(cgdem_ctx* ctx, const double* edges, int nclass, void* stream);

/* The cumulative produced mass [kg] and grain count per sample and class:
 * HOST arrays of cap >= 16 x n_samples entries, 16 per sample (classes past
 * nclass hold 0).  Either pointer may be NULL.  Synchronises stream. */
int cgdem_get_produced_psd(cgdem_ctx* ctx, double* mass, int64_t* count, int64_t cap, void* stream);

/* Step at which each particle left through the outlet (-1 if it did not). */
int cgdem_get_removed_step(cgdem_ctx* ctx, int32_t* removed_step, void* stream);

/* Steps completed, candidate-list rebuilds done, the largest number of
 * candidates any particle had at the last rebuild, and the total number of
 * candidate entries at the last rebuild. */
int cgdem_get_counters(cgdem_ctx* ctx, int64_t* steps, int64_t* rebuilds, int32_t* max_candidates,
                       int64_t* total_candidates, void* stream);

/* Kernel launches of cgdem_step (no synchronisation; host counters):
 * *step_kernels = kernels that cgdem_step calls on this context have
 * launched unconditionally so far (every node of the captured graphs that
 * runs on each replay); *rebuild_kernels = kernels of one candidate-list
 * rebuild sequence, which a conditional graph node runs only on the steps
 * whose rebuild falls due (0 when conditional nodes are unavailable: the
 * rebuild kernels are then captured plainly and counted in *step_kernels).
 * Kernels launched by a stretch of calls = the difference of step_kernels
 * + rebuild_kernels x the rebuilds done in it (cgdem_get_counters).  The
 * Darcy solves that conditional nodes run (fluid_mode 1) are not counted. */
int cgdem_get_launch_counts(cgdem_ctx* ctx, int64_t* step_kernels, int32_t* rebuild_kernels);

/* ---------------------------------------------------------------------
 * Pair search without device allocation.
 * ------------------------------------------------------------------- */

/* Fixed limits of the scratch memory of cgdem_touching_pairs_noalloc. */
#define CGDEM_NOALLOC_MAX_SPHERES 262144
#define CGDEM_NOALLOC_MAX_CELLS 262144

/* The paper has no counterpart of this call; it is a convenience of this
 * library.  It finds every pair i < j of spheres with
 *     d^2 < (Ri + Rj + skin)^2
 * (d^2 summed x, y, z in IEEE double, minimum image when periodic != 0) --
 * with skin = 0 exactly the touching test of the contact list -- and it
 * allocates no device memory.  It is meant for callers that cannot call
 * cudaMalloc: a host whose device memory is one pool fixed at start-up,
 * or a loop that must not stall on the device synchronisation an
 * allocation can cause.  Its working memory is a fixed array of about 5 MB
 * inside the library that each GPU using the call keeps until the process
 * exits; the first call on a device looks up that array's address (make
 * that first call before any stream capture), and every later call reuses
 * the array, so calls whose GPU work overlaps race with each other.  The
 * address is kept for the life of the process: the call assumes that the
 * device's primary context is never reset (cudaDeviceReset) in between.
 *   x [n,3], R [n]: DEVICE arrays of centres and radii (n <= 262144).
 *   box_lo, box_hi: HOST arrays of 3 doubles bounding the centres (the
 *     periodic cell when periodic != 0); the search grid has cells of edge
 *     >= 2 r_max + skin and at most 262144 of them.
 *   r_max: the largest radius; skin >= 0.
 *   pairs [cap,2]: DEVICE output, (i, j) with i < j, in no particular order.
 *   count: DEVICE unsigned long long receiving the number of pairs found
 *     (pairs beyond cap are counted but not written).
 * Returns CGDEM_E_CAPACITY (nothing enqueued) if n or the cell count exceeds
 * the limits, CGDEM_E_INVALID for bad arguments; otherwise enqueues the work
 * on stream and returns without synchronising. */
int cgdem_touching_pairs_noalloc(const double* x, const double* R, int64_t n,
                                 const double* box_lo, const double* box_hi, int periodic,
                                 double r_max, double skin, int32_t* pairs, int64_t cap,
                                 unsigned long long* count, void* stream);

/* ---------------------------------------------------------------------
 * Instrumentation.
 * ------------------------------------------------------------------- */

/* Same work as cgdem_step(ctx, nsteps, stream) but launched kernel by kernel
 * with CUDA events around the fused force/integrate kernel and around the
 * candidate-list rebuild sequence of every step.  out (6 doubles):
 * mean force-kernel time per step [ms], rebuild work [ms] (the per-step
 * rebuild-sequence times summed, less the shortest one on each step: the
 * cost of the early-returning launches, which a CUDA graph's conditional
 * node does not run), rebuilds done, total time [ms], steps timed, the
 * shortest per-step rebuild-sequence time [ms].  Synchronises stream. */
int cgdem_profile_step(cgdem_ctx* ctx, int64_t nsteps, double* out, void* stream);

/* ---------------------------------------------------------------------
 * Learned closure network (not part of the paper): a correction of the
 * coarse parcels' drag (Eq. 8) and surface energy (Eq. 13) per parcel,
 * c_d = exp(o_1) and c_g = exp(o_2), from a 5 -> 64 -> 64 -> 64 -> 2 SiLU
 * network of the inputs (local solid fraction 1 - n of Eq. 6-7, slip speed
 * |u - v| of Eq. 8-11, coarse-graining ratio k of Eq. 14, coordination
 * number, mean overlap / diameter).
 *
 * Parameters: CGDEM_MLP_NPARAMS floats, device memory, caller-owned:
 * mu[5], inv_sigma[5] (inputs are standardised as (x - mu) * inv_sigma),
 * then for each layer W[out][in] row by row and b[out].  The tensor-core
 * kernels round the inputs of every matrix product (standardised inputs,
 * hidden activations, weights, back-propagated gradients) to bfloat16 and
 * accumulate in FP32.
 * ------------------------------------------------------------------- */
#define CGDEM_MLP_NPARAMS 8844

/* Bytes of device workspace the training and inference calls need.  The
 * workspace is caller-owned and must be zero-filled before its first use. */
int cgdem_mlp_workspace_size(size_t* bytes);

/* Network outputs o[n][2] (device) of inputs X[n][5] (device, row-major).
 * Asynchronous on `stream`.  CGDEM_E_INVALID for bad arguments or
 * n > 2^28.  A device-side wait that expires is reported by
 * cgdem_mlp_status. */
int cgdem_mlp_forward(const float* theta, const float* X, int64_t n, float* out, void* workspace,
                      size_t workspace_bytes, void* stream);

/* One full-batch training step on samples X[n][5], targets Y[n][2] and a
 * 0/1 mask M[n][2] (all device, row-major) of the loss
 * L = 1/(2n) sum_b sum_k M_bk (o_bk - Y_bk)^2.  Writes the gradient
 * (CGDEM_MLP_NPARAMS floats, zero for mu and inv_sigma) to grad_out and L
 * to loss_out when they are non-NULL (device pointers).  When adam_m and
 * adam_v (device, CGDEM_MLP_NPARAMS floats each, zero before step t = 1)
 * are non-NULL, applies Adam step t (>= 1) with learning rate lr,
 * beta1 = 0.9, beta2 = 0.999, eps = 1e-8 to theta in place (mu and
 * inv_sigma unchanged).  The gradient sum over the batch is deterministic.
 * Asynchronous on `stream`. */
int cgdem_mlp_train_step(float* theta, float* adam_m, float* adam_v, int64_t t, double lr,
                         const float* X, const float* Y, const float* M, int64_t n, float* grad_out,
                         float* loss_out, void* workspace, size_t workspace_bytes, void* stream);

/* Synchronises `stream` and returns CGDEM_E_TIMEOUT (clearing the flag) if
 * a network kernel gave up a bounded wait since the last call. */
int cgdem_mlp_status(void* workspace, void* stream);

/* The closure inside the step (contexts created with cfg.closure = 1).
 * Every force evaluation of cgdem_step uses per-particle corrections
 * (c_d, c_g): the drag of Eq. 8 is multiplied by c_d,i and a bonded pair
 * uses the surface energy gamma_g sqrt(c_g,i c_g,j) in Eq. 12-13, in its
 * bond-break separation (Table 1, point C) and in F_C.  After the forces,
 * the same kernel evaluates the network on the inputs it measured in that
 * evaluation (tensor cores, one M = 128 tile per block) and stores the
 * corrections of the next evaluation: c = exp(clamp(o, -log_max, log_max)),
 * or c_d = c_g = 1 for a particle with an input outside [lo, hi] (plain
 * coarse-graining).  The compute_forces verb uses the corrections and
 * leaves them unchanged.  Corrections start at 1. */
typedef struct {
    float lo[5], hi[5];     /* range of the inputs the network was trained on */
    float cd_log_max;       /* |ln c_d| <= cd_log_max, in [0, 20] */
    float cg_log_max;       /* |ln c_g| <= cg_log_max, in [0, 20] */
} cgdem_closure_params;

/* Enable (theta: device pointer to CGDEM_MLP_NPARAMS floats, copied into
 * the context's BF16 form before the call returns on `stream`; cp: host) or
 * disable (enable = 0; theta and cp may be NULL) the closure; resets every
 * correction to 1.  CGDEM_E_INVALID if the skin does not exceed twice the
 * bond-break separation at the largest surface-energy correction;
 * CGDEM_E_STATE for a context without closure support. */
int cgdem_set_closure(cgdem_ctx* ctx, const float* theta, const cgdem_closure_params* cp, int enable,
                      void* stream);

/* While enabled, every force evaluation records per particle 12 floats:
 * the 5 closure inputs (solid fraction 1 - n, slip speed, k, active
 * contacts, mean overlap / diameter), the drag force as applied (3), half
 * the summed F_C of its bonded contacts, its fluid cell within its sample,
 * and the corrections c_d, c_g it used.  Inactive particles record zeros. */
int cgdem_closure_record(cgdem_ctx* ctx, int enable, void* stream);

/* Copies the rows recorded by the last force evaluation, in particle order
 * (out: host, rows >= particle count). */
int cgdem_get_closure_data(cgdem_ctx* ctx, float* out, int64_t rows, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* CGDEM_H */
