/*
 * cgdem_oracle.h -- FP64 CPU oracle for the coarse-grained CFD-DEM step of
 * Kazidenov, Khamitov & Amanbek, "Coarse-graining of CFD-DEM for simulation
 * of sand production in the modified cohesive contact model" (arXiv
 * 2211.06142).
 *
 * TEST INFRASTRUCTURE ONLY.  This library is a plain, slow restatement of
 * the paper's equations.  Its pair evaluations and per-particle loops may run
 * on several host threads (OpenMP, ora_set_threads) without changing a bit
 * of any result: each pair's evaluation is independent, and every sum is
 * taken in the same order as with one thread.  It exists so that tests and the
 * benchmark's CPU baseline can check the CUDA library against something
 * written independently from the paper.  It shares no code, header, table or
 * constant generator with the CUDA path and must never be linked into it.
 *
 * Units are SI.  Every function returns 0 on success and a negative value on
 * a bad argument.
 */
#ifndef CGDEM_ORACLE_H
#define CGDEM_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Problem description for ONE sample, at grain level (after coarse-graining). */
typedef struct {
    /* material (Table 3; E*, G*, beta derived inside) */
    double rho, E, nu, e, mu, gamma;
    /* fluid (Table 4) */
    double rho_f, mu_f;
    int use_drag;       /* 1: Di Felice drag, Eq. 8-11 */
    int use_buoyancy;   /* 1: Archimedes force -rho_f V g */
    /* domain: 0 periodic box [0,L0)x[0,L1)x[0,L2); 1 cylinder axis z through
       the origin, radius Rc, bottom plane z=0 open for r<r_out, top z=H */
    int kind;
    double L[3];
    double Rc, H, r_out;
    double g[3];
    double dt;
    int coulomb_mode;   /* 0: F_lim = F_ne + 2 F_C if bonded else F_ne; 1: |F_ne| */
    /* fluid grid: cell of x is floor((x - f_lo) * inv_hf) clamped to [0,nf-1] */
    int nf[3];
    double f_lo[3], hf[3], inv_hf[3];
    double V_cell;      /* cell volume used for the void-fraction quanta */
    double n_min;       /* lower clamp of the porosity */
    int vf_mode;        /* 0 centroid, 1 equal-volume cube overlap */
    int couple_every;   /* recompute the void fraction every k-th step */
    /* fluid: 0 the superficial velocity given at creation; 1 (cylinder only)
       Darcy flow from the porosity, solved at every coupling step: dynamic
       pressure p_inlet outside the cylinder wall, 0 at the outlet */
    int fluid_mode;
    double p_inlet;     /* [Pa] */
    double perm_d;      /* grain diameter of the Kozeny-Carman permeability [m] */
    double n_cap;       /* porosity cap of the permeability (n -> 1 has none) */
    /* particle-particle contact model: 0 the modified JKR (Fig. 2): bonds
       only between the pairs that touch when ora_bond_touching is called,
       broken at point C for good, new contacts Hertz; 1 the original JKR
       (Fig. 1): a contact forms when two particles touch (point A: F jumps
       to -8/9 F_C), follows Eq. 12-13 loading and unloading, and separates
       at point S (delta_S, F = -5/9 F_C); the pair forms a new contact the
       next time it touches */
    int jkr_mode;
} ora_params;

/* The moving boundaries and contact model of a preparation stage (Sec. 3.1:
 * generation with the original JKR, compression by the top plate to an
 * overburden stress, perforation by a penetrometer with the modified JKR).
 * Cylinder samples only. */
typedef struct {
    int jkr_mode;         /* as in ora_params */
    int plate_mode;       /* 0: the top plate holds its height; 1: it moves at
                             v = gain (stress - plate_stress), |v| <= plate_vmax,
                             stress = its force along z / (pi Rc^2) at the last
                             force evaluation */
    double plate_H;       /* > 0: the plate's height from now on [m] */
    double plate_stress;  /* target stress [Pa] */
    double plate_gain;    /* [m / (s Pa)] */
    double plate_vmax;    /* [m/s] */
    int pen_mode;         /* 1: a penetrometer (a rigid cylinder of radius
                             pen_radius on the axis ending below in a hemisphere
                             of the same radius, its tip the lowest point)
                             starts with its tip at pen_z_start, moves down at
                             pen_speed until the tip reaches pen_z_stop, then up
                             at the same speed until the tip is back at
                             pen_z_start, where it is removed; 2: the tool in
                             place goes back up from where it is (to pen_z_start);
                             0: none */
    double pen_radius, pen_speed, pen_z_start, pen_z_stop;
    double pen_force;     /* > 0: the driving force of the descent (Sec. 3.1: a
                             constant moving force): after each force evaluation
                             the descent's speed becomes pen_speed (1 - F / pen_force),
                             clamped to [0, pen_speed], F the force of the grains
                             on the tool along z; 0: always pen_speed */
    int outlet_closed;    /* 1: the bottom plane is closed over the outlet too
                             (the stages before the sand production) */
} ora_stage;

/* ---- closed forms and single-contact laws (pins and unit tests) ---- */
/* E* for one material (Eq. 12 definitions with E1=E2, nu1=nu2). */
double ora_estar(double E, double nu);
/* beta from the restitution coefficient (Eq. 33, squared log restored). */
double ora_beta(double e);
/* contact radius a on the stable branch a >= a_C solving Eq. 13 by bisection. */
double ora_jkr_contact_radius(double delta, double Rs, double Es, double gamma);
/* Eq. 12 */
double ora_jkr_force(double a, double Rs, double Es, double gamma);
/* Eq. 13 */
double ora_jkr_overlap(double a, double Rs, double Es, double gamma);
/* Table 1 point C overlap, delta_C (negative). */
double ora_delta_c(double Rs, double Es, double gamma);
/* modified-JKR break test: 1 when delta < delta_C (evaluated as documented). */
int ora_bond_breaks(double delta, double Rs, double Es, double gamma);
/* Point S of the original JKR curve (Fig. 1): the turning point of Eq. 13,
 * d delta / d a = 0, where a displacement-driven contact separates. */
double ora_delta_s(double Rs, double Es, double gamma);
/* original-JKR separation test: 1 when delta < delta_S (evaluated as documented). */
int ora_contact_separates(double delta, double Rs, double Es, double gamma);
/* contact radius on the branch a >= a_S solving Eq. 13 by bisection. */
double ora_jkr_contact_radius_s(double delta, double Rs, double Es, double gamma);
/* Rayleigh time step Eq. 37-38 with G = E/(2(1+nu)). */
double ora_rayleigh_dt(double Rbar, double rho, double E, double nu);

/* One particle-particle contact evaluated in isolation.
 * xi_inout: tangential spring (force-on-i convention), updated in place.
 * bonded_inout: bond state, cleared on break.
 * out: F_i[3], T_i[3], T_j[3], then Fn_elastic, a, delta (12 doubles).
 * Returns 1 if the contact is active (force applied), 0 if not. */
int ora_pair_contact(const ora_params* p,
                     const double xi_pos[3], const double vi[3], const double wi[3], double Ri, double mi,
                     const double xj_pos[3], const double vj[3], const double wj[3], double Rj, double mj,
                     double xi_inout[3], int* bonded_inout, double out[12]);

/* Di Felice drag on one particle, Eq. 8-11.  u = interstitial fluid velocity. */
void ora_drag(double rho_f, double mu_f, double d, const double u[3], const double v[3],
              double n, double f_out[3]);

/* ---- whole-sample simulation ---- */
typedef struct ora_sim ora_sim;

ora_sim* ora_create(const ora_params* p, int64_t n,
                    const double* x, const double* v, const double* w,
                    const double* R, const double* Us /* [nf0*nf1*nf2*3] superficial velocity */);
void ora_destroy(ora_sim* s);
/* Bond every touching pair, d^2 < (Ri + Rj)^2 (Sec. 3.1: the bonds of the
 * perforation stage); the other records keep their state and every record
 * its spring. */
int ora_bond_touching(ora_sim* s);
/* Cell sums of the void-fraction quanta at the current positions. */
int ora_couple_fluid(ora_sim* s);
/* Forces and torques at the current state; advances tangential history by dt. */
int ora_compute_forces(ora_sim* s);
/* nsteps of velocity Verlet (half kick, drift, contacts, fluid, forces, half kick, outlet). */
int ora_step(ora_sim* s, int64_t nsteps);
int ora_get_state(const ora_sim* s, double* x, double* v, double* w, double* F, double* T);
/* Overlap R - distance between a particle (centre x, radius R) and the
 * penetrometer (a cylinder of radius rp on the axis ending in a hemisphere
 * whose lowest point is at height zt), and the unit vector n from the centre
 * towards the tool's nearest point. */
double ora_tool_overlap(const double x[3], double R, double rp, double zt, double n[3]);
/* Start a preparation stage (the boundaries move from the next drift on). */
int ora_set_stage(ora_sim* s, const ora_stage* st);
/* out[6]: top-plate height, its velocity for the next drift, the stress on
 * it at the last force evaluation, the penetrometer tip's height, its
 * direction (-1 down, +1 up, 0 none), and the force along z that the
 * particles exert on it at the last force evaluation. */
int ora_get_boundaries(const ora_sim* s, double out[6]);
int ora_set_forces(ora_sim* s, const double* F, const double* T);
int64_t ora_num_contacts(const ora_sim* s);
/* Active particle contacts sorted by (id_i < id_j). xi has 3 entries per contact. */
int ora_get_contacts(const ora_sim* s, int32_t* id_i, int32_t* id_j, uint8_t* bonded,
                     double* xi, int64_t cap);
int ora_get_voidfrac(const ora_sim* s, uint64_t* cell_sums);
/* Per particle, two scales of the last force evaluation: the sum of the
 * magnitudes of every separate force term (Eq. 12 repulsion and adhesion,
 * Eq. 32 damping, tangential force, gravity, buoyancy, drag), and the sum of
 * the magnitudes of its contact, wall and body force vectors. */
int ora_get_force_scale(const ora_sim* s, double* scale);
int ora_get_force_scale_net(const ora_sim* s, double* scale);
/* Darcy flow on a Cartesian grid of nx x ny x nz cells (x fastest) with
 * spacing h: K permeability per cell [m^2]; type 0 unknown, 1 pressure fixed
 * at p[c], 2 no cell (no flux); outlet[c] != 0 joins a cell's lower z face to
 * the pressure p_out half a cell below.  Between neighbouring cells the face
 * conductance is A / (mu h) times the harmonic mean of their K; the outlet's
 * is A_z K / (mu h_z / 2).  Solves the unknown pressures (p holds the first
 * guess) by conjugate gradients with the diagonal as preconditioner until the
 * residual is below tol times the right-hand side.  Returns the iterations,
 * or -1 if max_iter did not reach tol. */
int ora_darcy_solve(int nx, int ny, int nz, const double h[3], double mu, const double* K,
                    const int8_t* type, const uint8_t* outlet, double p_out, double* p,
                    double tol, int max_iter);
/* Superficial velocity at cell centres from the solved pressures: per axis
 * the mean of the face velocities -(K_f / mu) dp / h of the cell's two faces
 * (0 through a domain edge or a cell of type 2); U[3 * c + k].  Cells of
 * type 1 and 2 get 0. */
int ora_darcy_velocity(int nx, int ny, int nz, const double h[3], double mu, const double* K,
                       const int8_t* type, const uint8_t* outlet, double p_out, const double* p,
                       double* U);
/* The sample's fluid state (fluid_mode 1): pressure [Cf], superficial
 * velocity [Cf,3], dynamic pressure gradient [Cf,3] = -mu U / K, the
 * iterations of the last solve; the drag reaction of Eq. 7 per cell [Cf,3]
 * as sums of the particles' drag forces in quanta of 2^-60 N (the cell's
 * force density is that sum over V_cell). */
int ora_get_fluid(const ora_sim* s, double* p, double* U, double* gradp, int64_t* iters);
int ora_get_reaction(const ora_sim* s, int64_t* sums);

/* Host threads for the following calls (<= 0 keeps the current number);
 * returns the number in use (1 without OpenMP). */
int ora_set_threads(int nthreads);
/* KE_trans, KE_rot, Px, Py, Pz, produced mass, n_active, n_bonds */
int ora_get_diagnostics(const ora_sim* s, double out[8]);
int ora_get_removed_step(const ora_sim* s, int64_t* removed_step);

/* Learned-closure hooks (the closure is not part of the paper).  With the
 * closure enabled, the drag of particle i (Eq. 8) is multiplied by c_d,i and
 * each pair uses the surface energy gamma sqrt(c_g,i c_g,j) in Eq. 12-13 and
 * in F_C = 3 pi gamma R* (Table 1).  Corrections start at 1. */
#define ORA_CL_COLS 12
int ora_set_closure(ora_sim* s, int enable, double k_feat);
int ora_set_corrections(ora_sim* s, const double* cd, const double* cg);
/* Per particle, from the last force evaluation (ORA_CL_COLS doubles each):
 * 0 solid fraction 1 - n of its fluid cell (Eq. 6-7), 1 slip speed
 * |U_s / n - v| (Eq. 8-11), 2 the feature k given to ora_set_closure,
 * 3 active pair contacts, 4 mean overlap of those contacts / (2 R),
 * 5-7 drag force as applied, 8 half the summed F_C of its bonded contacts,
 * 9 fluid cell, 10-11 the corrections c_d, c_g used. */
int ora_get_closure_data(const ora_sim* s, double* out);
/* Brute force O(N^2) list of pairs with d^2 < (Ri+Rj+skin)^2 (minimum image). */
int64_t ora_pairs_bruteforce(const ora_params* p, int64_t n, const double* x, const double* R,
                             double skin, int32_t* pi, int32_t* pj, int64_t cap);
/* Void-fraction quanta of one sample at given positions (no simulation). */
int ora_voidfrac(const ora_params* p, int64_t n, const double* x, const double* R,
                 uint64_t* cell_sums);

#ifdef __cplusplus
}
#endif
#endif
