// cgdem_internal.cuh -- device-side data layout and helpers of the GB300
// CFD-DEM step (arXiv 2211.06142).  Internal to the library.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "cgdem.h"

namespace cgdem {

// ---------------------------------------------------------------------------
// contact record flags (bits of the first word of a record)
// ---------------------------------------------------------------------------
constexpr uint32_t REC_BOND = 0x80000000u;    // bonded pair (modified JKR, Sec. 2.3)
constexpr uint32_t REC_ACTIVE = 0x40000000u;  // applied a force at the last evaluation
constexpr uint32_t REC_IDX = 0x3fffffffu;     // partner index (current order)

// largest candidate list per particle (max_neighbors)
#define CGDEM_MAX_NEIGHBORS 96
// size classes of the produced-sand accumulators (per sample)
#define CGDEM_PSD_MAX 16

// latched device status bits
constexpr unsigned ST_CAPACITY = 1u;
constexpr unsigned ST_BOND_LOST = 2u;
constexpr unsigned ST_NONFINITE = 4u;
constexpr unsigned ST_TIMEOUT = 8u;  // a bounded device-side wait expired
// wall spring histories per sphere: cylinder side, bottom, top plate, penetrometer
constexpr int CGDEM_WALLS = 4;

// FP64 record: partner/flags + tangential spring (32 bytes)
struct __align__(16) RecD {
  uint32_t pf, pad;
  double x, y, z;
};
// mixed record: partner/flags + tangential spring in FP32 (16 bytes)
struct __align__(16) RecF {
  uint32_t pf;
  float x, y, z;
};

// Per-sample constants, derived on the host (grain level).
struct SampleDev {
  // material (Table 3 after Eq. 24 scaling) and derived moduli
  double Es, Gs, beta, mu, gamma, rho;
  double dt, half_dt;
  double g[3];
  double rho_f, mu_f;
  int use_drag, use_buoyancy, kind, coulomb_mode;
  double L[3], Rc, H, r_out;
  // fixed-point shadow: q = round(x / dq) (low 32 bits)
  double inv_dq, dq;
  int q_exp;  // dq = 2^q_exp (cylinders); 0x7fffffff when dq is not a power of two
  int32_t skin_q;
  // search grid
  double c_lo[3], c_inv_h[3];
  int nc[3];
  int cell_off;
  // fluid grid
  int nf[3];
  int fcell_off;
  double f_lo[3], inv_hf[3];
  double inv_q, n_min;
  int vf_mode, couple_every;
  double hf[3];
  double skin, rebuild_disp;  // rebuild when 2 * displacement bound > rebuild_disp
  int64_t first, count;
  // FP32 copies
  float Es_f, Gs_f, beta_f, mu_f32, gamma_f, dt_f, dq_f, rho_f32, muf_f32, n_min_f;
  float g_f[3];
  float rho_s_f;  // particle density
  float f_lo_f[3], inv_hf_f[3];
  float L_f[3], Rc_f, H_f, r_out_f;
  float rebuild_q2;  // rebuild when (max displacement in fixed units)^2 exceeds this
  float c_inv_h_f[3], skin_f;
  float k_feat_f;  // coarse-graining ratio k as a closure input
  // Eq. 32 and its tangential twin with the contact radius and reduced mass
  // factored out: gamma_n = cdbn sqrt(a m*), gamma_t = cdbt sqrt(a m*)
  float cdbn_f, cdbt_f;  // 2 sqrt(5/6) beta sqrt(2 E*), 2 sqrt(5/6) beta sqrt(8 G*)
  double cdbn, cdbt;     // the same in FP64
  double inv_Es;         // 1 / E*
  // produced sand by size class (Sec. 3.4): a grain of radius R stands for
  // fine grains of diameter 2 R / k; class c holds psd_edge[c] <= 2 R / k <
  // psd_edge[c + 1] (the first and last classes also take what lies below or
  // above); masses are summed in quanta of psd_mq (0 classes: not recorded)
  // Darcy flow (fluid_mode 1): K = perm_d2 n^3 / (1 - n)^2 with perm_d2 =
  // perm_d^2 / 180 and n <= DARCY_N_CAP
  int fluid_mode;
  double p_inlet, perm_d2;
  double k_cg;
  int n_psd;
  double psd_edge[CGDEM_PSD_MAX + 1];
  double psd_mq;
  int jkr_mode;  // 0 modified JKR, 1 original JKR (cgdem_sample_params)
  double r_max;  // largest radius the sample admits
};

// A preparation stage's moving boundaries of one sample (cgdem_set_stage),
// and their state: the top plate's height and velocity, the penetrometer's
// tip height and direction; the forces along z the grains exert on each,
// summed in integer quanta of 2^-40 N over the running evaluation and kept
// from the last one.
struct StageDev {
  int plate_mode;
  int pen_dir;  // -1 down, +1 up, 0 no penetrometer
  int outlet_closed;
  double plate_stress, plate_gain, plate_vmax;
  double pen_radius, pen_speed, pen_z_start, pen_z_stop, pen_force;
  double H, v_plate, pen_z, v_pen;
  unsigned long long plate_q, pen_q;  // running sums (two's complement)
  long long plate_q_last, pen_q_last;
};

// Learned closure (not part of the paper): per-particle corrections
// (c_d, c_g) of drag and surface energy from a 5-64-64-64-2 SiLU network
// evaluated on the tensor cores in the epilogue of each step's force kernel.
// The network's BF16 weight tiles and FP32 constants form one blob that each
// block copies into shared memory with a bulk copy.
constexpr int CL_COLS = 12;               // recorded floats per particle
constexpr uint32_t CL_TILES = 20480;      // W1 [64x16] | W2 [64x64] | W3 [64x64] | W4 [16x64]
constexpr uint32_t CL_P_B1 = 0, CL_P_B2 = 64, CL_P_B3 = 128, CL_P_B4 = 192, CL_P_MU = 196,
                   CL_P_ISG = 204, CL_P_LO = 212, CL_P_HI = 220, CL_P_CMAX = 228;  // floats after the tiles
constexpr uint32_t CL_BLOB = CL_TILES + 232 * 4;  // 21408 bytes
constexpr uint32_t CL_SM_A0 = 22528;        // x_hat tile [128 x 16]
constexpr uint32_t CL_SM_AH = 26624;        // hidden tile [128 x 64]
constexpr uint32_t CL_SMEM = 43008 + 1024;  // dynamic shared memory of the force kernel (+ alignment)

// Device control block (one per context).
struct Ctl {
  int cur;           // buffer of the dynamic state (pos/vel/omg and shadows); flips every step
  int pcur;          // buffer of per-particle data permuted only at rebuilds (id, sample, ...)
  int rec_cur;       // contact-record buffer holding the current list
  int vf_cur;        // porosity buffer read by the next force evaluation
  int rebuild;       // 1: rebuild the candidate list before the next force evaluation
  long long step;    // completed steps
  long long rebuilds;
  unsigned status;   // latched error bits
  unsigned block_counter;
  int blk_next;      // next block of the running force launch (blocks take segments in start order)
  uint32_t epoch;    // force launches completed (segment flags of the running launch reach epoch + 1)
  int max_cand;
  unsigned coupled;
  long long cand_total;  // candidate entries summed over particles at the last rebuild
  int max_cand_next;     // accumulated by the running rebuild
  long long cand_total_next;  // set when the running step scattered porosity quanta
  int closure;            // 1: corrections applied and the network evaluated every step
  int record;             // 1: every force evaluation records per-particle closure data
  // first bonded pair found missing from a rebuilt list: ids, and its squared
  // distance and squared reach (fixed-point units) at the rebuild
  int lost_i, lost_j;
  unsigned long long lost_d2, lost_S2;
  // Darcy solve: a porosity update not yet followed by a solve; the
  // conjugate-gradient scalars of the running solve
  int fl_pending, fl_done, fl_it;
  long long fl_iters;  // iterations of the last solve (-1: stopped short of the tolerance)
  double fl_rz, fl_alpha, fl_beta, fl_bb;
  // grid barrier of the one-launch solve: arrivals, generation, and a flag a
  // block sets when its wait gave up (the others then stop waiting too)
  unsigned fl_bar_count, fl_bar_gen;
  int fl_abort;
  // input check of cgdem_init_particles: the lowest index of a particle with
  // a radius outside (0, r_max] and of one with a non-finite state
  long long init_bad_r, init_bad_f;
};
constexpr double DARCY_N_CAP = 0.95;  // the permeability's porosity cap

// All device pointers of a context (passed by value to kernels).
struct Dev {
  // particle state, double-buffered: (x,y,z,R), (vx,vy,vz,1/m), (wx,wy,wz,1/I)
  double4* pos[2];
  double4* vel[2];
  double4* omg[2];
  // mixed-precision shadows: fixed-point position + radius, FP32 v|R, w|m
  int4* posq[2];
  float4* velf[2];
  float4* omgf[2];
  double4* F;  // force (w unused)
  double4* T;  // torque
  int* id[2];
  int* sample[2];
  int* fcell[2];                  // fluid cell (global index) of the current position
  unsigned long long* vq[2];      // volume quantum round(V 2^40 / V_cell)
  double4* wallh[2];              // wall spring history [CGDEM_WALLS][Npad] (FP64 mode)
  float4* wallhf[2];              // wall spring history [CGDEM_WALLS][Npad] (mixed)
  // Candidate lists.  Mixed: every sphere lists all its candidates (a pair
  // is evaluated from both sides).  FP64: a pair is listed once, by its
  // lower-index sphere (the owner); the partner receives the result in its
  // inbox.
  void* rec[2];                   // contact records, one segment of ppw*cap per warp of the force kernel
  uint32_t* cnt[2];               // records of a particle
  uint32_t* roff[2];              // index of a particle's first record; entry k at roff + k * rstride
  // Mixed: the force kernel's lanes take the spheres in the order sched
  // gives (per tile of 1024 spheres in cell order, by decreasing candidate
  // count); the records of a warp are entry-major (rstride = ppw)
  uint32_t* sched;                // [Npad] slot -> sphere (UINT_MAX: no sphere)
  int rstride;                    // 1 (FP64: a sphere's records are consecutive) or ppw (mixed)
  uint32_t* inc;                  // FP64, rebuild scratch [cap][Npad]: lower-index partners
  uint32_t* inc_n;                // FP64: pairs a particle's lower-index partners own
  uint32_t* rslot;                // FP64, per record: slot k of the pair in the partner's inbox
  double4* inbox;                 // FP64 [cap][Npad] x 2: force on the owner and n x F_t of a pair
  float4* inbox_cl;               // FP64 [cap][Npad]: closure data of a pair (contact, overlap, bond capacity)
  uint32_t* seg_flag;             // FP64, per warp segment: launch epoch once its pairs are evaluated
  uint32_t* seg_wait;             // FP64, per warp segment: lowest segment owning a pair of its spheres
  int4* posq_ref;                 // fixed-point positions at the last rebuild
  uint32_t* cand_tmp;             // rebuild scratch: candidate partners [cap][Npad]
  uint32_t* cand_n;               // rebuild scratch: candidates found per particle
  uint32_t* big_list;             // rebuild scratch: spheres whose stencil a warp walks
  uint32_t* big_n;
  uint32_t* tile_sums;            // rebuild scratch: cell-scan tile sums
  unsigned* dmax2;                // per-sample max squared displacement since rebuild (float bits, fixed units)
  // rebuild scratch
  uint32_t* cell_count;           // [C+1]
  uint32_t* cell_start;           // [C+2]
  uint32_t* pcell;                // [N]
  uint32_t* pslot;                // [N]
  uint32_t* perm_tmp;             // [N]
  uint32_t* perm;                 // new -> old
  uint32_t* inv_perm;             // old -> new
  // fluid
  unsigned long long* vf[3];      // porosity cell sums, rotating
  double4* Us;                    // superficial velocity per fluid cell
  float4* Usf;
  int* removed_step;              // by id
  double* disp;                   // per-sample displacement bound since last rebuild
  unsigned long long* vmax2;      // per-sample max (|v| dt)^2 of the last drift (double bits)
  double* diag;                   // per-sample diagnostics [S][8]
  // Darcy flow, per fluid cell (allocated when a sample has fluid_mode 1)
  int* fl_sample;                 // the cell's sample
  signed char* fl_type;           // 0 unknown, 1 fixed pressure, 2 not solved, 3 unknown draining to the outlet
  double* fl_K;                   // permeability
  double* fl_p;                   // dynamic pressure (kept: the next solve starts from it)
  double *fl_r, *fl_z, *fl_d, *fl_q, *fl_M, *fl_b;  // conjugate-gradient vectors, diagonal, right-hand side
  StageDev* stage;                // per sample: moving boundaries of the preparation stages
  int prep;                       // 1: the force kernels that run the preparation stages
  double* fl_d2;                  // the one-launch solve's second direction buffer
  double4* fl_T;                  // its face conductances per cell: upper x, y, z faces, outlet face
  double* fl_part;                // per-block partial sums [4][fl_blocks]
  int fl_blocks;
  int fl_coop_blocks;             // blocks of the one-launch solve (0: the WHILE-node form)
  double4* gradp;                 // grad p per cell (w unused)
  float4* gradpf;
  unsigned long long* react[2];   // drag reaction [Cf][3], quanta of 2^-60 N; by parity of the evaluation
  int any_fluid;
  int fl_iters_max;
  double fl_tol;
  unsigned long long* psd_count;  // produced grains per sample and size class [S][CGDEM_PSD_MAX]
  unsigned long long* psd_mass;   // their mass in quanta of the sample's psd_mq [S][CGDEM_PSD_MAX]
  double* staging;                // [N * 16] host-transfer staging
  uint32_t* contact_out;          // [2 * cap_out] (i, j | bond << 31)
  unsigned long long* contact_n;
  // learned closure (allocated when the context supports it)
  float2* clc[2];                 // (c_d, c_g) per particle, double-buffered like the state
  float* clrec;                   // [Npad][CL_COLS] data recorded by the last evaluation
  uint8_t* clblob;                // network blob (CL_BLOB bytes)
  int cl_smem;                    // 1: force launches carry the network's shared memory (closure on)
  int cl_rec;                     // 1: closure data recorded (host mirror of Ctl::record)
  SampleDev* sp;
  Ctl* ctl;
  int N, Npad, cap, n_samples, C_total, Cf_total;
  int ppw;  // spheres per warp of the force kernel (32 or 16); a record segment holds ppw spheres
  int mixed;
};

// ---------------------------------------------------------------------------
// small math helpers
// ---------------------------------------------------------------------------
template <typename T>
struct V3 {
  T x, y, z;
};
template <typename T>
__device__ __forceinline__ V3<T> v3(T a, T b, T c) {
  return V3<T>{a, b, c};
}
template <typename T>
__device__ __forceinline__ T dot3(V3<T> a, V3<T> b) {
  return a.x * b.x + a.y * b.y + a.z * b.z;
}
template <typename T>
__device__ __forceinline__ V3<T> cross3(V3<T> a, V3<T> b) {
  return v3<T>(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x);
}

__device__ __forceinline__ float sqrtT(float a) { return sqrtf(a); }
__device__ __forceinline__ double sqrtT(double a) { return sqrt(a); }
__device__ __forceinline__ float cbrtT(float a) { return cbrtf(a); }
__device__ __forceinline__ double cbrtT(double a) { return cbrt(a); }
__device__ __forceinline__ float expT(float a) { return expf(a); }
__device__ __forceinline__ double expT(double a) { return exp(a); }
__device__ __forceinline__ float log10T(float a) { return log10f(a); }
__device__ __forceinline__ double log10T(double a) { return log10(a); }
__device__ __forceinline__ float powT(float a, float b) { return powf(a, b); }
__device__ __forceinline__ double powT(double a, double b) { return pow(a, b); }

// Minimum image in IEEE double without contraction (same rounding as the
// plain definition d > L/2 ? d - L : d < -L/2 ? d + L : d).
__device__ __forceinline__ double min_image(double d, double L) {
  double h = 0.5 * L;
  if (d > h) return __dsub_rn(d, L);
  if (d < -h) return __dadd_rn(d, L);
  return d;
}

// Fluid cell of a position: floor((x - lo) * inv_h) clamped, per axis.
__device__ __forceinline__ int fluid_cell_of(const SampleDev& s, double x, double y, double z) {
  double p[3] = {x, y, z};
  int c[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    double t = floor(__dmul_rn(__dsub_rn(p[k], s.f_lo[k]), s.inv_hf[k]));
    const double hi = (double)(s.nf[k] - 1);
    if (!(t >= 0.0)) t = 0.0;  // also catches NaN: a diverged state must not index out of range
    if (!(t <= hi)) t = hi;
    c[k] = (int)t;
  }
  return s.fcell_off + (c[2] * s.nf[1] + c[1]) * s.nf[0] + c[0];
}

// Volume quantum of a sphere: round(((4/3 pi) R) R R * inv_q), left to right.
__device__ __forceinline__ unsigned long long volume_quantum(double R, double inv_q) {
  const double c = 4.1887902047863905;  // fl(fl(4/3) * fl(pi))
  double V = __dmul_rn(__dmul_rn(__dmul_rn(c, R), R), R);
  return (unsigned long long)__double2ll_rn(__dmul_rn(V, inv_q));
}

// Fixed-point shadow of a position (low 32 bits of round(x / dq)).
__device__ __forceinline__ int32_t to_q(double x, double inv_dq) {
  long long t = __double2ll_rn(x * inv_dq);
  return (int32_t)(uint32_t)(unsigned long long)t;
}

// to_q for dq = 2^e by integer operations on the IEEE representation:
// round to nearest, ties to even, low 32 bits -- the value to_q gives -- with
// no FP64 instruction (GB300 issues two FP64 operations per SM per clock).
__device__ __forceinline__ int32_t to_q_pow2(double x, int e) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const int ex = (int)((b >> 52) & 0x7ffu);
  if (ex == 0) return 0;  // zero or subnormal
  const unsigned long long m = (b & 0xfffffffffffffull) | (1ull << 52);  // x = m 2^(ex - 1075)
  const int sh = ex - 1075 - e;
  unsigned long long q;
  if (sh >= 0) {
    q = sh < 64 ? (m << sh) : 0ull;  // exact; only the low bits are kept
  } else if (-sh > 54) {
    q = 0ull;
  } else {
    const int r = -sh;
    const unsigned long long half = 1ull << (r - 1);
    const unsigned long long rem = m & ((1ull << r) - 1ull);
    q = m >> r;
    if (rem > half || (rem == half && (q & 1ull))) q += 1ull;
  }
  if (b >> 63) q = 0ull - q;
  return (int32_t)(uint32_t)q;
}

// Search-grid cell of a position (global index).
__device__ __forceinline__ int search_cell_of(const SampleDev& s, double x, double y, double z,
                                              int* cxyz) {
  double p[3] = {x, y, z};
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    double t = floor((p[k] - s.c_lo[k]) * s.c_inv_h[k]);
    const double hi = (double)(s.nc[k] - 1);
    if (!(t >= 0.0)) t = 0.0;  // also catches NaN
    if (!(t <= hi)) t = hi;
    cxyz[k] = (int)t;
  }
  return s.cell_off + (cxyz[2] * s.nc[1] + cxyz[1]) * s.nc[0] + cxyz[0];
}

// Modified-JKR break test in IEEE double: delta < delta_C, evaluated as
// delta^3 Es^2 < C_C^3 pi^2 gamma^2 Rs (cubing keeps the order; Table 1 C).
__device__ __forceinline__ bool bond_breaks_exact(double delta, double Rs, double Es,
                                                  double gamma) {
  const double KC = -1.8505508252042548;  // ((81/16)^(1/3) - 12^(1/3))^3 pi^2
  if (!(delta < 0.0)) return false;
  double lhs = __dmul_rn(__dmul_rn(__dmul_rn(delta, delta), delta), __dmul_rn(Es, Es));
  double rhs = __dmul_rn(__dmul_rn(KC, __dmul_rn(gamma, gamma)), Rs);
  return lhs < rhs;
}

// The moving boundaries follow the grains' drift at the velocities of the
// last force evaluation: the penetrometer turns back at pen_z_stop and is
// removed back at pen_z_start.
__device__ __forceinline__ void drift_boundaries(StageDev& W, double dt) {
  if (W.plate_mode == 1) W.H = __dadd_rn(W.H, __dmul_rn(dt, W.v_plate));
  if (W.pen_dir != 0) {
    W.pen_z = __dadd_rn(W.pen_z, __dmul_rn(dt, W.v_pen));
    if (W.pen_dir < 0 && W.pen_z <= W.pen_z_stop) W.pen_dir = 1;
    else if (W.pen_dir > 0 && W.pen_z >= W.pen_z_start) W.pen_dir = 0;
  }
}

// After a force evaluation: the sums of the forces on the plate and the
// penetrometer become the evaluation's (the running sums restart at zero),
// and the penetrometer and a stress-controlled plate take their velocities
// for the next drift.
__device__ __forceinline__ void close_boundaries(StageDev& W, double Rc) {
  const long long pq = (long long)atomicExch(&W.plate_q, 0ull);
  const long long tq = (long long)atomicExch(&W.pen_q, 0ull);
  W.plate_q_last = pq;
  W.pen_q_last = tq;
  // the penetrometer's next velocity: up at its speed, down at its speed
  // reduced by the grains' push against the driving force
  if (W.pen_dir > 0) {
    W.v_pen = W.pen_speed;
  } else if (W.pen_dir < 0) {
    double f = 1.0;
    if (W.pen_force > 0.0) {
      f = __dsub_rn(1.0, __ddiv_rn(__dmul_rn((double)tq, 9.094947017729282379150390625e-13), W.pen_force));
      if (f < 0.0) f = 0.0;
      if (f > 1.0) f = 1.0;
    }
    W.v_pen = __dmul_rn(-W.pen_speed, f);
  }
  if (W.plate_mode == 1) {
    const double stress = __ddiv_rn(__dmul_rn((double)pq, 9.094947017729282379150390625e-13),
                                    __dmul_rn(__dmul_rn(3.14159265358979323846, Rc), Rc));
    double v = __dmul_rn(W.plate_gain, __dsub_rn(stress, W.plate_stress));
    if (v > W.plate_vmax) v = W.plate_vmax;
    if (v < -W.plate_vmax) v = -W.plate_vmax;
    W.v_plate = v;
  }
}

// Original-JKR separation test (point S of Fig. 1, the turning point of
// Eq. 13): delta < delta_S = C_S (pi^2 gamma^2 R* / E*^2)^(1/3), C_S =
// 4^(-2/3) - 2 4^(-1/6), cubed as in bond_breaks_exact.
__device__ __forceinline__ bool contact_separates_exact(double delta, double Rs, double Es,
                                                        double gamma) {
  const double KS = -16.654957426838293;  // C_S^3 pi^2
  if (!(delta < 0.0)) return false;
  double lhs = __dmul_rn(__dmul_rn(__dmul_rn(delta, delta), delta), __dmul_rn(Es, Es));
  double rhs = __dmul_rn(__dmul_rn(KS, __dmul_rn(gamma, gamma)), Rs);
  return lhs < rhs;
}

// Touching test of two spheres in IEEE double: d^2 < (Ri + Rj)^2 with the
// squared distance summed x, y, z without contraction.
__device__ __forceinline__ void exact_geometry(const SampleDev& s, double4 a, double4 b,
                                               double* d2_out, double* S_out) {
  double dx = __dsub_rn(b.x, a.x), dy = __dsub_rn(b.y, a.y), dz = __dsub_rn(b.z, a.z);
  if (s.kind == CGDEM_PERIODIC_BOX) {
    dx = min_image(dx, s.L[0]);
    dy = min_image(dy, s.L[1]);
    dz = min_image(dz, s.L[2]);
  }
  *d2_out = __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
  *S_out = __dadd_rn(fabs(a.w), fabs(b.w));
}

__device__ __forceinline__ void latch(Ctl* ctl, unsigned bits) { atomicOr(&ctl->status, bits); }

// A grain of sample s and radius R left through the outlet: its size class
// and its mass rho (4/3 pi) R^3 in fixed-point quanta (integer atomics: the
// sums do not depend on the order of the removals).
__device__ __forceinline__ void record_produced(const Dev& d, const SampleDev& S, int s, double R) {
  if (S.n_psd <= 0) return;
  const double dfine = 2.0 * R / S.k_cg;
  int c = 0;
  while (c + 1 < S.n_psd && !(dfine < S.psd_edge[c + 1])) ++c;
  const double m = S.rho * (4.1887902047863905 * R * R * R);
  const size_t k = (size_t)s * CGDEM_PSD_MAX + c;
  atomicAdd(&d.psd_count[k], 1ull);
  atomicAdd(&d.psd_mass[k], (unsigned long long)__double2ll_rn(m / S.psd_mq));
}

}  // namespace cgdem
